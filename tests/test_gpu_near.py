"""The field at finite points (on a sphere |M| = R about the origin) on the GPU against the oracle:
the ray records at the crossing points and the dense-ray field with its three components
(E_r, E_theta, E_phi), element by element at the FP64 path's 1e-6 bound; argument checks."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rtw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_13856_gb300 import build, rtw as R

    build.build()
    R.lib()
    return R


def near_field(rtw, spec, jones, p_max, nt, nph, n_rays, R, precision=0):
    obj = rtw.Object([rtw.ObjectSpec(**spec, jones=jones)])
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays, observe_radius=R,
                          precision=precision)
    rays = rtw.rtw_trace(obj, tp)
    out = torch.zeros((nt * nph, p_max + 1, 3), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    return out.cpu().numpy(), mask.cpu().numpy(), obj, rays


def oracle_object(oracle_mod, spec, jones):
    return oracle_mod.Object(spec["a"], spec["b"], spec["c"], quat=spec["quat"], m=spec["m"],
                             wavelength=spec["wavelength"], jones=jones)


@pytest.mark.parametrize("R", [160.0, 1000.0])
def test_near_field_ellipsoid_matches_oracle(rtw, oracle_mod, R):
    """The tilted ellipsoid (semi-axes 120, 100, 80 um), about 3e4 rays, orders 0..4, on a
    48 x 96 grid of points of the sphere of radius R: masks equal, every component of every point
    and order within 1e-6 of the largest."""
    from paper_2403_13856_gb300 import workloads as W

    jones = (1.0, 0.0)
    p_max, nt, nph = 4, 48, 96
    got, gm, _, _ = near_field(rtw, W.ELLIPSOID, jones, p_max, nt, nph, 30_000, R)
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    ref, rm, hits = o.field_sphere(p_max, nt, nph, R, n_target=30_000)
    ref = oracle_mod.complex_field(ref)
    assert hits > 5000
    assert np.array_equal(gm, rm)
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    radial = np.abs(ref[..., 0]).max() / scale
    print(f"R = {R}: max |dE| / max |E| = {err / scale:.2e}, radial part up to {radial:.2f} of the largest")
    assert scale > 0 and err <= 1e-6 * scale
    assert radial > 1e-3  # the rays through M are not radial at this distance


def test_near_records_match_oracle(rtw, oracle_mod):
    """Per-ray records at the crossing points (direction M / R, field, phase, flags) against the
    oracle's near record of the same rays."""
    from paper_2403_13856_gb300 import workloads as W

    R = 300.0
    p_max = 3
    _, _, obj, rays = near_field(rtw, W.ELLIPSOID, (0.6, 0.8j), p_max, 4, 8, 2_000, R)
    o = oracle_object(oracle_mod, W.ELLIPSOID, (0.6, 0.8j))
    h, nx, ny, xc, yc = o.square_grid(n_target=2_000)
    n = nx * ny
    checked = 0
    for p in range(p_max + 1):
        s = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        F = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
        psi = torch.zeros(n, dtype=torch.float64, device="cuda")
        fl = torch.zeros(n, dtype=torch.int32, device="cuda")
        rtw.rtw_rays_export(rays, p, 0, n, s, F, psi, fl)
        s, F, psi, fl = s.cpu().numpy(), F.cpu().numpy(), psi.cpu().numpy(), fl.cpu().numpy().view(np.uint32)
        for j in range(0, n, 7):
            ix, iy = j % nx, j // nx
            x = xc + (ix + 0.5 - nx // 2) * h
            y = yc + (iy + 0.5 - ny // 2) * h
            rec, _, hit = o.trace_ray(x, y, p_max)
            if not hit or rec[p, oracle_mod.VALID] == 0.0:
                continue
            near, ok = o.near_record(rec[p], R)
            assert ok and (fl[j] & 1)
            assert np.abs(s[j] - near[oracle_mod.S:oracle_mod.S + 3]).max() < 1e-12
            Fr = near[oracle_mod.F:oracle_mod.F + 6]
            assert np.abs(F[j] - Fr).max() <= 1e-9 * np.abs(Fr).max() + 1e-15
            assert abs(psi[j] - near[oracle_mod.PSI]) < 1e-8
            assert ((fl[j] >> 8) & 0xFF) == int(near[oracle_mod.NF])
            assert bool(fl[j] & 2) == (near[oracle_mod.ORIENT] > 0)
            checked += 1
    assert checked > 1000


def test_observe_radius_arguments(rtw):
    from paper_2403_13856_gb300 import workloads as W

    obj = rtw.Object([rtw.ObjectSpec(**W.ELLIPSOID)])
    with pytest.raises(rtw.RTWError):  # inside the object's bounding sphere
        rtw.rtw_trace(obj, rtw.trace_params(n_rays=1000, observe_radius=100.0))
    with pytest.raises(rtw.RTWError):  # fan grids keep the far field
        rtw.rtw_trace(obj, rtw.trace_params(grid=rtw.RTW_GRID_FAN, n_rays=1000, observe_radius=500.0))
    rays = rtw.rtw_trace(obj, rtw.trace_params(n_rays=1000, p_max=1, observe_radius=500.0))
    out = torch.zeros((8 * 16, 2, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(rtw.RTWError):  # Newton solves for far-field directions
        rtw.rtw_field(rays, rtw.dirs_grid(8, 16), out, None, mode=rtw.RTW_NEWTON, flags=rtw.RTW_FIELD_PER_ORDER)


def test_observe_radius_needs_fp64(rtw):
    from paper_2403_13856_gb300 import workloads as W

    obj = rtw.Object([rtw.ObjectSpec(**W.ELLIPSOID)])
    with pytest.raises(rtw.RTWError):
        rtw.rtw_trace(obj, rtw.trace_params(n_rays=1000, observe_radius=500.0, precision=rtw.RTW_MIXED))
