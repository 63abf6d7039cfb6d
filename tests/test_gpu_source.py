"""A point source as the incident wave on the GPU against the oracle: per-ray records from explicit
grid-plane points, and the dense-ray far field, element by element at the FP64 path's 1e-6 bound;
argument checks of the paths that take plane waves only."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SOURCE = (30.0, -20.0, -400.0)  # off the axis: the grid's plane is tilted against x, y


@pytest.fixture(scope="module")
def rtw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_13856_gb300 import build, rtw as R

    build.build()
    R.lib()
    return R


def objects(rtw, oracle_mod, jones, source=SOURCE):
    from paper_2403_13856_gb300 import workloads as W

    spec = W.ELLIPSOID
    g = rtw.Object([rtw.ObjectSpec(**spec, jones=jones, source=source)])
    o = oracle_mod.Object(spec["a"], spec["b"], spec["c"], quat=spec["quat"], m=spec["m"],
                          wavelength=spec["wavelength"], jones=jones, source=source)
    return g, o


def test_point_source_records_match_oracle(rtw, oracle_mod):
    """Rays toward 400 points of the grid's plane (inside and outside the lit region), orders
    0..3: direction, field, phase and flags against the oracle's rays."""
    g, o = objects(rtw, oracle_mod, (0.6, 0.8j))
    rng = np.random.default_rng(5)
    xy = rng.uniform(-160.0, 160.0, (400, 2))
    n, p_max = len(xy), 3
    s = torch.zeros((n, p_max + 1, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros((n, p_max + 1, 6), dtype=torch.float64, device="cuda")
    psi = torch.zeros((n, p_max + 1), dtype=torch.float64, device="cuda")
    fl = torch.zeros((n, p_max + 1), dtype=torch.int32, device="cuda")
    rtw.rtw_trace_points(g, 0, torch.tensor(xy).cuda(), p_max, s, F, psi, fl)
    torch.cuda.synchronize()
    s, F, psi, fl = s.cpu().numpy(), F.cpu().numpy(), psi.cpu().numpy(), fl.cpu().numpy().view(np.uint32)
    hits = 0
    for j in range(n):
        rec, _, hit = o.trace_ray(xy[j, 0], xy[j, 1], p_max)
        for p in range(p_max + 1):
            valid = hit and rec[p, oracle_mod.VALID] != 0.0
            assert bool(fl[j, p] & 1) == valid, (j, p)
            if not valid:
                continue
            hits += 1
            assert np.abs(s[j, p] - rec[p, oracle_mod.S:oracle_mod.S + 3]).max() < 1e-12
            Fr = rec[p, oracle_mod.F:oracle_mod.F + 6]
            assert np.abs(F[j, p] - Fr).max() <= 1e-9 * np.abs(Fr).max() + 1e-18
            assert abs(psi[j, p] - rec[p, oracle_mod.PSI]) < 1e-8
            assert ((fl[j, p] >> 8) & 0xFF) == int(rec[p, oracle_mod.NF])
            assert bool(fl[j, p] & 2) == (rec[p, oracle_mod.ORIENT] > 0)
            assert bool(fl[j, p] & 4) == (rec[p, oracle_mod.CAUSTIC] != 0.0)
    assert hits > 500


@pytest.mark.parametrize("source", [SOURCE, (0.0, 0.0, -3000.0)])
def test_point_source_field_matches_oracle(rtw, oracle_mod, source):
    """The tilted ellipsoid lit by a point source, about 3e4 rays, orders 0..4, 48 x 96 far-field
    directions: masks equal, every component within 1e-6 of the largest."""
    g, o = objects(rtw, oracle_mod, (1.0, 0.0), source)
    p_max, nt, nph = 4, 48, 96
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=30_000)
    rays = rtw.rtw_trace(g, tp)
    out = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    got, gm = out.cpu().numpy(), mask.cpu().numpy()
    ref, rm, hits, _ = o.field_grid(p_max, nt, nph, n_target=30_000)
    ref = oracle_mod.complex_field(ref)
    assert hits > 5000
    assert np.array_equal(gm, rm), f"{(gm != rm).sum()} mask entries differ"
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    print(f"source {source}: max |dF| / max |F| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_point_source_arguments(rtw, oracle_mod):
    from paper_2403_13856_gb300 import workloads as W

    g, _ = objects(rtw, oracle_mod, (1.0, 0.0))
    with pytest.raises(rtw.RTWError):  # fans stay plane-wave
        rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_FAN, n_rays=1000))
    with pytest.raises(rtw.RTWError):  # double precision only
        rtw.rtw_trace(g, rtw.trace_params(n_rays=1000, precision=rtw.RTW_MIXED))
    with pytest.raises(rtw.RTWError):  # a source inside the drop
        rtw.Object([rtw.ObjectSpec(**W.ELLIPSOID, source=(0.0, 0.0, 10.0))])
    out = torch.zeros((1, 8 * 16, 1, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(rtw.RTWError):  # the batched path takes plane waves
        rtw.rtw_far_field_batch(g, rtw.batch_params(np.array([1000]), p_max=1), rtw.dirs_grid(8, 16), out)


def test_point_source_on_a_sphere_of_points(rtw, oracle_mod):
    """Both extensions together: a point source lighting the drop, the field taken on the sphere
    |M| = 500 um (three components per point), against the oracle's sphere field."""
    g, o = objects(rtw, oracle_mod, (0.0, 1.0), (0.0, 0.0, -600.0))
    p_max, nt, nph, R = 3, 32, 64, 500.0
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=20_000, observe_radius=R)
    rays = rtw.rtw_trace(g, tp)
    out = torch.zeros((nt * nph, p_max + 1, 3), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    ref, rm, hits = o.field_sphere(p_max, nt, nph, R, n_target=20_000)
    ref = oracle_mod.complex_field(ref)
    assert hits > 2000
    assert np.array_equal(mask.cpu().numpy(), rm)
    scale = np.abs(ref).max()
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"point source, sphere of points: max |dE| / max |E| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_point_source_newton_vs_oracle_exact(rtw, oracle_mod):
    """RTW_NEWTON with a point source: every hit (about 1.5e4 rays, orders 0..3, 48 x 96
    directions) replaced by the exact ray found by Newton steps in the grid plane's coordinates;
    against the oracle's exact branch sum on the same hits, the same failures."""
    g, o = objects(rtw, oracle_mod, (1.0, 0.0))
    p_max, nt, nph = 3, 48, 96
    rtw.rtw_newton_failures()
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=15_000))
    out = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, mode=rtw.RTW_NEWTON, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    gfail = rtw.rtw_newton_failures()
    ref, rm, hits, nfail = o.field_grid(p_max, nt, nph, n_target=15_000, flags=oracle_mod.FIELD_EXACT)
    ref = oracle_mod.complex_field(ref)
    print(f"point source Newton: {hits} hits, {nfail} not converged (oracle), {gfail} (GPU)")
    assert hits > 3000 and gfail == nfail
    assert np.array_equal(mask.cpu().numpy(), rm)
    scale = np.abs(ref).max()
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-6 * scale
