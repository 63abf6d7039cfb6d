"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same inputs.

Tolerances (FP64 path): exit directions 1e-12, far-field amplitudes 1e-9 of the largest one,
phases 1e-8 rad (per ray); fields |dF| <= 1e-6 max|F| per direction and order (the relative
amplitude / 1e-6 rad phase bound of the FP64 path), masks identical.
"""
import math

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


def gpu_object(rtw, spec, jones):
    return rtw.Object([rtw.ObjectSpec(**spec, jones=jones)])


def oracle_object(oracle_mod, spec, jones):
    return oracle_mod.Object(spec["a"], spec["b"], spec["c"], quat=spec["quat"], m=spec["m"],
                             wavelength=spec["wavelength"], jones=jones)


def compare_records(oracle_mod, ref, s, F, psi, flags, s_tol=1e-12):
    """ref: oracle records (n, np, NFIELD); s (n, np, 3), F (n, np, 6), psi (n, np), flags (n, np)."""
    valid = ref[..., oracle_mod.VALID] != 0
    assert np.array_equal(valid, (flags & 1) != 0)
    v = valid
    assert np.allclose(s[v], ref[..., oracle_mod.S:oracle_mod.S + 3][v], atol=s_tol, rtol=0)
    Fr = ref[..., oracle_mod.F:oracle_mod.F + 6]
    scale = np.abs(Fr[v]).max()
    assert np.allclose(F[v], Fr[v], atol=1e-9 * scale, rtol=1e-9)
    assert np.allclose(psi[v], ref[..., oracle_mod.PSI][v], atol=1e-8, rtol=0)
    nf = (flags >> 8) & 0xFF
    assert np.array_equal(nf[v], ref[..., oracle_mod.NF][v].astype(np.int64))
    orient = np.where(flags & 2, 1, -1)
    assert np.array_equal(orient[v], ref[..., oracle_mod.ORIENT][v].astype(np.int64))
    caustic = (flags & 4) != 0
    assert np.array_equal(caustic[v], ref[..., oracle_mod.CAUSTIC][v] != 0)


def compare_fields(got, ref, gmask, rmask, tol=1e-6):
    """got, ref: complex (ndir, norders, 2)."""
    assert np.array_equal(gmask, rmask), f"{(gmask != rmask).sum()} mask entries differ"
    scale = np.abs(ref).max()
    assert scale > 0
    err = np.abs(got - ref).max()
    assert err <= tol * scale, f"max |dF| = {err:.3e}, scale {scale:.3e}"
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


# ------------------------------------------------------------------------------------------------
# per-ray parity
# ------------------------------------------------------------------------------------------------

def test_trace_points_ellipsoid(rtw, oracle_mod):
    from paper_2403_13856_gb300 import workloads as W

    jones = (0.6, 0.8j)
    obj = gpu_object(rtw, W.ELLIPSOID, jones)
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    rng = np.random.default_rng(1)
    xy = rng.uniform(-130, 130, size=(4000, 2))
    p_max = 5
    ref = o.trace_rays(xy, p_max)
    n = xy.shape[0]
    d = torch.from_numpy(xy).cuda()
    s = torch.zeros((n, p_max + 1, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros((n, p_max + 1, 6), dtype=torch.float64, device="cuda")
    psi = torch.zeros((n, p_max + 1), dtype=torch.float64, device="cuda")
    fl = torch.zeros((n, p_max + 1), dtype=torch.int32, device="cuda")
    rtw.rtw_trace_points(obj, 0, d, p_max, s, F, psi, fl)
    rtw.rtw_sync_status()
    assert (ref[..., oracle_mod.VALID] != 0).sum() > 10000
    compare_records(oracle_mod, ref, s.cpu().numpy(), F.cpu().numpy(), psi.cpu().numpy(),
                    fl.cpu().numpy().astype(np.int64) & 0xFFFFFFFF)


def export_all(rtw, rays, np_, first, count):
    out = []
    for p in range(np_):
        s = torch.zeros((count, 3), dtype=torch.float64, device="cuda")
        F = torch.zeros((count, 6), dtype=torch.float64, device="cuda")
        psi = torch.zeros(count, dtype=torch.float64, device="cuda")
        fl = torch.zeros(count, dtype=torch.int32, device="cuda")
        rtw.rtw_rays_export(rays, p, first, count, s, F, psi, fl)
        out.append((s.cpu().numpy(), F.cpu().numpy(), psi.cpu().numpy(), fl.cpu().numpy().astype(np.int64) & 0xFFFFFFFF))
    s = np.stack([o[0] for o in out], 1)
    F = np.stack([o[1] for o in out], 1)
    psi = np.stack([o[2] for o in out], 1)
    fl = np.stack([o[3] for o in out], 1)
    return s, F, psi, fl


@pytest.mark.parametrize("jones", [(0.0, 1.0), (1.0, 0.0)])
def test_trace_fan_sphere_full(rtw, oracle_mod, jones):
    """The 1-D sphere workload at full size: 1e4 rays, orders 0..3."""
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.SPHERE10_FAN
    obj = gpu_object(rtw, W.SPHERE10, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_FAN, p_max=cfg["p_max"], n_rays=cfg["n_rays"])
    rays = rtw.rtw_trace(obj, tp)
    R, npo, nob = rays.info()
    assert (R, npo, nob) == (cfg["n_rays"], cfg["p_max"] + 1, 1)
    s, F, psi, fl = export_all(rtw, rays, npo, 0, R)
    rtw.rtw_sync_status()
    o = oracle_object(oracle_mod, W.SPHERE10, jones)
    _, x, y = o.fan_impacts(cfg["n_rays"])
    ref = o.trace_rays(np.stack([x, y], 1), cfg["p_max"])
    compare_records(oracle_mod, ref, s, F, psi, fl)


@pytest.mark.parametrize("jones", [(1.0, 0.0), (0.6, 0.8j)])
def test_trace_double_float_vs_oracle(rtw, oracle_mod, jones):
    """The double-float trace (48-bit significands, positions and path in FP64) per ray against
    the FP64 oracle at the FP64 path's stated bounds: relative amplitude 1e-6 and phase 1e-6 rad
    per (ray, order), directions 1e-10, flags identical; 3000 sampled rays of the tilted
    ellipsoid's 4e5-ray grid, orders 0..5."""
    from paper_2403_13856_gb300 import workloads as W

    obj = gpu_object(rtw, W.ELLIPSOID, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=5, n_rays=400_000, precision=rtw.RTW_DFLOAT)
    rays = rtw.rtw_trace(obj, tp)
    R, npo, _ = rays.info()
    h, nx, ny = obj.grid(0, tp)
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    h2, _, _, xc, yc = o.square_grid(n_target=400_000)
    idx = np.sort(np.random.default_rng(9).choice(R, size=3000, replace=False))
    s, F, psi, fl = export_all(rtw, rays, npo, 0, R)
    ix, iy = idx % nx, idx // nx
    x = xc + (ix + 0.5 - nx // 2) * h2
    y = yc + (iy + 0.5 - ny // 2) * h2
    ref = o.trace_rays(np.stack([x, y], 1), 5)
    inside = (fl[idx, 0] & 1) != 0  # rays outside the projected section are not traced
    ref[~inside] = 0.0
    flags = fl[idx]
    v = ref[..., oracle_mod.VALID] != 0
    assert np.array_equal(v, (flags & 1) != 0)
    assert np.array_equal(flags[v] >> 8 & 0xFF, ref[..., oracle_mod.NF][v].astype(np.int64))
    assert np.abs(s[idx][v] - ref[..., oracle_mod.S:oracle_mod.S + 3][v]).max() <= 1e-10
    Fr = ref[..., oracle_mod.F:oracle_mod.F + 6][v]
    aF = np.linalg.norm(Fr, axis=-1)
    rel = np.linalg.norm(F[idx][v] - Fr, axis=-1) / aF
    dpsi = np.abs(psi[idx][v] - ref[..., oracle_mod.PSI][v])
    print(f"double-float trace: max relative amplitude {rel.max():.1e}, max phase {dpsi.max():.1e} rad")
    assert rel.max() <= 1e-6 and dpsi.max() <= 1e-6
    assert inside.sum() > 1500


def test_field_grid_double_float_vs_oracle(rtw, oracle_mod):
    """The tilted ellipsoid's field from the double-float trace (3e4 rays, orders 0..5) against the
    FP64 oracle at the FP64 field tolerance."""
    from paper_2403_13856_gb300 import workloads as W

    jones = (1.0, 0.0)
    obj = gpu_object(rtw, W.ELLIPSOID, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=5, n_rays=30_000, precision=rtw.RTW_DFLOAT)
    rays = rtw.rtw_trace(obj, tp)
    out = torch.zeros((96 * 192, 6, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(96 * 192, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(96, 192), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    ref, rm, hits, _ = o.field_grid(5, 96, 192, n_target=30_000)
    compare_fields(out.cpu().numpy(), oracle_mod.complex_field(ref), mask.cpu().numpy(), rm)


def test_square_grid_layout(rtw, oracle_mod):
    from paper_2403_13856_gb300 import workloads as W

    obj = gpu_object(rtw, W.ELLIPSOID, (1.0, 0.0))
    o = oracle_object(oracle_mod, W.ELLIPSOID, (1.0, 0.0))
    for n in (1000, 123457, 4_000_000):
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=5, n_rays=n)
        h, nx, ny = obj.grid(0, tp)
        h2, nx2, ny2, _, _ = o.square_grid(n_target=n)
        assert (nx, ny) == (nx2, ny2) and h == pytest.approx(h2, rel=1e-15)


# ------------------------------------------------------------------------------------------------
# field parity
# ------------------------------------------------------------------------------------------------

def fan_field(rtw, spec, jones, nrays, p_max, ndir, alpha0, dalpha, po):
    obj = gpu_object(rtw, spec, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_FAN, p_max=p_max, n_rays=nrays,
                          flags=rtw.RTW_TRACE_APERTURE if po else 0)
    rays = rtw.rtw_trace(obj, tp)
    d = rtw.dirs_plane(ndir, alpha0, dalpha)
    out = torch.zeros((ndir, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(ndir, dtype=torch.uint8, device="cuda")
    flags = rtw.RTW_FIELD_PER_ORDER | (rtw.RTW_FIELD_PO if po else 0)
    rtw.rtw_field(rays, d, out, mask, flags=flags)
    rtw.rtw_sync_status()
    return out.cpu().numpy(), mask.cpu().numpy(), np.array(rtw.plane_angles(d))


@pytest.mark.parametrize("jones", [(0.0, 1.0), (1.0, 0.0)])
@pytest.mark.parametrize("po", [False, True])
def test_field_fan_sphere_full(rtw, oracle_mod, jones, po):
    """The 1-D sphere workload at full size: 1e4 rays, orders 0..3, 1801 angles 0..180 deg."""
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.SPHERE10_FAN
    got, gm, alpha = fan_field(rtw, W.SPHERE10, jones, cfg["n_rays"], cfg["p_max"], cfg["n_dirs"], cfg["alpha0"],
                               cfg["dalpha"], po)
    o = oracle_object(oracle_mod, W.SPHERE10, jones)
    ref, rm = o.field_fan(cfg["n_rays"], alpha, cfg["p_max"], flags=oracle_mod.FIELD_PO if po else 0)
    compare_fields(got, oracle_mod.complex_field(ref), gm, rm)
    if po:
        assert (rm & oracle_mod.MASK_PO).sum() > 100


def test_field_fan_ragged_and_negative_angles(rtw, oracle_mod):
    """Odd ray count, directions on both sides of the axis (alpha < 0 is the half-plane
    phi = fan_phi + pi), an ellipsoid in a principal plane."""
    spec = dict(a=9.0, b=11.0, c=7.5, quat=(1.0, 0.0, 0.0, 0.0), m=1.55, wavelength=0.5)
    got, gm, alpha = fan_field(rtw, spec, (0.3, 0.9), 3331, 4, 997, -math.pi + 0.001, 2 * math.pi / 997, False)
    o = oracle_object(oracle_mod, spec, (0.3, 0.9))
    ref, rm = o.field_fan(3331, alpha, 4)
    compare_fields(got, oracle_mod.complex_field(ref), gm, rm)


def grid_field(rtw, spec, jones, p_max, nt, nph, n_rays=0, spacing=0.0, window=None, mode=0):
    obj = gpu_object(rtw, spec, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays, spacing=spacing)
    rays = rtw.rtw_trace(obj, tp)
    d = rtw.dirs_grid(nt, nph, window)
    out = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, d, out, mask, mode=mode, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    return out.cpu().numpy(), mask.cpu().numpy(), obj, rays


def test_field_grid_ellipsoid_reduced(rtw, oracle_mod):
    """The tilted ellipsoid at reduced size: about 3e4 rays, 96 x 192 directions, orders 0..5."""
    from paper_2403_13856_gb300 import workloads as W

    jones = (1.0, 0.0)
    got, gm, _, _ = grid_field(rtw, W.ELLIPSOID, jones, 5, 96, 192, n_rays=30_000)
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    ref, rm, hits, _ = o.field_grid(5, 96, 192, n_target=30_000)
    assert hits > 10000
    compare_fields(got, oracle_mod.complex_field(ref), gm, rm)


@pytest.mark.parametrize("jones", [(1.0, 0.0), (0.3, 0.7j)])
def test_field_grid_newton_vs_oracle_exact(rtw, oracle_mod, jones):
    """RTW_NEWTON on a square grid: every hit of the tilted ellipsoid (about 2e4 rays, orders
    0..5, 64 x 128 directions) replaced by the exact ray; against the oracle's exact branch sum
    (O3) on the same hits."""
    from paper_2403_13856_gb300 import workloads as W

    rtw.rtw_newton_failures()
    got, gm, _, _ = grid_field(rtw, W.ELLIPSOID, jones, 5, 64, 128, n_rays=20_000, mode=rtw.RTW_NEWTON)
    gfail = rtw.rtw_newton_failures()
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    ref, rm, hits, nfail = o.field_grid(5, 64, 128, n_target=20_000, flags=oracle_mod.FIELD_EXACT)
    print(f"grid Newton: {hits} hits, {nfail} not converged (oracle), {gfail} (GPU)")
    assert hits > 5000 and gfail == nfail
    compare_fields(got, oracle_mod.complex_field(ref), gm, rm)


def test_field_grid_newton_removes_interpolation_error(rtw, oracle_mod):
    """The exact branch sum does not depend on the ray grid: Newton fields from grids of 1e4 and
    4e4 rays agree far better than the interpolated fields do (sphere, orders 0..2)."""
    spec = dict(a=8.0, b=8.0, c=8.0, quat=(1.0, 0.0, 0.0, 0.0), m=1.333, wavelength=0.6328)
    f = {}
    for n in (10_000, 40_000):
        for mode in (rtw.RTW_DENSE, rtw.RTW_NEWTON):
            out, m, _, _ = grid_field(rtw, spec, (1.0, 0.0), 2, 48, 96, n_rays=n, mode=mode)
            f[n, mode] = (out.sum(axis=1), m)
    # directions where the two grids see the same branches (all but a few next to masked cells)
    both = (f[10_000, 0][1] == 0) & (f[40_000, 0][1] == 0)
    d_dense = np.abs(f[10_000, 0][0] - f[40_000, 0][0])[both].max(axis=-1)
    d_newton = np.abs(f[10_000, 1][0] - f[40_000, 1][0])[both].max(axis=-1)
    scale = np.abs(f[40_000, 1][0]).max()
    q_dense, q_newton = np.quantile(d_dense, 0.9) / scale, np.quantile(d_newton, 0.9) / scale
    print(f"grid change 1e4 -> 4e4 rays, 90th percentile |dF| / max|F|: dense {q_dense:.2e}, Newton {q_newton:.2e}")
    assert q_newton < 1e-9 and q_dense > 1e-5


def direction_list(n, seed):
    """n directions uniform on the sphere plus the poles, the phi seam and a duplicate."""
    g = np.random.default_rng(seed)
    z = g.uniform(-1, 1, n)
    th = np.arccos(z)
    ph = g.uniform(-np.pi, np.pi, n)
    extra = np.array([[0.0, 0.0], [np.pi, 1.0], [1.0, -np.pi], [1.0, np.pi], [2.0, 0.5], [2.0, 0.5]])
    return np.concatenate([np.stack([th, ph], 1), extra])


@pytest.mark.parametrize("mode", ["dense", "newton"])
def test_field_direction_list_vs_oracle(rtw, oracle_mod, mode):
    """Arbitrary directions of interest: 3000 directions on the sphere (poles, seam, duplicate)
    for the tilted ellipsoid at about 3e4 rays, orders 0..5, per order."""
    from paper_2403_13856_gb300 import workloads as W

    jones = (1.0, 0.0)
    dirs = direction_list(3000, 5)
    obj = gpu_object(rtw, W.ELLIPSOID, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=5, n_rays=30_000)
    rays = rtw.rtw_trace(obj, tp)
    d = rtw.dirs_list(torch.tensor(dirs).cuda())
    out = torch.zeros((len(dirs), 6, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(len(dirs), dtype=torch.uint8, device="cuda")
    m = rtw.RTW_NEWTON if mode == "newton" else rtw.RTW_DENSE
    rtw.rtw_newton_failures()
    rtw.rtw_field(rays, d, out, mask, mode=m, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    gfail = rtw.rtw_newton_failures()
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    ref, rm, hits, nfail = o.field_dirs(5, dirs, n_target=30_000,
                                        flags=oracle_mod.FIELD_EXACT if mode == "newton" else 0)
    assert hits > 1000 and gfail == nfail
    compare_fields(out.cpu().numpy(), oracle_mod.complex_field(ref), mask.cpu().numpy(), rm)


def test_field_direction_list_equals_grid(rtw):
    """The grid's own directions given as a shuffled list (and a single direction) reproduce the
    grid field."""
    spec = dict(a=6.0, b=5.0, c=4.0, quat=(0.9659258262890683, 0.2588190451025207, 0.0, 0.0), m=1.333,
                wavelength=0.6328)
    nt, nph = 24, 48
    got, gm, obj, rays = grid_field(rtw, spec, (0.0, 1.0), 2, nt, nph, n_rays=20_000)
    th = (np.arange(nt) + 0.5) * np.pi / nt
    ph = -np.pi + (np.arange(nph) + 0.5) * 2 * np.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    dirs = np.stack([T.ravel(), P.ravel()], 1)
    perm = np.random.default_rng(4).permutation(len(dirs))
    out = torch.zeros((len(dirs), 3, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(len(dirs), dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_list(torch.tensor(dirs[perm]).cuda()), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    scale = np.abs(got).max()
    assert np.abs(out.cpu().numpy() - got[perm]).max() <= 1e-12 * scale
    assert np.array_equal(mask.cpu().numpy(), gm[perm])
    k = int(np.argmax(np.abs(got).sum(axis=(1, 2))))
    one = torch.zeros((1, 3, 2), dtype=torch.complex128, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_list(torch.tensor(dirs[k:k + 1]).cuda()), one, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    assert np.abs(one.cpu().numpy()[0] - got[k]).max() <= 1e-12 * scale


def test_field_grid_small_sphere_edge_cases(rtw, oracle_mod):
    """A sphere on a coarse grid (many directions per triangle, poles of the direction grid inside
    triangles) and a ragged direction grid."""
    spec = dict(a=5.0, b=5.0, c=5.0, quat=(1.0, 0.0, 0.0, 0.0), m=1.333, wavelength=0.6328)
    got, gm, _, _ = grid_field(rtw, spec, (0.0, 1.0), 2, 37, 70, spacing=0.37)
    o = oracle_object(oracle_mod, spec, (0.0, 1.0))
    ref, rm, hits, _ = o.field_grid(2, 37, 70, h=0.37)
    compare_fields(got, oracle_mod.complex_field(ref), gm, rm)


def test_field_grid_full_size_windows(rtw, oracle_mod):
    """The full-size ellipsoid workload (4e6 rays, 512 x 1024 directions, orders 0..5), field of
    sampled 40 x 40-cell windows of the ray grid against the oracle on the same windows."""
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.ELLIPSOID_GRID
    jones = (1.0, 0.0)
    obj = gpu_object(rtw, W.ELLIPSOID, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=cfg["p_max"], n_rays=cfg["n_rays"])
    rays = rtw.rtw_trace(obj, tp)
    h, nx, ny = obj.grid(0, tp)
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    nt, nph = cfg["n_theta"], cfg["n_phi"]
    out = torch.zeros((nt * nph, cfg["p_max"] + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    for fx, fy in [(0.5, 0.5), (0.3, 0.62), (0.8, 0.25)]:
        ix0, iy0 = int(fx * nx), int(fy * ny)
        win = [ix0, ix0 + 40, iy0, iy0 + 40]
        rtw.rtw_field(rays, rtw.dirs_grid(nt, nph, win), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
        rtw.rtw_sync_status()
        ref, rm, hits, _ = o.field_grid(cfg["p_max"], nt, nph, n_target=cfg["n_rays"], window=win)
        assert hits > 0
        compare_fields(out.cpu().numpy(), oracle_mod.complex_field(ref), mask.cpu().numpy(), rm)


def test_trace_full_size_sampled_rays(rtw, oracle_mod):
    """Full-size ellipsoid trace: 2000 sampled rays of the 4e6-ray grid against the oracle."""
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.ELLIPSOID_GRID
    jones = (1.0, 0.0)
    obj = gpu_object(rtw, W.ELLIPSOID, jones)
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=cfg["p_max"], n_rays=cfg["n_rays"])
    rays = rtw.rtw_trace(obj, tp)
    R, npo, _ = rays.info()
    h, nx, ny = obj.grid(0, tp)
    assert R == nx * ny
    o = oracle_object(oracle_mod, W.ELLIPSOID, jones)
    h2, nx2, ny2, xc, yc = o.square_grid(n_target=cfg["n_rays"])
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(R, size=2000, replace=False))
    s, F, psi, fl = export_all(rtw, rays, npo, 0, R)
    ix, iy = idx % nx, idx // nx
    x = xc + (ix + 0.5 - nx // 2) * h2
    y = yc + (iy + 0.5 - ny // 2) * h2
    ref = o.trace_rays(np.stack([x, y], 1), cfg["p_max"])
    # rays outside the projected section are not traced
    S = None
    inside = (fl[idx, 0] & 1) != 0
    ref[~inside] = 0.0
    compare_records(oracle_mod, ref, s[idx], F[idx], psi[idx], fl[idx])
    assert inside.sum() > 1000


# ------------------------------------------------------------------------------------------------
# Table 1 on the GPU
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("a,nrays", [(50.0, 8000), (500.0, 40000)])
def test_table1_gpu(rtw, oracle_mod, a, nrays):
    import os

    spec = dict(a=a, b=a, c=a, quat=(1.0, 0.0, 0.0, 0.0), m=1.333, wavelength=0.6328)
    alpha0, dalpha, n = math.radians(137.5), math.radians(0.002), 11750
    got, gm, alpha = fan_field(rtw, spec, (0.0, 1.0), nrays, 2, n, alpha0, dalpha, True)
    I = np.abs(got[:, 2, 1]) ** 2
    pk = []
    for i in range(1, n - 1):
        if I[i] > I[i - 1] and I[i] >= I[i + 1]:
            y0, y1, y2 = I[i - 1], I[i], I[i + 1]
            pk.append(alpha[i] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * dalpha)
    pk = np.degrees(np.array(pk))
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_rainbow_peaks.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            at, K, want = line.split()
            if float(at) == a:
                assert pk[int(K)] == pytest.approx(float(want), abs=0.02)
    o = oracle_object(oracle_mod, spec, (0.0, 1.0))
    ref, rm = o.field_fan(nrays, alpha, 2, flags=oracle_mod.FIELD_PO)
    compare_fields(got, oracle_mod.complex_field(ref), gm, rm)


def test_grid_field_is_reproducible_bit_for_bit(rtw):
    """The grid field sums its contributions as fixed-point integers, whose sum does not depend on
    the order in which the hits arrive: two calls on the same rays give the same doubles bit for
    bit, for the far field (per order and summed) and for the field at finite points."""
    from paper_2403_13856_gb300 import workloads as W

    obj = rtw.Object([rtw.ObjectSpec(**W.ELLIPSOID, jones=(0.6, 0.8j))])
    for radius in (0.0, 1000.0):
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=5, n_rays=200_000, observe_radius=radius)
        rays = rtw.rtw_trace(obj, tp)
        nc = 3 if radius > 0 else 2
        for flags in (0, rtw.RTW_FIELD_PER_ORDER):
            nout = 6 if flags else 1
            outs = []
            for _ in range(2):
                out = torch.zeros((128 * 256, nout, nc), dtype=torch.complex128, device="cuda")
                rtw.rtw_field(rays, rtw.dirs_grid(128, 256), out, flags=flags)
                outs.append(out)
            rtw.rtw_sync_status()
            assert torch.count_nonzero(outs[0]).item() > 1000
            assert torch.equal(outs[0].view(torch.int64), outs[1].view(torch.int64))
