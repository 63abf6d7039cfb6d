"""Superellipsoids (sum_i |u_i|^(2e) = 1) on the GPU against the oracle: per-ray records of the
square grid, the dense-ray far field element by element at the FP64 path's 1e-6 bound, an object
set that mixes an ellipsoid with superellipsoids, and the argument checks of the paths that take
ellipsoids only."""
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


def spec(e, **kw):
    from paper_2403_13856_gb300 import workloads as W

    d = dict(W.SUPERELLIPSOID)
    d["shape_e"] = e
    d.update(kw)
    return d


@pytest.mark.parametrize("source", [None, (30.0, -20.0, -400.0)])
def test_super_records_match_oracle(rtw, oracle_mod, source):
    """Every third ray of a square grid of about 2e3 rays, orders 0..3: direction, field, phase and
    flags (near-caustic included: the flat faces bring order 0 of a point source near the cap)
    against the oracle's ray at the same grid point."""
    sp = spec(2.0) if source is None else spec(2.0, source=source)
    p_max = 3
    g = rtw.Object([rtw.ObjectSpec(**sp, jones=(0.6, 0.8j))])
    o = oracle_mod.Object(**sp, jones=(0.6, 0.8j))
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=2_000))
    h, nx, ny, xc, yc = o.square_grid(n_target=2_000)
    n = nx * ny
    assert rays.info()[0] == n
    checked = 0
    for p in range(p_max + 1):
        s = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        F = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
        psi = torch.zeros(n, dtype=torch.float64, device="cuda")
        fl = torch.zeros(n, dtype=torch.int32, device="cuda")
        rtw.rtw_rays_export(rays, p, 0, n, s, F, psi, fl)
        s, F, psi, fl = s.cpu().numpy(), F.cpu().numpy(), psi.cpu().numpy(), fl.cpu().numpy().view(np.uint32)
        for j in range(0, n, 3):
            ix, iy = j % nx, j // nx
            x = xc + (ix + 0.5 - nx // 2) * h
            y = yc + (iy + 0.5 - ny // 2) * h
            rec, _, hit = o.trace_ray(x, y, p_max)
            valid = hit and rec[p, oracle_mod.VALID] != 0.0
            # grid points outside the bounding ellipsoid's silhouette are not traced on either side
            if not valid:
                assert not (fl[j] & 1), (p, j)
                continue
            assert fl[j] & 1, (p, j)
            assert np.abs(s[j] - rec[p, oracle_mod.S:oracle_mod.S + 3]).max() < 1e-11
            Fr = rec[p, oracle_mod.F:oracle_mod.F + 6]
            assert np.abs(F[j] - Fr).max() <= 1e-9 * np.abs(Fr).max() + 1e-15
            assert abs(psi[j] - rec[p, oracle_mod.PSI]) < 1e-7
            assert ((fl[j] >> 8) & 0xFF) == int(rec[p, oracle_mod.NF])
            assert bool(fl[j] & 2) == (rec[p, oracle_mod.ORIENT] > 0)
            assert bool(fl[j] & 4) == (rec[p, oracle_mod.CAUSTIC] != 0.0)
            checked += 1
    assert checked > 1000


@pytest.mark.parametrize("e", [1.5, 1.7, 2.0, 4.0, 8.0])
def test_super_field_matches_oracle(rtw, oracle_mod, e):
    """About 3e4 rays, orders 0..4, 48 x 96 far-field directions: masks equal, every component
    within 1e-6 of the largest.  2e = 3, 4, 8, 16 take powers by products, 2e = 3.4 the pow
    function; e = 8 is nearly a box, whose flat faces leave most directions masked as caustic."""
    sp = spec(e)
    p_max, nt, nph = 4, 48, 96
    g = rtw.Object([rtw.ObjectSpec(**sp, jones=(1.0, 0.0))])
    o = oracle_mod.Object(**sp, jones=(1.0, 0.0))
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=30_000))
    out = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    got, gm = out.cpu().numpy(), mask.cpu().numpy()
    ref, rm, hits, _ = o.field_grid(p_max, nt, nph, n_target=30_000)
    ref = oracle_mod.complex_field(ref)
    assert hits > 5000
    # On the nearly flat faces of e = 8 one principal curvature vanishes to rounding: where it is
    # exactly zero on one side and not on the other, the ray is a valid near-caustic ray on both (a
    # flat exit wave is a caustic at infinity), so the masks agree everywhere.
    differ = gm != rm
    assert differ.sum() == 0, f"{differ.sum()} mask entries differ"
    scale = np.abs(ref).max()
    err = np.abs(got - ref)[~differ].max()
    print(f"e = {e}: max |dF| / max |F| = {err / scale:.2e}, {differ.sum()} masks differ")
    assert scale > 0 and err <= 1e-6 * scale


@pytest.mark.parametrize("window", [None, (60, 110, 50, 100)])
def test_super_field_sliced(rtw, oracle_mod, window):
    """e = 4 with orders 0..5 sweeps the sphere about a thousand times (rounded edges fan the rays
    out at every internal reflection), so the (triangle, direction) pairs outgrow the hit list and
    the field is summed over halved slices of ray-grid rows; the sum equals the oracle's, also inside
    a cell window of the ray grid."""
    sp = spec(4.0)
    p_max, nt, nph, n_rays = 5, 48, 96, 20_000
    g = rtw.Object([rtw.ObjectSpec(**sp, jones=(0.0, 1.0))])
    o = oracle_mod.Object(**sp, jones=(0.0, 1.0))
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    out = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph, cell_window=window), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    # a second call starts from the slices that fitted; the sum is the same up to the order
    # of the atomic additions
    out2 = torch.zeros_like(out)
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph, cell_window=window), out2, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    assert (out2 - out).abs().max().item() <= 1e-12 * out.abs().max().item()
    ref, rm, hits, _ = o.field_grid(p_max, nt, nph, n_target=n_rays, window=window)
    ref = oracle_mod.complex_field(ref)
    assert hits > 500
    assert np.array_equal(mask.cpu().numpy(), rm)
    scale = np.abs(ref).max()
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"e = 4, window {window}: max |dF| / max |F| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_super_mixed_object_set(rtw, oracle_mod):
    """An ellipsoid between two superellipsoids in one object set: the set is traced by the
    superellipsoid kernel, in which the ellipsoid keeps its quadric path, so its field equals the
    field of the ellipsoid traced alone bit for bit; the superellipsoids match the oracle."""
    from paper_2403_13856_gb300 import workloads as W

    p_max, nt, nph, n_rays = 3, 32, 64, 12_000
    specs = [spec(2.0, jones=(1.0, 0.0)), dict(W.ELLIPSOID, jones=(1.0, 0.0)),
             spec(3.0, a=60.0, b=50.0, c=70.0, center=(5.0, -3.0, 2.0), jones=(0.0, 1.0))]
    g = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    out = torch.zeros((3, nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros((3, nt * nph), dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    got, gm = out.cpu().numpy(), mask.cpu().numpy()
    g1 = rtw.Object([rtw.ObjectSpec(**specs[1])])
    rays1 = rtw.rtw_trace(g1, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    out1 = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask1 = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays1, rtw.dirs_grid(nt, nph), out1, mask1, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    assert np.array_equal(got[1], out1.cpu().numpy())
    assert np.array_equal(gm[1], mask1.cpu().numpy())
    for k in (0, 2):
        o = oracle_mod.Object(**specs[k])
        ref, rm, hits, _ = o.field_grid(p_max, nt, nph, n_target=n_rays)
        ref = oracle_mod.complex_field(ref)
        assert hits > 2000
        assert np.array_equal(gm[k], rm)
        scale = np.abs(ref).max()
        assert scale > 0 and np.abs(got[k] - ref).max() <= 1e-6 * scale


def test_super_field_direction_list(rtw, oracle_mod):
    """A list of 20000 random directions (binned on the device), orders 0..5 at e = 3, whose pairs
    outgrow the hit list: sliced runs on a list against the oracle's field on the same list."""
    sp = spec(3.0, jones=(0.3, 0.9 + 0.3j))
    p_max, n_rays = 5, 20_000
    rng = np.random.default_rng(12)
    dirs = np.stack([np.arccos(rng.uniform(-1.0, 1.0, 20_000)), rng.uniform(-np.pi, np.pi, 20_000)], 1)
    g = rtw.Object([rtw.ObjectSpec(**sp)])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    d = torch.tensor(dirs, dtype=torch.float64, device="cuda")
    out = torch.zeros((len(dirs), p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(len(dirs), dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_list(d), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    o = oracle_mod.Object(**sp)
    ref, rm, hits, _ = o.field_dirs(p_max, dirs, n_target=n_rays)
    ref = oracle_mod.complex_field(ref)
    assert hits > 5000
    assert np.array_equal(mask.cpu().numpy(), rm)
    scale = np.abs(ref).max()
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"list of 20000 directions, e = 3: max |dF| / max |F| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_super_with_point_source_ellipsoid(rtw, oracle_mod):
    """A superellipsoid beside an ellipsoid lit by a point source, in one object set (the set takes
    the superellipsoid kernel; the point source keeps its own start): both against the oracle."""
    from paper_2403_13856_gb300 import workloads as W

    p_max, nt, nph, n_rays = 3, 32, 64, 12_000
    specs = [spec(2.0, jones=(1.0, 0.0)), dict(W.ELLIPSOID, jones=(0.0, 1.0), source=(30.0, -20.0, -400.0))]
    g = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    out = torch.zeros((2, nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros((2, nt * nph), dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    got, gm = out.cpu().numpy(), mask.cpu().numpy()
    for k in range(2):
        ref, rm, hits, _ = oracle_mod.Object(**specs[k]).field_grid(p_max, nt, nph, n_target=n_rays)
        ref = oracle_mod.complex_field(ref)
        assert hits > 2000
        assert np.array_equal(gm[k], rm)
        scale = np.abs(ref).max()
        assert scale > 0 and np.abs(got[k] - ref).max() <= 1e-6 * scale


def test_super_field_on_a_sphere_of_points(rtw, oracle_mod):
    """The superellipsoid's field at the points of the sphere |M| = 600 um (three components per
    point; the superellipsoid kernel with records at the crossing points) against the oracle."""
    sp = spec(2.0, jones=(0.6, 0.8j))
    p_max, nt, nph, R, n_rays = 3, 32, 64, 600.0, 20_000
    g = rtw.Object([rtw.ObjectSpec(**sp)])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays, observe_radius=R))
    out = torch.zeros((nt * nph, p_max + 1, 3), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    ref, rm, hits = oracle_mod.Object(**sp).field_sphere(p_max, nt, nph, R, n_target=n_rays)
    ref = oracle_mod.complex_field(ref)
    assert hits > 2000
    assert np.array_equal(mask.cpu().numpy(), rm)
    scale = np.abs(ref).max()
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"superellipsoid, sphere of points: max |dE| / max |E| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


@pytest.mark.parametrize("source", [(30.0, -20.0, -400.0), (0.0, 0.0, -3000.0)])
def test_super_point_source_field(rtw, oracle_mod, source):
    """A point source lighting the superellipsoid (e = 2), about 2e4 rays through the source's grid
    plane, orders 0..4, 48 x 96 directions, against the oracle."""
    sp = spec(2.0, jones=(1.0, 0.0), source=source)
    p_max, nt, nph, n_rays = 4, 48, 96, 20_000
    g = rtw.Object([rtw.ObjectSpec(**sp)])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    out = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    ref, rm, hits, _ = oracle_mod.Object(**sp).field_grid(p_max, nt, nph, n_target=n_rays)
    ref = oracle_mod.complex_field(ref)
    assert hits > 3000
    assert np.array_equal(mask.cpu().numpy(), rm)
    scale = np.abs(ref).max()
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"superellipsoid, source {source}: max |dF| / max |F| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_super_arguments(rtw, oracle_mod):
    g = rtw.Object([rtw.ObjectSpec(**spec(2.0))])
    with pytest.raises(rtw.RTWError):  # fans stay ellipsoidal
        rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_FAN, n_rays=1000))
    with pytest.raises(rtw.RTWError):  # double precision only
        rtw.rtw_trace(g, rtw.trace_params(n_rays=1000, precision=rtw.RTW_MIXED))
    with pytest.raises(rtw.RTWError):  # 150 um encloses the semi-axes but not the bounding ellipsoid (158 um)
        rtw.rtw_trace(g, rtw.trace_params(n_rays=1000, observe_radius=150.0))
    with pytest.raises(rtw.RTWError):  # not convex
        rtw.Object([rtw.ObjectSpec(**spec(0.7))])
    with pytest.raises(rtw.RTWError):  # a source outside the body but inside its bounding ellipsoid
        rtw.Object([rtw.ObjectSpec(**spec(2.0, source=(0.0, 0.0, -100.0)))])
    with pytest.raises(rtw.RTWError):
        rtw.rtw_trace_points(g, 0, torch.zeros((4, 2), dtype=torch.float64, device="cuda"), 1)
    rays = rtw.rtw_trace(g, rtw.trace_params(n_rays=1000, p_max=1))
    out = torch.zeros((8 * 16, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(rtw.RTWError):  # dense mode only
        rtw.rtw_field(rays, rtw.dirs_grid(8, 16), out, mode=rtw.RTW_NEWTON, flags=rtw.RTW_FIELD_PER_ORDER)
    outb = torch.zeros((1, 8 * 16, 1, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(rtw.RTWError):  # the batched path takes ellipsoids
        rtw.rtw_far_field_batch(g, rtw.batch_params(np.array([1000]), p_max=1), rtw.dirs_grid(8, 16), outb)


def test_super_full_size_windows(rtw, oracle_mod):
    """The full-size superellipsoid workload (4e6 grid rays, 512 x 1024 directions, orders 0..5):
    field of sampled 40 x 40-cell windows of the ray grid against the oracle on the same windows."""
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.ELLIPSOID_GRID
    sp = dict(W.SUPERELLIPSOID, jones=(1.0, 0.0))
    g = rtw.Object([rtw.ObjectSpec(**sp)])
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=cfg["p_max"], n_rays=cfg["n_rays"])
    rays = rtw.rtw_trace(g, tp)
    h, nx, ny = g.grid(0, tp)
    o = oracle_mod.Object(**sp)
    nt, nph = cfg["n_theta"], cfg["n_phi"]
    out = torch.zeros((nt * nph, cfg["p_max"] + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    for fx, fy in [(0.5, 0.5), (0.3, 0.62), (0.75, 0.3)]:
        ix0, iy0 = int(fx * nx), int(fy * ny)
        win = [ix0, ix0 + 40, iy0, iy0 + 40]
        rtw.rtw_field(rays, rtw.dirs_grid(nt, nph, win), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
        rtw.rtw_sync_status()
        ref, rm, hits, _ = o.field_grid(cfg["p_max"], nt, nph, n_target=cfg["n_rays"], window=win)
        ref = oracle_mod.complex_field(ref)
        assert hits > 0
        assert np.array_equal(mask.cpu().numpy(), rm)
        scale = np.abs(ref).max()
        err = np.abs(out.cpu().numpy() - ref).max()
        print(f"window {win}: {hits} hits, max |dF| / max |F| = {err / scale:.2e}")
        assert scale > 0 and err <= 1e-6 * scale


def test_super_full_size_sampled_rays(rtw, oracle_mod):
    """Full-size superellipsoid trace: 2000 sampled rays of the 4e6-ray grid, orders 0..5, against
    the oracle's rays at the same grid points."""
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.ELLIPSOID_GRID
    sp = dict(W.SUPERELLIPSOID, jones=(1.0, 0.0))
    p_max = cfg["p_max"]
    g = rtw.Object([rtw.ObjectSpec(**sp)])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=cfg["n_rays"]))
    R, npo, _ = rays.info()
    o = oracle_mod.Object(**sp)
    h, nx, ny, xc, yc = o.square_grid(n_target=cfg["n_rays"])
    assert R == nx * ny
    idx = np.sort(np.random.default_rng(8).choice(R, size=2000, replace=False))
    x = xc + (idx % nx + 0.5 - nx // 2) * h
    y = yc + (idx // nx + 0.5 - ny // 2) * h
    ref = o.trace_rays(np.stack([x, y], 1), p_max)
    checked = 0
    for p in range(npo):
        s = torch.zeros((R, 3), dtype=torch.float64, device="cuda")
        F = torch.zeros((R, 6), dtype=torch.float64, device="cuda")
        psi = torch.zeros(R, dtype=torch.float64, device="cuda")
        fl = torch.zeros(R, dtype=torch.int32, device="cuda")
        rtw.rtw_rays_export(rays, p, 0, R, s, F, psi, fl)
        ii = torch.tensor(idx, device="cuda")
        s, F, psi = s[ii].cpu().numpy(), F[ii].cpu().numpy(), psi[ii].cpu().numpy()
        fl = fl[ii].cpu().numpy().view(np.uint32)
        for k in range(len(idx)):
            r = ref[k, p]
            assert bool(fl[k] & 1) == (r[oracle_mod.VALID] != 0.0), (p, k)
            if not fl[k] & 1:
                continue
            assert np.abs(s[k] - r[oracle_mod.S:oracle_mod.S + 3]).max() < 1e-11
            Fr = r[oracle_mod.F:oracle_mod.F + 6]
            assert np.abs(F[k] - Fr).max() <= 1e-9 * np.abs(Fr).max() + 1e-15
            assert abs(psi[k] - r[oracle_mod.PSI]) < 1e-7
            assert ((fl[k] >> 8) & 0xFF) == int(r[oracle_mod.NF])
            assert bool(fl[k] & 2) == (r[oracle_mod.ORIENT] > 0)
            assert bool(fl[k] & 4) == (r[oracle_mod.CAUSTIC] != 0.0)
            checked += 1
    assert checked > 4000
