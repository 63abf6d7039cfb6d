"""2-D physical optics over an aperture of rays on the GPU (rtw_field_po2d) against the oracle's
or_field_po2d on the same rays, element by element at the FP64 path's 1e-6 bound: the sphere's
rainbow (order 2, the case pinned by Table 1 and the 1-D PO) and one order of a tilted ellipsoid
away from caustics (the case pinned by the exact ray field); argument checks."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M_WATER = 1.333
LAM = 0.6328


@pytest.fixture(scope="module")
def rtw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_13856_gb300 import build, rtw as R

    build.build()
    R.lib()
    return R


def po2d_gpu(rtw, spec, jones, h, p_max, order, window, axis, cone, dirs):
    g = rtw.Object([rtw.ObjectSpec(**spec, jones=jones)])
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, spacing=h, flags=rtw.RTW_TRACE_APERTURE)
    rays = rtw.rtw_trace(g, tp)
    d = torch.tensor(dirs, dtype=torch.float64, device="cuda")
    out = torch.zeros((len(dirs), 2), dtype=torch.complex128, device="cuda")
    used = rtw.rtw_field_po2d(rays, rtw.po2d_params(order, window, axis, cone), d, out, count=True)
    rtw.rtw_sync_status()
    return out.cpu().numpy(), used, g, tp


@pytest.mark.parametrize("a,h", [(50.0, 0.1), (500.0, 0.25)])
def test_po2d_rainbow_matches_oracle(rtw, oracle_mod, a, h):
    spec = dict(a=a, b=a, c=a, quat=(1.0, 0.0, 0.0, 0.0), m=M_WATER, wavelength=LAM)
    o = oracle_mod.Object(a, a, a, m=M_WATER, wavelength=LAM, jones=(0.0, 1.0))
    Aw, Fw = (LAM / a) ** (2.0 / 3.0), 1.0 / math.sqrt(o.k0 * a)
    thc = math.radians(137.922)
    th = thc + np.linspace(-0.4 * Aw, 1.5 * Aw, 200)
    dirs = np.stack([th, np.zeros_like(th)], 1)
    _, nx, ny, _, _ = o.square_grid(h=h)
    win = [0, nx // 2, 0, ny - 1]
    cone = (3 * Aw + 3 * Fw, 3 * Aw + 6 * Fw)
    got, gused, g, tp = po2d_gpu(rtw, spec, (0.0, 1.0), h, 2, 2, win, (thc, 0.0), cone, dirs)
    assert g.grid(0, tp)[1:] == (nx, ny)
    ref, used = o.field_po2d(2, win, dirs, (thc, 0.0), cone, h=h)
    assert used > 100_000 and gused == used
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    print(f"a = {a}: {used} rays, max |dF| / max |F| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_po2d_ellipsoid_matches_oracle(rtw, oracle_mod):
    """Order 1 of a tilted ellipsoid (elliptical polarisation), 25 directions around one ray, the
    whole grid as the window."""
    quat = (0.9, 0.25, -0.3, 0.15)
    n = math.sqrt(sum(q * q for q in quat))
    quat = tuple(q / n for q in quat)
    spec = dict(a=50.0, b=40.0, c=30.0, quat=quat, m=M_WATER, wavelength=LAM)
    o = oracle_mod.Object(50.0, 40.0, 30.0, quat=quat, m=M_WATER, wavelength=LAM, jones=(0.6, 0.8j))
    h = 0.1
    _, nx, ny, _, _ = o.square_grid(h=h)
    rec, _, hit = o.trace_ray(10.0, 5.0, 1)
    s0 = rec[1, oracle_mod.S:oracle_mod.S + 3]
    th0, ph0 = math.acos(s0[2]), math.atan2(s0[1], s0[0])
    dirs = np.array([[th0 + dt, ph0 + dp] for dt in np.linspace(-0.02, 0.02, 5) for dp in np.linspace(-0.02, 0.02, 5)])
    win = [0, nx - 1, 0, ny - 1]
    got, gused, _, _ = po2d_gpu(rtw, spec, (0.6, 0.8j), h, 1, 1, win, (th0, ph0), (0.2, 0.35), dirs)
    ref, used = o.field_po2d(1, win, dirs, (th0, ph0), (0.2, 0.35), h=h)
    assert gused == used
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    print(f"ellipsoid order 1: {used} rays, max |dF| / max |F| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_po2d_edge_window_and_empty_cone(rtw, oracle_mod):
    """A window on the grid's edge (one-sided differences, rays that miss) matches the oracle; a cone
    that keeps no ray sums nothing."""
    spec = dict(a=10.0, b=10.0, c=10.0, quat=(1.0, 0.0, 0.0, 0.0), m=M_WATER, wavelength=LAM)
    o = oracle_mod.Object(10.0, 10.0, 10.0, m=M_WATER, wavelength=LAM, jones=(0.0, 1.0))
    _, nx, ny, _, _ = o.square_grid(h=0.1)
    dirs = np.array([[2.4, 0.0], [2.41, 0.01], [2.45, -0.02]])
    got, gused, _, _ = po2d_gpu(rtw, spec, (0.0, 1.0), 0.1, 2, 2, [0, 40, 0, ny - 1], (2.4, 0.0), (0.3, 0.5), dirs)
    ref, used = o.field_po2d(2, [0, 40, 0, ny - 1], dirs, (2.4, 0.0), (0.3, 0.5), h=0.1)
    assert used > 1000 and gused == used
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
    got, gused, _, _ = po2d_gpu(rtw, spec, (0.0, 1.0), 0.1, 2, 2, [0, nx - 1, 0, ny - 1], (0.3, 0.0), (0.01, 0.02),
                                dirs)
    assert gused == 0 and np.all(got == 0)


def test_po2d_arguments(rtw):
    spec = dict(a=10.0, b=10.0, c=10.0, quat=(1.0, 0.0, 0.0, 0.0), m=M_WATER, wavelength=LAM)
    g = rtw.Object([rtw.ObjectSpec(**spec)])
    d = torch.tensor([[2.4, 0.0]], dtype=torch.float64, device="cuda")
    out = torch.zeros((1, 2), dtype=torch.complex128, device="cuda")
    plain = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=2, spacing=0.5))
    ok = rtw.po2d_params(2, [0, 10, 0, 10], (2.4, 0.0), (0.1, 0.2))
    with pytest.raises(rtw.RTWError):  # traced without the aperture data
        rtw.rtw_field_po2d(plain, ok, d, out)
    with pytest.raises(rtw.RTWError):  # the mixed trace keeps no aperture data on square grids
        rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=2, spacing=0.5,
                                          precision=rtw.RTW_MIXED, flags=rtw.RTW_TRACE_APERTURE))
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=2, spacing=0.5, flags=rtw.RTW_TRACE_APERTURE)
    rays = rtw.rtw_trace(g, tp)
    _, nx, ny = g.grid(0, tp)
    for bad in (rtw.po2d_params(3, [0, 10, 0, 10], (2.4, 0.0), (0.1, 0.2)),        # order > p_max
                rtw.po2d_params(2, [0, nx, 0, 10], (2.4, 0.0), (0.1, 0.2)),        # beyond the grid
                rtw.po2d_params(2, [5, 6, 0, 10], (2.4, 0.0), (0.1, 0.2)),         # under 3 x 3 vertices
                rtw.po2d_params(2, [0, 10, 0, 10], (2.4, 0.0), (0.2, 0.1))):       # cone_end <= cone_full
        with pytest.raises(rtw.RTWError):
            rtw.rtw_field_po2d(rays, bad, d, out)
    rtw.rtw_field_po2d(rays, ok, d, out)
    rtw.rtw_sync_status()
