"""The oblate spheroid a = b = 100 um, c = 90 um lit along its x axis (the body turned so that the
incident wave travels along +z), against the oracle; and a direction grid fine enough to take the
sliced field run on an ellipsoid, against an unsliced list of the same directions and the oracle."""
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


def test_spheroid_side_lit_matches_oracle(rtw, oracle_mod):
    from paper_2403_13856_gb300 import workloads as W

    sp = dict(W.SPHEROID_SIDE, jones=(0.0, 1.0))
    p_max, nt, nph, n_rays = 5, 96, 192, 30_000
    g = rtw.Object([rtw.ObjectSpec(**sp)])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    out = torch.zeros((nt * nph, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nt * nph, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(nt, nph), out, mask, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    ref, rm, hits, _ = oracle_mod.Object(**sp).field_grid(p_max, nt, nph, n_target=n_rays)
    ref = oracle_mod.complex_field(ref)
    assert hits > 10_000
    assert np.array_equal(mask.cpu().numpy(), rm)
    scale = np.abs(ref).max()
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"side-lit spheroid: max |dF| / max |F| = {err / scale:.2e}")
    assert scale > 0 and err <= 1e-6 * scale


def test_fine_grid_takes_the_sliced_run(rtw, oracle_mod):
    """12000 x 12000 directions and orders 0..5 (four pairs per direction and order would exceed the
    hit list, and the pairs the orders want do: the run is split into row slices): sampled cells of
    the grid field equal the same directions given as a list (an unsliced run) and the oracle's
    field on them, and no capacity error is left behind."""
    from paper_2403_13856_gb300 import workloads as W

    sp = dict(W.ELLIPSOID, jones=(1.0, 0.0))
    p_max, n, n_rays = 5, 12_000, 50_000
    g = rtw.Object([rtw.ObjectSpec(**sp)])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=n_rays))
    out = torch.zeros((n * n, 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_grid(n, n), out, mask)
    rtw.rtw_sync_status()
    rng = np.random.default_rng(21)
    idx = rng.choice(n * n, size=3000, replace=False)
    th = (idx // n + 0.5) * np.pi / n
    ph = -np.pi + (idx % n + 0.5) * 2 * np.pi / n
    dirs = np.stack([th, ph], 1)
    got = out[torch.tensor(idx, device="cuda")].cpu().numpy()[:, 0]
    gm = mask[torch.tensor(idx, device="cuda")].cpu().numpy()
    d = torch.tensor(dirs, dtype=torch.float64, device="cuda")
    out_l = torch.zeros((len(dirs), 1, 2), dtype=torch.complex128, device="cuda")
    mask_l = torch.zeros(len(dirs), dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, rtw.dirs_list(d), out_l, mask_l)
    rtw.rtw_sync_status()
    lst = out_l.cpu().numpy()[:, 0]
    assert np.array_equal(gm, mask_l.cpu().numpy())
    scale = np.abs(lst).max()
    assert scale > 0 and np.abs(got - lst).max() <= 1e-9 * scale
    ref, rm, _, _ = oracle_mod.Object(**sp).field_dirs(p_max, dirs, n_target=n_rays)
    ref = oracle_mod.complex_field(ref).sum(axis=1)
    assert np.array_equal(gm, rm)
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
