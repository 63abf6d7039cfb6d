"""Batched far field (many ellipsoids, one launch sequence) on the GPU against the FP64 oracle.

Objects come from the batched-drop recipe (uneven size, shape, orientation, index, wavelength);
small batches use the same distributions at reduced radii so that the oracle computes every object,
the full-size batch (4096 objects, about 1.4e9 rays) is checked on sampled objects.  Tolerances
as the single-object grid field: |dF| <= 1e-6 max|F| per object and masks identical (FP64);
the mixed-precision batch is bounded by the normwise error stated in its test.
"""
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


def make_batch(rtw, specs, jones=(1.0, 0.0)):
    return rtw.Object([rtw.ObjectSpec(**s, jones=jones) for s in specs])


def run_batch(rtw, obj, rays, p_max, nt, nph, flags=0, batch=None, out=None, mask=None, **kw):
    nout = p_max + 1 if flags & rtw.RTW_FIELD_PER_ORDER else 1
    n = len(rays)
    if out is None:
        out = torch.zeros((n, nt * nph, nout, 2), dtype=torch.complex128, device="cuda")
        mask = torch.zeros((n, nt * nph), dtype=torch.uint8, device="cuda")
    bp = rtw.batch_params(rays, p_max=p_max, **kw)
    batch = rtw.rtw_far_field_batch(obj, bp, rtw.dirs_grid(nt, nph), out, mask, flags=flags, batch=batch)
    rtw.rtw_sync_status()
    return out, mask, batch


def oracle_field(oracle_mod, spec, jones, p_max, nt, nph, n_rays):
    o = oracle_mod.Object(spec["a"], spec["b"], spec["c"], quat=spec["quat"], m=spec["m"],
                          wavelength=spec["wavelength"], jones=jones)
    ref, rm, hits, _ = o.field_grid(p_max, nt, nph, n_target=int(n_rays))
    return oracle_mod.complex_field(ref), rm


def compare(got, ref, gm, rm, tol=1e-6):
    assert np.array_equal(gm, rm), f"{(gm != rm).sum()} mask entries differ"
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= tol * scale, f"max |dF| {err:.3e} vs scale {scale:.3e}"


SMALL = dict(r0=(3.0, 12.0), rays_ref=(2.0e4, 12.0), rays_clamp=(300, 20_000))


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
def test_batch_small_per_order_vs_oracle(rtw, oracle_mod, variant):
    """12 drops of the batched recipe at radii 3-12 um, orders 0..4 per order, 32 x 64 directions;
    a chunk bound of 6e4 ray-orders splits them into several chunks; every trace variant."""
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(12, **SMALL)
    obj = make_batch(rtw, specs)
    p_max, nt, nph = 4, 32, 64
    out, mask, batch = run_batch(rtw, obj, rays, p_max, nt, nph, flags=rtw.RTW_FIELD_PER_ORDER,
                                 chunk_ray_orders=60_000, trace_variant=variant)
    total, nchunks, _ = batch.info()
    assert nchunks >= 3
    got, gm = out.cpu().numpy(), mask.cpu().numpy()
    for i, s in enumerate(specs):
        ref, rm = oracle_field(oracle_mod, s, (1.0, 0.0), p_max, nt, nph, rays[i])
        compare(got[i], ref, gm[i], rm)


def test_batch_classification_blocks_give_identical_fields(rtw):
    """The classification queues its block's small triangles in shared memory and finishes them after
    a barrier, so the block size changes which thread tests which triangle and the order of the hits,
    never the result: with the hits summed as fixed-point integers the field of every block size the
    autotuner may choose (64, 128, 256 threads) is the same bit for bit, summed and per order, masks
    included."""
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(12, **SMALL)
    obj = make_batch(rtw, specs)
    p_max, nt, nph = 4, 48, 96
    for flags in (0, rtw.RTW_FIELD_PER_ORDER):
        res = [run_batch(rtw, obj, rays, p_max, nt, nph, flags=flags, classify_block=cb)[:2] for cb in (64, 128, 256)]
        out0, mask0 = res[0]
        assert torch.count_nonzero(out0).item() > 1000
        for out, mask in res[1:]:
            assert torch.equal(out.view(torch.int64), out0.view(torch.int64))
            assert torch.equal(mask, mask0)


def test_batch_graph_replay_and_chunking_agree(rtw):
    """Graph replay reproduces the eager run; one chunk and many chunks agree (the same sums in
    another order of atomic additions: relative 1e-12)."""
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(40, **SMALL)
    obj = make_batch(rtw, specs, jones=(0.6, 0.8j))
    p_max, nt, nph = 4, 24, 48
    eager, em, _ = run_batch(rtw, obj, rays, p_max, nt, nph)
    out = torch.zeros_like(eager)
    mask = torch.zeros_like(em)
    b = None
    for k in range(3):
        out.zero_()
        _, _, b = run_batch(rtw, obj, rays, p_max, nt, nph, batch=b, out=out, mask=mask, use_graph=1,
                            chunk_ray_orders=100_000)
        assert b.info()[2] == (k > 0)
        scale = eager.abs().max().item()
        assert (out - eager).abs().max().item() <= 1e-12 * scale
        assert torch.equal(mask, em)


def test_batch_mixed_precision_vs_oracle(rtw, oracle_mod):
    """Mixed precision batch against the FP64 oracle: normwise error per object <= 1e-4, the
    largest error of any direction <= 1e-3 of the object's largest component, identical masks."""
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(8, **SMALL)
    obj = make_batch(rtw, specs)
    p_max, nt, nph = 4, 32, 64
    out, mask, _ = run_batch(rtw, obj, rays, p_max, nt, nph, precision=rtw.RTW_MIXED)
    got, gm = out.cpu().numpy()[:, :, 0], mask.cpu().numpy()
    worst = worst_dir = 0.0
    for i, s in enumerate(specs):
        ref, rm = oracle_field(oracle_mod, s, (1.0, 0.0), p_max, nt, nph, rays[i])
        ref = ref.sum(axis=1)
        assert np.array_equal(gm[i], rm)
        worst = max(worst, np.linalg.norm(got[i] - ref) / np.linalg.norm(ref))
        worst_dir = max(worst_dir, np.abs(got[i] - ref).max() / np.abs(ref).max())
    print(f"mixed batch: worst normwise field error {worst:.2e}, worst direction {worst_dir:.2e} of the largest")
    assert worst <= 1e-4 and worst_dir <= 1e-3


def test_batch_newton_vs_oracle_exact(rtw, oracle_mod):
    """mode RTW_NEWTON in the batch: 6 drops, every hit refined on the exact trace, against the
    oracle's exact branch sum per object."""
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(6, **SMALL)
    obj = make_batch(rtw, specs)
    p_max, nt, nph = 4, 32, 64
    rtw.rtw_newton_failures()
    out, mask, _ = run_batch(rtw, obj, rays, p_max, nt, nph, flags=rtw.RTW_FIELD_PER_ORDER, mode=rtw.RTW_NEWTON)
    gfail = rtw.rtw_newton_failures()
    got, gm = out.cpu().numpy(), mask.cpu().numpy()
    total_fail = 0
    for i, s in enumerate(specs):
        o = oracle_mod.Object(s["a"], s["b"], s["c"], quat=s["quat"], m=s["m"], wavelength=s["wavelength"])
        ref, rm, _, nfail = o.field_grid(p_max, nt, nph, n_target=int(rays[i]), flags=oracle_mod.FIELD_EXACT)
        total_fail += nfail
        compare(got[i], oracle_mod.complex_field(ref), gm[i], rm)
    assert gfail == total_fail


def test_batch_direction_list_vs_oracle(rtw, oracle_mod):
    """The batch on a list of 1500 directions (poles, seam, duplicate included), 5 drops."""
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(5, **SMALL)
    obj = make_batch(rtw, specs)
    g = np.random.default_rng(8)
    dirs = np.concatenate([np.stack([np.arccos(g.uniform(-1, 1, 1494)), g.uniform(-np.pi, np.pi, 1494)], 1),
                           [[0.0, 0.0], [np.pi, 1.0], [1.0, -np.pi], [1.0, np.pi], [2.0, 0.5], [2.0, 0.5]]])
    n = len(dirs)
    out = torch.zeros((5, n, 5, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros((5, n), dtype=torch.uint8, device="cuda")
    bp = rtw.batch_params(rays, p_max=4, chunk_ray_orders=80_000)
    rtw.rtw_far_field_batch(obj, bp, rtw.dirs_list(torch.tensor(dirs).cuda()), out, mask,
                            flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
    got, gm = out.cpu().numpy(), mask.cpu().numpy()
    for i, s in enumerate(specs):
        o = oracle_mod.Object(s["a"], s["b"], s["c"], quat=s["quat"], m=s["m"], wavelength=s["wavelength"])
        ref, rm, _, _ = o.field_dirs(4, dirs, n_target=int(rays[i]))
        compare(got[i], oracle_mod.complex_field(ref), gm[i], rm)


def test_batch_argument_errors(rtw):
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(2, **SMALL)
    obj = make_batch(rtw, specs)
    out = torch.zeros((2, 8 * 16, 1, 2), dtype=torch.complex128, device="cuda")
    d = rtw.dirs_grid(8, 16)
    for kw in [dict(trace_variant=9), dict(classify_block=96), dict(p_max=16), dict(chunk_ray_orders=-1)]:
        args = dict(p_max=4)
        args.update(kw)
        with pytest.raises(rtw.RTWError):
            rtw.rtw_far_field_batch(obj, rtw.batch_params(rays, **args), d, out)
    with pytest.raises(rtw.RTWError):
        rtw.rtw_far_field_batch(obj, rtw.batch_params([0, 100]), d, out)
    with pytest.raises(rtw.RTWError):
        rtw.rtw_far_field_batch(obj, rtw.batch_params(rays), rtw.dirs_grid(8, 16, [0, 4, 0, 4]), out)


def test_batch_full_size_sampled_objects(rtw, oracle_mod):
    """The full batched workload (4096 drops, r0 20-500 um, about 1.4e9 rays, orders 0..4, 128 x 256
    directions each) in the launch configuration the benchmark times (FP64, graph); the fields of
    sampled objects (smallest, median, largest ray count, and two more) against the oracle."""
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.BATCH
    specs, rays = W.batch_objects()
    obj = make_batch(rtw, specs)
    nt, nph = cfg["n_theta"], cfg["n_phi"]
    out, mask, batch = run_batch(rtw, obj, rays, cfg["p_max"], nt, nph, use_graph=1)
    order = np.argsort(rays)
    picks = [order[0], order[len(order) // 2], order[-1], 7, 1000]
    got = out[picks].cpu().numpy()[:, :, 0]
    gm = mask[picks].cpu().numpy()
    for k, i in enumerate(picks):
        ref, rm = oracle_field(oracle_mod, specs[i], (1.0, 0.0), cfg["p_max"], nt, nph, rays[i])
        ref = ref.sum(axis=1)
        assert np.array_equal(gm[k], rm), f"object {i}: {(gm[k] != rm).sum()} mask entries differ"
        scale = np.abs(ref).max()
        err = np.abs(got[k] - ref).max()
        print(f"object {i} ({rays[i]} rays, a={specs[i]['a']:.1f} um): max |dF| / max |F| = {err / scale:.2e}")
        assert err <= 1e-6 * scale


def test_autotuner_on_gpu_picks_valid_options(rtw, tmp_path):
    """The autotuner times every candidate through the library on a sample and caches the choice;
    the tuned options reproduce the default run's field."""
    from paper_2403_13856_gb300 import autotune as A
    from paper_2403_13856_gb300 import workloads as W

    specs, rays = W.batch_objects(24, **SMALL)
    p_max, nt, nph = 4, 32, 64
    path = str(tmp_path / "tune.json")
    best = A.tune(specs, rays, p_max, rtw.RTW_FP64, nt, nph, cache_path=path, budget_ray_orders=200_000, reps=1)
    assert best["trace_variant"] in A.TRACE_VARIANTS and best["classify_block"] in A.CLASSIFY_BLOCKS
    entry = list(A.load(path).values())[0]
    assert all(v > 0 for v in entry["ms"].values())
    obj = make_batch(rtw, specs)
    ref, rm, _ = run_batch(rtw, obj, rays, p_max, nt, nph)
    got, gm, _ = run_batch(rtw, obj, rays, p_max, nt, nph, **best)
    assert torch.equal(gm, rm)
    assert (got - ref).abs().max().item() <= 1e-12 * ref.abs().max().item()
