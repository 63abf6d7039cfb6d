"""Host logic of the batched-launch autotuner: search order, cache keys and cache reuse."""
from paper_2403_13856_gb300 import autotune as A


def fake_timer(calls):
    # trace fastest for variant 4 at 0 CTAs/SM, field fastest with 128-thread blocks
    def timer(o):
        calls.append(dict(o))
        tr = 10.0 + abs(o["trace_variant"] - 4) + 0.5 * o["trace_ctas_per_sm"]
        fi = 5.0 + abs(o["classify_block"] - 128) / 64.0
        return tr, fi
    return timer


def test_search_finds_the_best_options():
    calls = []
    best, table = A.search(fake_timer(calls), reps=1)
    assert best == {"trace_variant": 4, "trace_ctas_per_sm": 0, "classify_block": 128}
    assert len(calls) == len(A.TRACE_VARIANTS) * len(A.CTAS_PER_SM) + len(A.CLASSIFY_BLOCKS)
    # the classification candidates run with the best trace options
    assert all(c["trace_variant"] == 4 for c in calls[-len(A.CLASSIFY_BLOCKS):])
    assert table["classify 128"] == 5.0


def test_cache_is_written_and_reused(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []
    kw = dict(p_max=4, precision=0, n_theta=128, n_phi=256, cache_path=path, gpu="GB300|152sm", reps=1)
    best = A.tune(None, [1000, 2000, 3000], timer=fake_timer(calls), **kw)
    n = len(calls)
    again = A.tune(None, [1000, 2000, 3000], timer=fake_timer(calls), **kw)
    assert again == best and len(calls) == n
    # another GPU or another precision is another entry
    A.tune(None, [1000, 2000, 3000], timer=fake_timer(calls), **dict(kw, gpu="other|100sm"))
    assert len(calls) == 2 * n
    assert len(A.load(path)) == 2


def test_keys_and_samples():
    k1 = A.workload_key("g", 4, 0, 128, 256, [1_234_567, 10])
    k2 = A.workload_key("g", 4, 0, 128, 256, [1_230_000, 10])
    assert k1 == k2 and "mixed" in A.workload_key("g", 4, 1, 128, 256, [5])
    idx = A.sample_indices([1000] * 100, 4, 50_000)
    assert idx == list(range(0, 100, 10))
    assert A.sample_indices([10 ** 6] * 3, 4, 10) == [1]
