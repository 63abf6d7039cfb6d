"""Autotuner of the batched far field (rtw_far_field_batch).

Searches the launch shapes that the library exposes as options: the persistent trace kernel's
variant (block size and register cap, template instances 1..5) with its resident CTAs per SM, and
the block size of the grid classification kernel.  Each candidate is timed by the library itself
(CUDA events around the trace and the field of every chunk, ``timing = 1``) on an evenly spaced
sample of the batch's objects; the trace and the field are tuned one after the other since they
are separate kernels.  Results are kept in a JSON cache keyed by the GPU and the workload's shape,
so that a later run of the same workload on the same kind of GPU skips the search.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, Optional, Sequence, Tuple

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache", "autotune.json")

TRACE_VARIANTS = (1, 2, 3, 4, 5)
CTAS_PER_SM = (0, 1, 2)
CLASSIFY_BLOCKS = (64, 128, 256)
DEFAULT = {"trace_variant": 2, "trace_ctas_per_sm": 0, "classify_block": 256}


def workload_key(gpu: str, p_max: int, precision: int, n_theta: int, n_phi: int, rays: Sequence[int]) -> str:
    """Cache key: GPU name, orders, precision, direction grid, object count and total rays (to 2
    significant digits, so that seeds of the same recipe share an entry)."""
    total = int(sum(int(r) for r in rays))
    mag = 10 ** max(0, int(math.log10(max(total, 1))) - 1)
    return (f"{gpu}|p{p_max}|{'mixed' if precision else 'fp64'}|{n_theta}x{n_phi}|{len(rays)}obj|"
            f"{round(total / mag) * mag}rays")


def sample_indices(rays: Sequence[int], p_max: int, budget_ray_orders: int) -> list:
    """Evenly spaced objects whose (ray, order) pairs add up to about the budget (at least one)."""
    n = len(rays)
    total = sum(int(r) for r in rays) * (p_max + 1)
    step = max(1, int(math.ceil(total / max(budget_ray_orders, 1))))
    return list(range(0, n, step)) if step < n else [n // 2]


def load(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(path: str, cache: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def search(timer: Callable[[dict], Tuple[float, float]], reps: int = 2) -> Tuple[dict, dict]:
    """Coordinate search: the trace options first (field options at their defaults), then the
    classification block with the best trace options.  timer(options) -> (trace_ms, field_ms).
    Returns the best options and the measured table."""
    table = {}

    def best_of(opts):
        t = [timer(opts) for _ in range(reps)]
        return min(x[0] for x in t), min(x[1] for x in t)

    best = dict(DEFAULT)
    best_trace = None
    for v in TRACE_VARIANTS:
        for c in CTAS_PER_SM:
            opts = dict(best, trace_variant=v, trace_ctas_per_sm=c)
            tr, fi = best_of(opts)
            table[f"trace v{v} ctas{c}"] = tr
            if best_trace is None or tr < best_trace:
                best_trace = tr
                best.update(trace_variant=v, trace_ctas_per_sm=c)
    best_field = None
    for cb in CLASSIFY_BLOCKS:
        opts = dict(best, classify_block=cb)
        tr, fi = best_of(opts)
        table[f"classify {cb}"] = fi
        if best_field is None or fi < best_field:
            best_field = fi
            best["classify_block"] = cb
    return best, table


def tune(specs, rays, p_max: int, precision: int, n_theta: int, n_phi: int, jones=(1.0, 0.0),
         cache_path: Optional[str] = CACHE, budget_ray_orders: int = 1 << 27, reps: int = 2, gpu: Optional[str] = None,
         timer: Optional[Callable[[dict], Tuple[float, float]]] = None, force: bool = False) -> dict:
    """Best launch options for this batch on this GPU (from the cache when present).  `timer`
    replaces the library timing (tests of the search on a host without a GPU)."""
    if gpu is None:
        import torch

        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        gpu = f"{p.name}|{p.multi_processor_count}sm"
    key = workload_key(gpu, p_max, precision, n_theta, n_phi, rays)
    cache = load(cache_path) if cache_path else {}
    if not force and key in cache:
        return dict(cache[key]["options"])
    if timer is None:
        timer = _library_timer(specs, rays, p_max, precision, n_theta, n_phi, jones, budget_ray_orders)
    best, table = search(timer, reps)
    if cache_path:
        cache = load(cache_path)
        cache[key] = {"options": best, "ms": table}
        store(cache_path, cache)
    return best


def _library_timer(specs, rays, p_max, precision, n_theta, n_phi, jones, budget_ray_orders):
    import torch

    from . import rtw

    idx = sample_indices(rays, p_max, budget_ray_orders)
    obj = rtw.Object([rtw.ObjectSpec(**specs[i], jones=jones) for i in idx])
    sub = [int(rays[i]) for i in idx]
    dirs = rtw.dirs_grid(n_theta, n_phi)
    out = torch.empty((len(idx), n_theta * n_phi, 1, 2), dtype=torch.complex128, device="cuda")
    batch = rtw.Batch()

    def timer(opts):
        bp = rtw.batch_params(sub, p_max=p_max, precision=precision, timing=1, **opts)
        rtw.rtw_far_field_batch(obj, bp, dirs, out, batch=batch)
        t = batch.times()
        rtw.rtw_sync_status()
        return t

    timer(dict(DEFAULT))  # first call allocates
    return timer
