"""Benchmark of the RTW far-field hot path on GB300 (one JSON line on rank 0).

Workload: the tilted ellipsoidal water drop, semi-axes (120, 100, 80) um rotated 20 deg about x,
m = 1.333, lambda = 0.6328 um, x polarisation, orders p = 0..5, about 4e6 rays on a square grid
over the projected cross-section, 3-D far field on 512 x 1024 (theta, phi) directions, FP64.
A step is one pass of the whole path: rtw_trace (all rays, all orders) + rtw_field (binning,
interpolation, superposition, singularity mask).  value = rays*interfaces / s (interactions
computed per second over the step); directions/s is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own copy of the workload (independent problems, weak
scaling, no data-path collective); rank 0 prints value = all ranks' units / max time.
The reference arm (--impl reference) times the FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays·interfaces/s and far-field directions/s on 1 GB300 at stated error vs FP64"
UNIT = "rays*interfaces/s"
# FP64 flops of one interaction of the trace kernel (both outgoing waves and one far-field record),
# counted from its source: adds, multiplies, divisions and square roots as one, FMA as two
KERNEL_FLOPS_PER_INTERACTION = 430


def _oracle_flops():
    """The algorithmic flops of one interaction: the operations the oracle's trace executes per
    interaction on the benchmark ellipsoid, counted by its counting build and stored by the test
    suite's script (tests/golden/oracle_flops_per_interaction.json)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_flops_per_interaction.json")) as f:
            return float(json.load(f)["flops_per_interaction"]), "oracle operation count (counting build, stored)"
    except (OSError, KeyError, ValueError):
        return float(KERNEL_FLOPS_PER_INTERACTION), "hand count of the kernel source (stored oracle count missing)"
FP64_NOMINAL_GFLOPS = 1250.0
# DRAM bytes (read + write) of one trace_kernel_fp64 launch on the ellipsoid workload at 4e6 rays
# (ncu: 6.68 MB + 3.18 GB, the ray-state write)
TRACE_TRAFFIC_BYTES = 6_674_944 + 3_180_807_168
TRACE_TRAFFIC_NOTE = "DRAM bytes of one launch at 4e6 rays (ncu); profiles/trace_kernel_fp64_ellipsoid_4e6rays.md"
# FP64 flops the kernel executes per interaction (ncu: DFMA x 2 + DMUL + DADD over the interactions)
EXECUTED_FLOPS_PER_INTERACTION = 407
FLOPS_PER_INTERACTION, FLOPS_SOURCE = _oracle_flops()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-systems", action="store_true",
                    help="ellipsoid line: leave out the batched (4096 drops) and learned (1024 drops) entries")
    ap.add_argument("--cpu-sample-rows", type=int, default=0)
    ap.add_argument("--workload", default="ellipsoid", choices=["ellipsoid", "batch", "learned"],
                    help="ellipsoid: the single tilted drop (default); batch: 4096 seed-drawn drops; "
                         "learned: learned proposals vs dense tracing on 1024 drops")
    ap.add_argument("--retrain", action="store_true", help="learned workload: train even if a checkpoint exists")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "dfloat"], help="batch workload only")
    ap.add_argument("--no-tune", action="store_true", help="batch workload: default launch options")
    args = ap.parse_args()
    if args.workload == "batch" and args.steps == 50:
        args.steps = 5  # a batch step takes seconds
    if args.workload == "learned" and args.steps == 50:
        args.steps, args.warmup = 1, 1  # a learned step takes tens of seconds
    return args


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(dist, x: float) -> float:
    """The largest x over the ranks of the process group (the slowest rank's time); the tensor
    lives where the backend wants it (CUDA for NCCL, host memory for gloo)."""
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank: float, steps: int, world: int, slowest_s: float) -> float:
    """Weak scaling: every rank runs its own copy of the workload, so the job processed world x
    units per step; the rate divides by the slowest rank's time."""
    return world * units_per_rank * steps / slowest_s


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp64_peak_gflops(torch):
    """Measured double-precision throughput of this GPU: cuBLAS DGEMM 4096^3, best of 5."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e9


def pipe_peaks(torch, rtw, local):
    """Throughput of the FP64 (DFMA) and FP32 (FFMA, packed FFMA2) pipes of this GPU, measured with
    the library's dependency-free FMA chain kernels (rtw_pipe_peak), best of 5 launches of about
    50 ms each timed with CUDA events; the SM clock is sampled while they run."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    with ClockSampler(local) as clk:
        for name, kind, iters in (("fp64", rtw.RTW_PEAK_FP64, 1600), ("fp32", rtw.RTW_PEAK_FP32, 100_000),
                                  ("fp32x2", rtw.RTW_PEAK_FP32X2, 50_000)):
            rtw.rtw_pipe_peak(kind, max(1, iters // 20), 4, sink, stream)
            best = 1e30
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                flops = rtw.rtw_pipe_peak(kind, iters, 4, sink, stream)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            res[name] = flops / best / 1e9
    c = clk.summary()
    return {"fp64_gflops": res["fp64"], "fp32_gflops": max(res["fp32"], res["fp32x2"]),
            "fp32_scalar_gflops": res["fp32"], "fp32x2_gflops": res["fp32x2"], "sm_mhz": c.get("sm_mhz"),
            "how": "rtw_pipe_peak: 8 independent FMA chains per thread, 4 blocks of 256 per SM, best of 5"}


def cpu_baseline(rows: int, single_thread_rows: int = 0):
    """The FP64 oracle on a band of `rows` rows of cells of the same ray grid (all columns, all
    orders, same direction grid; rows <= 0: every row, the whole workload), OpenMP over the host's
    cores."""
    import oracle
    from paper_2403_13856_gb300 import workloads as W

    oracle.build()
    spec, cfg = W.ELLIPSOID, W.ELLIPSOID_GRID
    o = oracle.Object(spec["a"], spec["b"], spec["c"], quat=spec["quat"], m=spec["m"], wavelength=spec["wavelength"],
                      jones=(1.0, 0.0))
    h, nx, ny, xc, yc = o.square_grid(n_target=cfg["n_rays"])
    if rows <= 0 or rows >= ny - 1:
        rows = ny - 1
    iy0 = ny // 2 - rows // 2 if rows < ny - 1 else 0
    win = [0, nx - 1, iy0, iy0 + rows]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    out, mask, hits, _ = o.field_grid(cfg["p_max"], cfg["n_theta"], cfg["n_phi"], n_target=cfg["n_rays"],
                                      window=win, threads=cores)
    dt = time.perf_counter() - t0
    # rays of the band that hit the object, times the interactions traced per ray
    import numpy as np

    ys = yc + (np.arange(iy0, iy0 + rows + 1) + 0.5 - ny // 2) * h
    xs = xc + (np.arange(nx) + 0.5 - nx // 2) * h
    X, Y = np.meshgrid(xs, ys)
    rec = o.trace_rays(np.stack([X.ravel(), Y.ravel()], 1), 0, threads=cores)
    nhit = int((rec[:, 0, oracle.VALID] != 0).sum())
    units = nhit * (cfg["p_max"] + 1)
    line = {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{rows + 1} of {ny} grid rows ({nhit} rays), all {cfg['p_max'] + 1} orders, "
                      f"{cfg['n_theta']}x{cfg['n_phi']} directions, trace + field, {dt:.1f} s"}
    if single_thread_rows > 0:
        # the same oracle on one thread, on a central band of rows (bounded to a few seconds)
        r1 = min(single_thread_rows, ny - 1)
        j0 = ny // 2 - r1 // 2
        t1 = time.perf_counter()
        o.field_grid(cfg["p_max"], cfg["n_theta"], cfg["n_phi"], n_target=cfg["n_rays"], window=[0, nx - 1, j0, j0 + r1],
                     threads=1)
        d1 = time.perf_counter() - t1
        ys1 = yc + (np.arange(j0, j0 + r1 + 1) + 0.5 - ny // 2) * h
        X1, Y1 = np.meshgrid(xs, ys1)
        rec1 = o.trace_rays(np.stack([X1.ravel(), Y1.ravel()], 1), 0, threads=cores)
        n1 = int((rec1[:, 0, oracle.VALID] != 0).sum())
        line["single_thread"] = {"value": n1 * (cfg["p_max"] + 1) / d1, "unit": UNIT, "cores": 1,
                                 "sample": f"{r1 + 1} central grid rows ({n1} rays), {d1:.1f} s"}
    return line


def reference_arm(args, rank, world):
    """--impl reference: the oracle, bounded sample per step, on rank 0 only."""
    if rank != 0:
        return
    if args.workload == "batch":
        return reference_arm_batch(args, world)
    rows = args.cpu_sample_rows or 200
    for _ in range(args.warmup):
        cpu_baseline(max(2, rows // 4))
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(rows))
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ellipsoid (120,100,80) um tilt 20 deg, m=1.333, lambda=0.6328 um, p=0..5, "
                               "4e6 rays, 512x1024 directions; oracle on a band of grid rows",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                         "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_arm_batch(args, world):
    for _ in range(args.warmup):
        cpu_baseline_batch(every=1024)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline_batch())
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "4096 seed-drawn drops, p=0..4, 128x256 directions each; oracle on every 256th object",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                         "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch

    from paper_2403_13856_gb300 import build as B
    from paper_2403_13856_gb300 import rtw

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    rtw.lib()
    if args.workload == "batch":
        return bench_batch(args, rank, world, local, dist)
    if args.workload == "learned":
        return bench_learned(args, rank, world, local, dist)
    return bench_ellipsoid(args, rank, world, local, dist)


def timed_on(torch, stream, fn, steps, warmup):
    """mean seconds of fn over steps calls after warmup calls, CUDA events on stream"""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3 / steps


def system_batch(torch, rtw, precision, steps=2, warmup=1):
    """The 4096-drop batched form (one graph-replayed call per step, autotuned launch options):
    rays*interfaces/s, seconds per step and the trace / field split."""
    from paper_2403_13856_gb300 import autotune
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.BATCH
    p_max, nt, nph = cfg["p_max"], cfg["n_theta"], cfg["n_phi"]
    specs, rays = W.batch_objects()
    n = len(specs)
    stream = torch.cuda.current_stream()
    opts = autotune.tune(specs, rays, p_max, precision, nt, nph)
    obj = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
    dirs = rtw.dirs_grid(nt, nph)
    out = torch.empty((n, nt * nph, 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.empty((n, nt * nph), dtype=torch.uint8, device="cuda")
    units = sum(batch_hits(rtw, torch, specs, rays, stream)) * (p_max + 1)
    bp = rtw.batch_params(rays, p_max=p_max, precision=precision, use_graph=1, **opts)
    batch = rtw.rtw_far_field_batch(obj, bp, dirs, out, mask, stream=stream)
    t = timed_on(torch, stream, lambda: rtw.rtw_far_field_batch(obj, bp, dirs, out, mask, batch=batch, stream=stream),
                 steps, warmup)
    rtw.rtw_sync_status(stream)
    bpt = rtw.batch_params(rays, p_max=p_max, precision=precision, timing=1, **opts)
    tb = rtw.rtw_far_field_batch(obj, bpt, dirs, out, mask, stream=stream)
    t_trace, t_field = tb.times()
    total_rays, nchunks, _ = batch.info()
    del tb, batch, out, mask
    return {"value": units / t, "unit": UNIT, "s_per_step": t, "ms_trace": t_trace, "ms_field": t_field,
            "directions_per_s": n * nt * nph / t, "objects": n, "rays_grid": total_rays, "chunks": nchunks,
            "launch_options": opts, "steps": steps, "warmup": warmup}


def precision_errors(torch, rtw, ref_rays, rays, dirs, nt, nph, p_max):
    """Per-order errors of a field summed from rays traced in another precision against the FP64 one
    on the same (theta, phi) grid.  Directions compared: the FP64 field of the order at least 1e-3 of
    its largest, and the direction and its eight neighbours (phi periodic) unmasked and reached by the
    order in both fields -- the edge of an order's support, where one triangle more or less covers a
    direction, and the cells next to caustics are left out.  Reported per order: the directions
    compared and left out, the median, 99.9th percentile and largest relative amplitude error
    | |F| - |F_64| | / |F_64| and phase error |arg(F . conj(F_64))| (rad), and the directions above
    1e-2 in either (directions where the order's branches nearly cancel, or whose triangles hold a ray
    whose focal line lies at an interface, where single precision loses the digits of det(I + d Q), or
    that took a different caustic decision in the two precisions); and the largest |F - F_64| /
    max |F_64| of the order over the directions compared and over every direction unmasked in both
    (normwise; the second includes the edges of the support), with the number of directions unmasked
    in both where |F - F_64| exceeds 1e-3 max |F_64| (on the ellipsoid workload a handful, where the
    two precisions' triangles cover a direction differently: the edge of an order's image, or of one
    branch of it, whose rim triangles map very different directions)."""
    ndir = nt * nph
    outs = []
    for r in (ref_rays, rays):
        o = torch.zeros((ndir, p_max + 1, 2), dtype=torch.complex128, device="cuda")
        m = torch.zeros(ndir, dtype=torch.uint8, device="cuda")
        rtw.rtw_field(r, dirs, o, m, flags=rtw.RTW_FIELD_PER_ORDER)
        outs.append((o, m))
    torch.cuda.synchronize()
    (f64, m64), (fx, mx) = outs

    def all_neighbours(good):
        g = good.reshape(nt, nph)
        pad = torch.nn.functional.pad(g[None, None].float(), (0, 0, 1, 1), value=1.0)[0, 0] > 0
        acc = g.clone()
        for di in (-1, 0, 1):
            rows = pad[1 + di:1 + di + nt]
            for dj in (-1, 0, 1):
                acc &= torch.roll(rows, shifts=dj, dims=1)
        return acc.reshape(-1)

    unmasked = (m64 == 0) & (mx == 0)
    res = []
    for p in range(p_max + 1):
        a = f64[:, p].abs().pow(2).sum(-1).sqrt()
        b = fx[:, p].abs().pow(2).sum(-1).sqrt()
        big = a >= 1e-3 * a.max()
        keep = big & all_neighbours(unmasked & (a > 0) & (b > 0))
        rel = ((b - a).abs() / a)[keep]
        ph = torch.angle((fx[:, p] * f64[:, p].conj()).sum(-1))[keep].abs()
        dF = (fx[:, p] - f64[:, p]).abs().pow(2).sum(-1).sqrt()
        amax = float(a.max().item())
        e = {"order": p, "directions": int(keep.sum().item()), "left_out": int((big & ~keep).sum().item()),
             "normwise_max": float(dF[unmasked].max().item()) / amax if amax > 0 and bool(unmasked.any()) else None,
             "normwise_interior": float(dF[keep].max().item()) / amax if amax > 0 and bool(keep.any()) else None,
             "dF_above_1e-3_max": int((unmasked & big & (dF > 1e-3 * amax)).sum().item())}
        if rel.numel():
            q = torch.tensor([0.5, 0.999], dtype=torch.float64, device=rel.device)
            ra, pa = torch.quantile(rel, q).tolist(), torch.quantile(ph, q).tolist()
            e.update({"rel_amplitude": {"median": ra[0], "q999": ra[1], "max": float(rel.max().item())},
                      "phase_rad": {"median": pa[0], "q999": pa[1], "max": float(ph.max().item())},
                      "above_1e-2": int(((rel > 1e-2) | (ph > 1e-2)).sum().item())})
        res.append(e)
    return res


def caustic_forms(torch, rtw, W, stream):
    """The 2-D physical optics at the 3-D caustics (rtw_field_caustic, default widths, 16 x 16 tiles,
    summed orders) on the drop of the headline workload and on the Fig. 3 spheroid at 0.1 deg: time of
    the corrected field against the plain one on the same rays (traced with the aperture records), and
    the directions masked as caustic before and after."""
    res = {}
    cases = (("ellipsoid_512x1024", W.ELLIPSOID, W.ELLIPSOID_GRID, 512, 1024, (1.0, 0.0),
              "ellipsoid (120,100,80) um tilt 20 deg about x, 4e6 rays, p=0..5, 512x1024 directions"),
             ("spheroid_1800x3600", W.SPHEROID_SIDE, W.SPHEROID_PATTERN, 1800, 3600, (0.0, 1.0),
              "oblate spheroid a=b=100, c=90 um along its x axis, 4e6 rays, p=0..5, 1800x3600 = 0.1 deg"))
    for name, spec, cfg, nt, nph, jv, desc in cases:
        obj = rtw.Object([rtw.ObjectSpec(**spec, jones=jv)])
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=cfg["p_max"], n_rays=cfg["n_rays"],
                              flags=rtw.RTW_TRACE_APERTURE)
        rays = rtw.rtw_trace(obj, tp, stream=stream)
        nd = nt * nph
        d = rtw.dirs_grid(nt, nph)
        out = torch.zeros((nd, 1, 2), dtype=torch.complex128, device="cuda")
        m0 = torch.zeros(nd, dtype=torch.uint8, device="cuda")
        m1 = torch.zeros(nd, dtype=torch.uint8, device="cuda")
        cp = rtw.caustic_params()
        rtw.rtw_field(rays, d, out, m0, stream=stream)
        rtw.rtw_field_caustic(rays, d, cp, out, m1, stream=stream)  # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        rtw.rtw_field(rays, d, out, m0, stream=stream)
        ev[1].record(stream)
        for _ in range(2):
            rtw.rtw_field_caustic(rays, d, cp, out, m1, stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        rtw.rtw_sync_status(stream)
        res[name] = {"workload": desc + ", FP64 trace with aperture records",
                     "ms_field": ev[0].elapsed_time(ev[1]), "ms_field_caustic": ev[1].elapsed_time(ev[2]) / 2,
                     "masked_caustic_before": float(((m0 & 1) != 0).float().mean().item()),
                     "masked_caustic_after": float(((m1 & 1) != 0).float().mean().item()),
                     "corrected_fraction": float(((m1 & 4) != 0).float().mean().item()),
                     "note": "orders 1..5 corrected; caustic directions left after are those of order 0"}
        del rays, out, m0, m1
    return res


def bench_ellipsoid(args, rank, world, local, dist):
    import torch

    from paper_2403_13856_gb300 import rtw
    from paper_2403_13856_gb300 import workloads as W

    spec, cfg = W.ELLIPSOID, W.ELLIPSOID_GRID
    p_max, nt, nph = cfg["p_max"], cfg["n_theta"], cfg["n_phi"]
    obj = rtw.Object([rtw.ObjectSpec(**spec, jones=(1.0, 0.0))])
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=cfg["n_rays"])
    dirs = rtw.dirs_grid(nt, nph)
    ndir = nt * nph
    stream = torch.cuda.current_stream()
    out = torch.zeros((ndir, 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(ndir, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rays = rtw.rtw_trace(obj, tp, stream=stream)
    R, npo, _ = rays.info()
    # units: interactions traced = (p_max + 1) per ray that hits the object
    fl = torch.zeros(R, dtype=torch.int32, device="cuda")
    rtw.rtw_rays_export(rays, 0, 0, R, flags=fl)
    n_hit = int(((fl & 1) != 0).sum().item())
    units = n_hit * (p_max + 1)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        rtw.rtw_trace(obj, tp, rays, stream=stream)
        if ev:
            ev[1].record(stream)
        rtw.rtw_field(rays, dirs, out, mask)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    rtw.rtw_sync_status(stream)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()  # L2 flush between steps, outside the timed events
            step(evs[k])
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    rtw.rtw_sync_status(stream)
    t_step = [e[0].elapsed_time(e[2]) / 1e3 for e in evs]
    t_trace = [e[0].elapsed_time(e[1]) / 1e3 for e in evs]
    t_field = [e[1].elapsed_time(e[2]) / 1e3 for e in evs]
    total = sum(t_step)
    if dist:
        total = max_over_ranks(dist, total)
    value = whole_job_rate(units, args.steps, world, total)
    dps = whole_job_rate(ndir, args.steps, world, total)

    # the other precisions of the trace on the same step (secondary numbers; the line's value is
    # FP64): mixed (1e-4 amplitude, 1e-5 rad phase per ray) and double-float (within the FP64
    # path's 1e-6 bounds)
    forms = {}
    for name, prec in (("mixed", rtw.RTW_MIXED), ("double_float", rtw.RTW_DFLOAT)):
        tpf = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=cfg["n_rays"], precision=prec)
        rf = rtw.rtw_trace(obj, tpf, stream=stream)
        for _ in range(3):
            rtw.rtw_trace(obj, tpf, rf, stream=stream)
            rtw.rtw_field(rf, dirs, out, mask)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(10)]
        for e in ev:
            flush.zero_()
            e[0].record(stream)
            rtw.rtw_trace(obj, tpf, rf, stream=stream)
            e[1].record(stream)
            rtw.rtw_field(rf, dirs, out, mask)
            e[2].record(stream)
        torch.cuda.synchronize()
        tt = statistics.median([e[0].elapsed_time(e[1]) for e in ev])
        ts = statistics.median([e[0].elapsed_time(e[2]) for e in ev])
        forms[name] = {"value": units / (ts / 1e3), "ms_per_step": ts, "ms_trace": tt}
        if name == "mixed":
            forms[name]["errors_per_order"] = precision_errors(torch, rtw, rays, rf, dirs, nt, nph, p_max)
        del rf
    rtw.rtw_sync_status(stream)

    def timed_trace_field(o, tpx, rx, outx, reps=10):
        """median ms of (trace, trace + field) over reps steps after 3 warm-up steps, L2 flushed"""
        for _ in range(3):
            rtw.rtw_trace(o, tpx, rx, stream=stream)
            rtw.rtw_field(rx, dirs, outx, mask)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(reps)]
        for e in ev:
            flush.zero_()
            e[0].record(stream)
            rtw.rtw_trace(o, tpx, rx, stream=stream)
            e[1].record(stream)
            rtw.rtw_field(rx, dirs, outx, mask)
            e[2].record(stream)
        torch.cuda.synchronize()
        rtw.rtw_sync_status(stream)
        return (statistics.median([e[0].elapsed_time(e[1]) for e in ev]),
                statistics.median([e[0].elapsed_time(e[2]) for e in ev]))

    def hit_units(rx):
        flx = torch.zeros(rx.info()[0], dtype=torch.int32, device="cuda")
        rtw.rtw_rays_export(rx, 0, 0, rx.info()[0], flags=flx)
        return int(((flx & 1) != 0).sum().item()) * (p_max + 1)

    # the field at finite points: the same rays recorded where they cross the sphere |M| = 1000 um
    # (about 8 semi-axes), the same 512 x 1024 grid of points on it, three components per point
    near_r = 1000.0
    tpn = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=cfg["n_rays"], observe_radius=near_r)
    rn = rtw.rtw_trace(obj, tpn, stream=stream)
    outn = torch.zeros((ndir, 1, 3), dtype=torch.complex128, device="cuda")
    tt, ts = timed_trace_field(obj, tpn, rn, outn)
    near = {"radius_um": near_r, "value": units / (ts / 1e3), "unit": UNIT, "ms_per_step": ts, "ms_trace": tt,
            "ms_field": ts - tt, "points_per_s": ndir / (ts / 1e3), "kernel": "trace_kernel_fp64_near"}
    del rn, outn

    # an incident wave that is not plane: a point source 1000 um below the centre, rays through the
    # same number of grid points of the plane through the centre, the same far-field grid
    objs = rtw.Object([rtw.ObjectSpec(**spec, jones=(1.0, 0.0), source=(0.0, 0.0, -1000.0))])
    rs = rtw.rtw_trace(objs, tp, stream=stream)
    units_s = hit_units(rs)
    tt, ts = timed_trace_field(objs, tp, rs, out)
    point = {"source_um": [0.0, 0.0, -1000.0], "value": units_s / (ts / 1e3), "unit": UNIT, "ms_per_step": ts,
             "ms_trace": tt, "ms_field": ts - tt}
    del rs, objs

    # another smooth convex body: the superellipsoid |u|^4 + |v|^4 + |w|^4 = 1 on the same semi-axes,
    # turned about all three axes, 4e6 rays over the bounding ellipsoid's silhouette, the same grid
    obje = rtw.Object([rtw.ObjectSpec(**W.SUPERELLIPSOID, jones=(1.0, 0.0))])
    re_ = rtw.rtw_trace(obje, tp, stream=stream)
    units_e = hit_units(re_)
    tt, ts = timed_trace_field(obje, tp, re_, out)
    superellipsoid = {"shape_e": W.SUPERELLIPSOID["shape_e"], "value": units_e / (ts / 1e3), "unit": UNIT,
                      "ms_per_step": ts, "ms_trace": tt, "ms_field": ts - tt, "rays_hit": units_e // (p_max + 1),
                      "kernel": "trace_kernel_fp64_super"}
    del re_, obje

    # 2-D physical optics at the rainbow of a 500 um sphere (order 2, perpendicular polarisation):
    # 4002 x 4002 grid rays traced with the aperture data, the left half as the window, rays tapered
    # like the 1-D window (3 Airy + 3 Fresnel widths, to zero at + 6), 64 x 64 directions around the bow
    a_s = 500.0
    sph = rtw.Object([rtw.ObjectSpec(a=a_s, b=a_s, c=a_s, quat=(1.0, 0.0, 0.0, 0.0), m=W.WATER, wavelength=W.HE_NE,
                                     jones=(0.0, 1.0))])
    tpa = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=2, spacing=0.25, flags=rtw.RTW_TRACE_APERTURE)
    ra = rtw.rtw_trace(sph, tpa, stream=stream)
    _, nxa, nya = sph.grid(0, tpa)
    k0s = 2.0 * math.pi / W.HE_NE
    aw, fw, thc = (W.HE_NE / a_s) ** (2.0 / 3.0), 1.0 / math.sqrt(k0s * a_s), math.radians(137.922)
    tg, pg = torch.meshgrid(thc + torch.linspace(-0.4 * aw, 1.5 * aw, 64, dtype=torch.float64),
                            torch.linspace(-math.radians(2.0), math.radians(2.0), 64, dtype=torch.float64), indexing="ij")
    dirs_po = torch.stack([tg.reshape(-1), pg.reshape(-1)], 1).cuda()
    out_po = torch.zeros((dirs_po.shape[0], 2), dtype=torch.complex128, device="cuda")
    pp = rtw.po2d_params(2, [0, nxa // 2, 0, nya - 1], (thc, 0.0), (3 * aw + 3 * fw, 3 * aw + 6 * fw))
    used_po = rtw.rtw_field_po2d(ra, pp, dirs_po, out_po, count=True, stream=stream)
    for _ in range(3):
        rtw.rtw_trace(sph, tpa, ra, stream=stream)
        rtw.rtw_field_po2d(ra, pp, dirs_po, out_po, stream=stream)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(5)]
    for e in ev:
        flush.zero_()
        e[0].record(stream)
        rtw.rtw_trace(sph, tpa, ra, stream=stream)
        e[1].record(stream)
        rtw.rtw_field_po2d(ra, pp, dirs_po, out_po, stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    rtw.rtw_sync_status(stream)
    tt = statistics.median([e[0].elapsed_time(e[1]) for e in ev])
    tpo = statistics.median([e[1].elapsed_time(e[2]) for e in ev])
    po2d = {"sphere_um": a_s, "grid_rays": nxa * nya, "rays_in_sum": used_po, "directions": int(dirs_po.shape[0]),
            "ms_trace_aperture": tt, "ms_po2d": tpo, "terms_per_s": used_po * dirs_po.shape[0] / (tpo / 1e3),
            "kernel": "po2d_sum_kernel (FP64: one sincos per ray-direction term)"}
    del ra, sph, out_po, dirs_po

    # the 10 um sphere (W1): a fan of 1e4 rays, orders 0..3, 1801 in-plane angles, s and p polarisation;
    # too small to fill the GPU (launch and latency bound), timed over 50 steps of both polarisations
    c1 = W.SPHERE10_FAN
    fans = [rtw.Object([rtw.ObjectSpec(**W.SPHERE10, jones=jv)]) for jv in ((0.0, 1.0), (1.0, 0.0))]
    tpf = rtw.trace_params(grid=rtw.RTW_GRID_FAN, p_max=c1["p_max"], n_rays=c1["n_rays"])
    dpl = rtw.dirs_plane(c1["n_dirs"], c1["alpha0"], c1["dalpha"])
    rf1 = [rtw.rtw_trace(f, tpf, stream=stream) for f in fans]
    outf = torch.zeros((c1["n_dirs"], 1, 2), dtype=torch.complex128, device="cuda")
    for _ in range(5):
        for f, r in zip(fans, rf1):
            rtw.rtw_trace(f, tpf, r, stream=stream)
            rtw.rtw_field(r, dpl, outf, stream=stream)
    e1a, e1b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e1a.record(stream)
    for _ in range(50):
        for f, r in zip(fans, rf1):
            rtw.rtw_trace(f, tpf, r, stream=stream)
            rtw.rtw_field(r, dpl, outf, stream=stream)
    e1b.record(stream)
    torch.cuda.synchronize()
    rtw.rtw_sync_status(stream)
    us1 = 1e3 * e1a.elapsed_time(e1b) / 100  # per polarisation
    flf = torch.zeros(c1["n_rays"], dtype=torch.int32, device="cuda")
    rtw.rtw_rays_export(rf1[0], 0, 0, c1["n_rays"], flags=flf)
    units1 = int(((flf & 1) != 0).sum().item()) * (c1["p_max"] + 1)
    sphere_fan = {"workload": "sphere a=10 um, m=1.333, fan of 1e4 rays, p=0..3, 1801 angles, s and p, FP64",
                  "us_per_step": us1, "value": units1 / (us1 / 1e6), "unit": UNIT,
                  "directions_per_s": c1["n_dirs"] / (us1 / 1e6)}
    del rf1, fans

    # the paper's Fig. 3 setting: the oblate spheroid a = b = 100, c = 90 um lit along its x axis, its
    # whole 3-D pattern at 0.01 deg (18000 x 36000 directions), 4e6 rays, orders 0..5 (the paper's
    # own timing of this pattern, 9.4 min on a desktop CPU with an unstated ray count, is context)
    cf = W.SPHEROID_PATTERN
    sph3 = rtw.Object([rtw.ObjectSpec(**W.SPHEROID_SIDE, jones=(0.0, 1.0))])
    tp3 = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=cf["p_max"], n_rays=cf["n_rays"])
    r3 = rtw.rtw_trace(sph3, tp3, stream=stream)
    nd3 = cf["n_theta"] * cf["n_phi"]
    out3 = torch.zeros((nd3, 1, 2), dtype=torch.complex128, device="cuda")
    mask3 = torch.zeros(nd3, dtype=torch.uint8, device="cuda")
    dirs3 = rtw.dirs_grid(cf["n_theta"], cf["n_phi"])
    rtw.rtw_trace(sph3, tp3, r3, stream=stream)
    rtw.rtw_field(r3, dirs3, out3, mask3, stream=stream)  # warm-up (also finds the slice height)
    ev3 = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(2)]
    for e in ev3:
        e[0].record(stream)
        rtw.rtw_trace(sph3, tp3, r3, stream=stream)
        e[1].record(stream)
        rtw.rtw_field(r3, dirs3, out3, mask3, stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    rtw.rtw_sync_status(stream)
    t3 = statistics.median([e[0].elapsed_time(e[2]) for e in ev3])
    fig3 = {"workload": "oblate spheroid a=b=100, c=90 um, m=1.333, incidence along its x axis, 4e6 rays, "
                        "p=0..5, 18000x36000 (theta,phi) = 0.01 deg over the whole sphere, FP64",
            "s_per_pattern": t3 / 1e3, "ms_trace": statistics.median([e[0].elapsed_time(e[1]) for e in ev3]),
            "directions_per_s": nd3 / (t3 / 1e3), "masked_fraction": float((mask3 != 0).float().mean().item()),
            "paper_context": "9.4 min for this pattern on an Intel i9-13900KS (CPU, ray count not stated)"}
    del r3, out3, mask3, sph3

    caustics = caustic_forms(torch, rtw, W, stream)

    # the system forms on their own workloads: 4096 drops batched (FP64 and mixed), and the learned
    # proposal on 1024 drops against dense tracing
    systems = {}
    if not args.no_systems:
        systems["batch_4096_drops"] = {"fp64": system_batch(torch, rtw, rtw.RTW_FP64),
                                       "mixed": system_batch(torch, rtw, rtw.RTW_MIXED)}
        systems["learned_1024_drops"] = system_learned(torch, rtw, args, local)

    # end to end through the public API: host descriptor in, field copied to pinned host memory
    host_out = torch.empty((ndir, 1, 2), dtype=torch.complex128, pin_memory=True)
    host_mask = torch.empty(ndir, dtype=torch.uint8, pin_memory=True)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        o2 = rtw.Object([rtw.ObjectSpec(**spec, jones=(1.0, 0.0))])
        rtw.rtw_trace(o2, tp, rays, stream=stream)
        rtw.rtw_field(rays, dirs, out, mask)
        host_out.copy_(out, non_blocking=True)
        host_mask.copy_(mask, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    h2d = 464  # the object table entry uploaded by rtw_trace (sizeof(ObjDev))
    d2h = host_out.numel() * 16 + host_mask.numel()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    pipes = pipe_peaks(torch, rtw, local)
    fp64_dgemm = fp64_peak_gflops(torch)
    tr = statistics.median(t_trace)
    tf = statistics.median(t_field)
    achieved = FLOPS_PER_INTERACTION * units / tr / 1e9
    peak = pipes["fp64_gflops"]
    clocks = clk.summary()
    # the field's algorithmic bytes: the ray state it reads once (the 64-byte single-precision field
    # record of every (ray, order) that hit) and the complex128 grid it writes
    field_bytes = units * 64 + ndir * 32
    hbm = peaks.get("hbm_gbs")
    mixed_tr = forms["mixed"]["ms_trace"] / 1e3
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        # default: the whole workload on every core (about 1 s on 16 cores), and one thread on 150 rows
        cpu = cpu_baseline(args.cpu_sample_rows, single_thread_rows=150)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ellipsoid (120,100,80) um tilt 20 deg about x, m=1.333, lambda=0.6328 um, "
                               "x-pol, p=0..5, 4e6 rays square grid, 512x1024 (theta,phi) directions, FP64",
                   "rays_grid": R, "rays_hit": n_hit, "directions": ndir,
                   "l2": "flushed (256 MB write) between timed steps; ray state 2.6 GB > L2"},
        "directions_per_s": dps,
        "ms_trace": 1e3 * tr, "ms_field": 1e3 * statistics.median(t_field),
        # per step: trace_kernel_fp64, dir_tables_kernel, grid_cells_kernel, field_grid_kernel,
        # field_grid_big_kernel, hit_sum_kernel, tile_convert_kernel, finalize_mask_kernel
        "gpu_launches": 8 * args.steps, "gpu_launches_per_step": 8,
        "roofline": {"kernel": "trace_kernel_fp64", "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "GFLOP/s FP64", "frac": achieved / peak,
                     "peak_source": f"measured: DFMA chains (rtw_pipe_peak) at {pipes['sm_mhz']} MHz; "
                                    f"cuBLAS DGEMM 4096^3 {fp64_dgemm:.0f}; nominal {FP64_NOMINAL_GFLOPS:.0f}",
                     "flops_per_interaction": FLOPS_PER_INTERACTION, "flops_source": FLOPS_SOURCE,
                     "frac_executed": EXECUTED_FLOPS_PER_INTERACTION * units / tr / 1e9 / peak,
                     "executed_flops_per_interaction": EXECUTED_FLOPS_PER_INTERACTION,
                     "note": "the oracle's operation count per interaction (760) exceeds what the kernel "
                             "executes (407: two reciprocals where the oracle divides, reduced reflection and "
                             "transmission forms), so the algorithmic rate passes the DFMA-chain peak; the FP64 "
                             "pipe is 87.6 % busy (ncu)",
                     "traffic": TRACE_TRAFFIC_BYTES, "traffic_note": TRACE_TRAFFIC_NOTE},
        "roofline_field": {"kernels": "field_grid_kernel, field_grid_big_kernel, hit_sum_kernel, tile_convert_kernel",
                           "bound": "hbm", "achieved": field_bytes / tf / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": (field_bytes / tf / 1e9 / hbm) if hbm else None, "bytes": field_bytes,
                           "bytes_note": "the ray state read once (the 64-byte field record of every hit ray and "
                                         "order) + the complex128 grid written; the classification is "
                                         "instruction-bound (profiles/field_kernels_ellipsoid_4e6rays.md)"},
        "roofline_mixed": {"kernel": "trace_kernel_mixed", "bound": "alu",
                           "achieved": FLOPS_PER_INTERACTION * units / mixed_tr / 1e9,
                           "peak": pipes["fp32_gflops"], "unit": "GFLOP/s FP32",
                           "frac": FLOPS_PER_INTERACTION * units / mixed_tr / 1e9 / pipes["fp32_gflops"],
                           "note": "the same algorithmic flops as the FP64 trace over the mixed trace's time, "
                                   "against the FP32 pipe (the larger of FFMA and packed FFMA2); the kernel is "
                                   "bound by its residual double-precision work instead (FP64 pipe 86.5 % busy, "
                                   "profiles/trace_kernel_mixed_ellipsoid_1e6rays.md)"},
        "pipe_peaks": pipes,
        "e2e": {"value": units / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
        "precision_forms": forms,
        "near_field": near,
        "point_source": point,
        "superellipsoid": superellipsoid,
        "po2d_rainbow": po2d,
        "paper_fig3_pattern": fig3,
        "caustic_po": caustics,
        "sphere_fan": sphere_fan,
    }
    line.update(systems)
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batch_hits(rtw, torch, specs, rays, stream):
    """Rays of every object's square grid that hit it (order-0 valid flags of a p = 0 trace)."""
    hits = []
    for spec, n in zip(specs, rays):
        o = rtw.Object([rtw.ObjectSpec(**spec)])
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=0, n_rays=int(n))
        r = rtw.rtw_trace(o, tp, stream=stream)
        R, _, _ = r.info()
        fl = torch.empty(R, dtype=torch.int32, device="cuda")
        rtw.rtw_rays_export(r, 0, 0, R, flags=fl, stream=stream)
        hits.append(((fl & 1) != 0).sum())
        del r, o
    return [int(h.item()) for h in hits]


def cpu_baseline_batch(every: int = 256):
    """The FP64 oracle on every `every`-th object of the batched workload (trace + field, all
    orders, the same direction grid), OpenMP over the host's cores."""
    import numpy as np

    import oracle
    from paper_2403_13856_gb300 import workloads as W

    oracle.build()
    cfg = W.BATCH
    specs, rays = W.batch_objects()
    cores = os.cpu_count() or 1
    idx = list(range(0, len(specs), every))
    units, dt = 0, 0.0
    for i in idx:
        s = specs[i]
        o = oracle.Object(s["a"], s["b"], s["c"], quat=s["quat"], m=s["m"], wavelength=s["wavelength"])
        t0 = time.perf_counter()
        o.field_grid(cfg["p_max"], cfg["n_theta"], cfg["n_phi"], n_target=int(rays[i]), threads=cores)
        dt += time.perf_counter() - t0
        h, nx, ny, xc, yc = o.square_grid(n_target=int(rays[i]))
        xs = xc + (np.arange(nx) + 0.5 - nx / 2) * h
        ys = yc + (np.arange(ny) + 0.5 - ny / 2) * h
        X, Y = np.meshgrid(xs, ys)
        rec = o.trace_rays(np.stack([X.ravel(), Y.ravel()], 1), 0, threads=cores)
        units += int((rec[:, 0, oracle.VALID] != 0).sum()) * (cfg["p_max"] + 1)
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} of {len(specs)} objects (every {every}th, {sum(int(rays[i]) for i in idx)} target "
                      f"rays), all {cfg['p_max'] + 1} orders, {cfg['n_theta']}x{cfg['n_phi']} directions, "
                      f"trace + field, {dt:.1f} s"}


def bench_batch(args, rank, world, local, dist):
    """4096 seed-drawn drops in one batched call per step (graph replay, autotuned options)."""
    import torch

    from paper_2403_13856_gb300 import autotune
    from paper_2403_13856_gb300 import rtw
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.BATCH
    p_max, nt, nph = cfg["p_max"], cfg["n_theta"], cfg["n_phi"]
    precision = {"mixed": rtw.RTW_MIXED, "dfloat": rtw.RTW_DFLOAT}.get(args.precision, rtw.RTW_FP64)
    specs, rays = W.batch_objects()
    n = len(specs)
    ndir = nt * nph
    stream = torch.cuda.current_stream()
    opts = dict(autotune.DEFAULT) if args.no_tune else autotune.tune(specs, rays, p_max, precision, nt, nph)
    obj = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
    dirs = rtw.dirs_grid(nt, nph)
    out = torch.empty((n, ndir, 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.empty((n, ndir), dtype=torch.uint8, device="cuda")
    hits = batch_hits(rtw, torch, specs, rays, stream)
    units = sum(hits) * (p_max + 1)
    bp = rtw.batch_params(rays, p_max=p_max, precision=precision, use_graph=1, **opts)
    batch = rtw.rtw_far_field_batch(obj, bp, dirs, out, mask, stream=stream)
    for _ in range(args.warmup):
        rtw.rtw_far_field_batch(obj, bp, dirs, out, mask, batch=batch, stream=stream)
    rtw.rtw_sync_status(stream)
    total_rays, nchunks, replayed = batch.info()
    assert replayed
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            evs[k][0].record(stream)
            rtw.rtw_far_field_batch(obj, bp, dirs, out, mask, batch=batch, stream=stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    rtw.rtw_sync_status(stream)
    t_step = [e[0].elapsed_time(e[1]) / 1e3 for e in evs]
    total = sum(t_step)
    if dist:
        total = max_over_ranks(dist, total)
    value = whole_job_rate(units, args.steps, world, total)
    dps = whole_job_rate(n * ndir, args.steps, world, total)

    # trace and field split: one eager run with the library's own events (same options)
    bpt = rtw.batch_params(rays, p_max=p_max, precision=precision, timing=1, **opts)
    tb = rtw.rtw_far_field_batch(obj, bpt, dirs, out, mask, stream=stream)
    t_trace, t_field = tb.times()
    del tb

    # end to end through the public API: host descriptors in (object table uploaded by the eager
    # call), every object's field copied to pinned host memory
    host_out = torch.empty((n, ndir, 1, 2), dtype=torch.complex128, pin_memory=True)
    host_mask = torch.empty((n, ndir), dtype=torch.uint8, pin_memory=True)
    bpe = rtw.batch_params(rays, p_max=p_max, precision=precision, **opts)
    e2e_steps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        o2 = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
        rtw.rtw_far_field_batch(o2, bpe, dirs, out, mask, batch=batch, stream=stream)
        host_out.copy_(out, non_blocking=True)
        host_mask.copy_(mask, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    h2d = 464 * n  # the object table (464-byte entries)
    d2h = host_out.numel() * 16 + host_mask.numel()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    pipes = pipe_peaks(torch, rtw, local)
    achieved = FLOPS_PER_INTERACTION * units / (t_trace / 1e3) / 1e9
    pk = pipes["fp64_gflops"] if precision == rtw.RTW_FP64 else pipes["fp32_gflops"]
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_batch()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {rtw.RTW_FP64: "f64", rtw.RTW_MIXED: "f32+f64"}.get(precision, "f32x2+f64"), "data": "synthetic",
        "config": {"workload": "4096 drops: r0 U[20,500] um, b,c = r0 U[0.8,1.2], uniform orientation, "
                               "m U[1.33,1.55], lambda U[0.4,0.8] um, x-pol, rays clamp(1e6 (r0/500)^2, 1e3, 1e6), "
                               f"p=0..4, 128x256 (theta,phi) directions each, {args.precision}",
                   "objects": n, "rays_grid": total_rays, "rays_hit": sum(hits), "chunks": nchunks,
                   "launch_options": opts, "graph": True,
                   "l2": "inputs larger than L2 (ray state of a chunk up to 62 GB, output 4.3 GB)"},
        "directions_per_s": dps,
        "ms_trace": t_trace, "ms_field": t_field,
        # per call: dir_tables_kernel, then per chunk (one launch group each at these sizes)
        # trace_items_kernel, grid_cells_kernel, field_grid_kernel, field_grid_big_kernel,
        # hit_sum_kernel, tile_convert_kernel, finalize_mask_kernel
        "gpu_launches_per_step": 1 + nchunks * 7,
        "roofline": {"kernel": "trace_items_kernel", "bound": "alu", "achieved": achieved, "peak": pk,
                     "unit": "GFLOP/s " + ("FP64" if precision == rtw.RTW_FP64 else "FP32"),
                     "frac": achieved / pk,
                     "peak_source": f"measured: FMA chains (rtw_pipe_peak) at {pipes['sm_mhz']} MHz",
                     "flops_per_interaction": FLOPS_PER_INTERACTION, "flops_source": FLOPS_SOURCE,
                     "traffic": None},
        "pipe_peaks": pipes,
        "e2e": {"value": units / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
    }
    if precision != rtw.RTW_FP64:
        line["roofline"]["note"] = "mixed: the algorithmic flops of the FP64 trace against the FP32 pipe"
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def field_errors(torch, got, ref, gmask, rmask):
    """Per-direction errors of a summed field against a reference on the directions unmasked in
    both whose reference intensity exceeds 1e-3 of its object's largest: fraction within 1e-3
    relative intensity and 1e-3 rad phase (dominant component), normwise error."""
    g = got[:, :, 0, :]
    r = ref[:, :, 0, :]
    ir = (r.abs() ** 2).sum(-1)
    ig = (g.abs() ** 2).sum(-1)
    sel = (gmask == 0) & (rmask == 0) & (ir > 1e-3 * ir.amax(dim=1, keepdim=True))
    k = r.abs().argmax(-1, keepdim=True)
    ph = torch.angle(torch.gather(g, -1, k) / torch.gather(r, -1, k))[..., 0].abs()
    rel = (ig - ir).abs() / ir.clamp_min(1e-300)
    ok = sel & (rel <= 1e-3) & (ph <= 1e-3)
    nsel = int(sel.sum().item())
    d = (g - r)[sel]
    return {"directions": nsel, "within_1e-3": int(ok.sum().item()) / max(nsel, 1),
            "normwise": float((d.abs() ** 2).sum().sqrt() / (r[sel].abs() ** 2).sum().sqrt())}


def learned_networks(torch, rtw, retrain=False):
    """The per-order networks of the learned proposal: trained once on traced rays of the training
    drops (stream 2) and kept as a checkpoint; (handle, training seconds or None when loaded)."""
    from paper_2403_13856_gb300 import learned as Lr
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.LEARNED
    np_ = cfg["p_max"] + 1
    ck = os.path.join(ROOT, "paper_2403_13856_gb300", "_cache", "learned_p%d" % cfg["p_max"])
    if os.path.exists(ck + ".json") and not retrain:
        return Lr.load(ck), None
    t0 = time.perf_counter()
    tspecs, _ = W.batch_objects(cfg["train_objects"], stream=W.STREAM_TRAIN)
    tobj = rtw.Object([rtw.ObjectSpec(**s) for s in tspecs])
    samples = [Lr.Samples(tobj, cfg["train_rays"], cfg["p_max"])]
    mlp = rtw.MLP(np_, Lr.init_params(np_))
    losses = Lr.train(mlp, samples, range(np_), steps=cfg["train_steps"], batch=cfg["batch"], lr=3e-3, lr_end=3e-5)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    Lr.save(mlp, ck, {"losses": losses, "train_s": t_train})
    return mlp, t_train


def system_learned(torch, rtw, args, local, steps=1, warmup=1):
    """Learned proposals + Newton on the exact trace against dense tracing on 1024 drops: seconds
    per field of each form, and the errors of the learned and dense fields against the exact
    branch sum (dense FP64 trace with every hit refined by Newton)."""
    from paper_2403_13856_gb300 import autotune
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.LEARNED
    p_max, nt, nph = cfg["p_max"], cfg["n_theta"], cfg["n_phi"]
    np_ = p_max + 1
    stream = torch.cuda.current_stream()
    mlp, t_train = learned_networks(torch, rtw, getattr(args, "retrain", False))
    specs, rays = W.batch_objects(cfg["n_objects"], stream=W.STREAM_EVAL)
    n = len(specs)
    obj = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
    dirs = rtw.dirs_grid(nt, nph)
    ndir = nt * nph
    shape = (n, ndir, 1, 2)
    out_l = torch.empty(shape, dtype=torch.complex128, device="cuda")
    mask_l = torch.empty((n, ndir), dtype=torch.uint8, device="cuda")
    roots = torch.empty((n, ndir, np_), dtype=torch.uint8, device="cuda")
    lp = rtw.learned_params(p_max)
    with ClockSampler(local) as clk:
        t_learned = timed_on(torch, stream, lambda: rtw.rtw_field_learned(obj, mlp, lp, dirs, out_l, mask_l, roots,
                                                                           stream=stream), steps, warmup)
    rtw.rtw_sync_status(stream)
    # the same with a single-precision first approach to each root, and with the dense fallback for
    # the rows where a confident head did not converge (per-order output, summed afterwards)
    out_m = torch.empty(shape, dtype=torch.complex128, device="cuda")
    mask_m = torch.empty((n, ndir), dtype=torch.uint8, device="cuda")
    lpm = rtw.learned_params(p_max, precision=rtw.RTW_MIXED)
    t_mixed = timed_on(torch, stream, lambda: rtw.rtw_field_learned(obj, mlp, lpm, dirs, out_m, mask_m, stream=stream),
                       1, 0)
    out_fp = torch.empty((n, ndir, np_, 2), dtype=torch.complex128, device="cuda")
    mask_f = torch.empty((n, ndir), dtype=torch.uint8, device="cuda")
    roots_f = torch.empty((n, ndir, np_), dtype=torch.uint8, device="cuda")
    lpf = rtw.learned_params(p_max, fallback_rays=rays)
    t_fb = timed_on(torch, stream, lambda: rtw.rtw_field_learned(obj, mlp, lpf, dirs, out_fp, mask_f, roots_f,
                                                                  flags=rtw.RTW_FIELD_PER_ORDER, stream=stream), 1, 0)
    rtw.rtw_sync_status(stream)
    out_f = out_fp.sum(dim=2, keepdim=True)
    del out_fp
    # dense tracing on the same drops (autotuned batched launch, graph replay)
    opts = autotune.tune(specs, rays, p_max, rtw.RTW_FP64, nt, nph)
    res = {}
    for name, prec, mode in (("dense_fp64", rtw.RTW_FP64, rtw.RTW_DENSE), ("dense_mixed", rtw.RTW_MIXED, rtw.RTW_DENSE),
                             ("exact", rtw.RTW_FP64, rtw.RTW_NEWTON)):
        o_ = torch.empty(shape, dtype=torch.complex128, device="cuda")
        m_ = torch.empty((n, ndir), dtype=torch.uint8, device="cuda")
        bp = rtw.batch_params(rays, p_max=p_max, precision=prec, use_graph=1, mode=mode, **opts)
        b = rtw.Batch()
        t = timed_on(torch, stream, lambda: rtw.rtw_far_field_batch(obj, bp, dirs, o_, m_, batch=b, stream=stream),
                     1, 1)
        rtw.rtw_sync_status(stream)
        res[name] = (t, o_, m_)
    ref, rmask = res["exact"][1], res["exact"][2]
    e_learned = field_errors(torch, out_l, ref, mask_l, rmask)
    e_dense = field_errors(torch, res["dense_fp64"][1], ref, res["dense_fp64"][2], rmask)
    e_mixed = field_errors(torch, res["dense_mixed"][1], ref, res["dense_mixed"][2], rmask)
    e_lmixed = field_errors(torch, out_m, ref, mask_m, rmask)
    e_fb = field_errors(torch, out_f, ref, mask_f, rmask)
    unc_rows = int(((roots_f & 0x80) != 0).any(dim=-1).sum().item())
    t_dense = res["dense_fp64"][0]
    found = (roots & 0x7F).to(torch.int64).sum(dim=(0, 1)).tolist()
    uncertain = ((roots & 0x80) != 0).to(torch.int64).sum(dim=(0, 1)).tolist()
    return {"workload": "1024 drops of the batched recipe (stream 3), 256x512 (theta,phi) directions, p=0..4; "
                        "networks trained on 2e7 traced rays of 16384 drops (stream 2)",
            "learned": {"s_per_field": t_learned, "directions_per_s": n * ndir / t_learned,
                        "roots_per_order": found, "uncertain_rows_per_order": uncertain,
                        "params": {"p_min": lp.p_min or 0.05, "max_steps": lp.max_steps or 3,
                                   "max_halvings": lp.max_halvings or 3, "tol": "min(1e-6, 1e-4/(k0 L))"},
                        "errors_vs_exact": e_learned},
            "learned_mixed_first_approach": {"s_per_field": t_mixed, "errors_vs_exact": e_lmixed,
                                             "speedup_vs_dense_fp64": t_dense / t_mixed},
            "learned_with_dense_fallback": {"s_per_field": t_fb, "errors_vs_exact": e_fb,
                                            "rows_redone": unc_rows, "rows": n * ndir,
                                            "speedup_vs_dense_fp64": t_dense / t_fb},
            "dense_fp64": {"s_per_field": t_dense, "errors_vs_exact": e_dense},
            "dense_mixed": {"s_per_field": res["dense_mixed"][0], "errors_vs_exact": e_mixed},
            "exact_reference": {"s_per_field": res["exact"][0],
                                "what": "dense FP64 trace with every hit refined by Newton on the exact trace"},
            "speedup_learned_vs_dense_fp64": t_dense / t_learned,
            "train_s": t_train, "clocks": clk.summary()}


def bench_learned(args, rank, world, local, dist):
    """Learned proposals + Newton on the exact trace against dense tracing on 1024 drops."""
    import torch

    from paper_2403_13856_gb300 import rtw
    from paper_2403_13856_gb300 import workloads as W

    cfg = W.LEARNED
    r = system_learned(torch, rtw, args, local, steps=args.steps, warmup=args.warmup)
    n = cfg["n_objects"]
    t_learned = r["learned"]["s_per_field"]
    line = {
        "metric": METRIC, "value": n * cfg["n_theta"] * cfg["n_phi"] / t_learned, "unit": "directions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_learned,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f64", "data": "synthetic",
        "config": {"workload": r["workload"], "learned_params": r["learned"]["params"], "l2": "inputs larger than L2"},
    }
    line.update({k: v for k, v in r.items() if k != "workload"})
    if not args.no_cpu_baseline and world == 1:
        specs, _ = W.batch_objects(n, stream=W.STREAM_EVAL)
        line["cpu_baseline"] = cpu_baseline_learned(specs[0], cfg["p_max"], cfg["n_theta"], cfg["n_phi"])
    print(json.dumps(line), flush=True)


def cpu_baseline_learned(spec, p_max, nt, nph):
    """The oracle's learned-field pipeline on one evaluation drop (every direction and order),
    OpenMP over the host's cores.  Its networks are fixed outputs (all heads at the disk centre):
    the trained weights are outputs of the GPU and stay off the oracle."""
    import numpy as np

    import oracle

    oracle.build()
    th = np.zeros((p_max + 1, oracle.MLP_NPARAM))
    o = oracle.Object(spec["a"], spec["b"], spec["c"], quat=spec["quat"], m=spec["m"], wavelength=spec["wavelength"])
    t0 = time.perf_counter()
    o.field_learned(th, p_max, nt, nph)
    dt = time.perf_counter() - t0
    return {"value": nt * nph / dt, "unit": "directions/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"1 drop, {nt}x{nph} directions, orders 0..{p_max}, seeds at the disk centre, {dt:.1f} s"}


if __name__ == "__main__":
    main()
