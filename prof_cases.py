"""Small, fixed launches of the library's kernels for profilers (ncu) and quick timings.

    python prof_cases.py mlp_forward [--rows N]
    python prof_cases.py mlp_train [--rows N]
    python prof_cases.py caustic [--rays N]
    python prof_cases.py batch [--objects N]
    python prof_cases.py learned [--objects N]
    python prof_cases.py ellipsoid [--rays N]
    python prof_cases.py superellipsoid [--rays N] [--shape-e E]
    python prof_cases.py po2d [--sphere A] [--spacing H]
    python prof_cases.py pattern [--rays N] [--res DEG]

Each case builds its inputs (seeded), runs the launch sequence `--reps` times (default 3) after
one warm-up and prints the CUDA-event time of the last repetition.  Sizes default to cases that
hold a few GB at most, with inputs larger than L2 where the kernel streams memory.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def _timed(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    t = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1)
    return t


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["mlp_forward", "mlp_train", "caustic", "batch", "learned", "ellipsoid", "superellipsoid", "po2d",
                                     "pattern"])
    ap.add_argument("--rows", type=int, default=1 << 22)
    ap.add_argument("--objects", type=int, default=64)
    ap.add_argument("--rays", type=int, default=1_000_000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--shape-e", type=float, default=2.0, help="superellipsoid exponent e")
    ap.add_argument("--sphere", type=float, default=200.0, help="po2d: sphere radius (um)")
    ap.add_argument("--spacing", type=float, default=0.25, help="po2d: ray grid spacing (um)")
    ap.add_argument("--res", type=float, default=0.05, help="pattern: angular resolution (deg)")
    ap.add_argument("--mixed", action="store_true", help="ellipsoid / batch: mixed-precision trace")
    ap.add_argument("--dfloat", action="store_true", help="ellipsoid / batch: double-float trace")
    a = ap.parse_args()
    import torch

    from paper_2403_13856_gb300 import build, learned, rtw
    from paper_2403_13856_gb300 import workloads as W

    build.build()
    rtw.lib()
    prec = rtw.RTW_MIXED if a.mixed else (rtw.RTW_DFLOAT if a.dfloat else rtw.RTW_FP64)
    pname = {rtw.RTW_MIXED: "mixed", rtw.RTW_DFLOAT: "dfloat"}.get(prec, "fp64")
    if a.case == "mlp_forward":
        mlp = rtw.MLP(1, learned.init_params(1))
        g = np.random.default_rng(1)
        X = torch.tensor(g.uniform(-1, 1, (a.rows, 16)), dtype=torch.float32).to(torch.bfloat16).cuda()
        Y = torch.empty((a.rows, 16), dtype=torch.float32, device="cuda")
        ms = _timed(torch, lambda: rtw.rtw_mlp_forward(mlp, 0, X, Y), a.reps)
        flops = 2.0 * a.rows * (16 * 128 + 2 * 128 * 128 + 128 * 16)
        print(f"mlp_forward rows={a.rows}: {ms:.3f} ms, {flops / ms / 1e9:.1f} TFLOP/s")
    elif a.case == "mlp_train":
        # one training step of one network: gradient (tensor-core forward, backward and weight
        # gradients) and Adam on a batch of rows
        mlp = rtw.MLP(1, learned.init_params(1))
        g = np.random.default_rng(3)
        X = torch.tensor(g.uniform(-1, 1, (a.rows, 16)), dtype=torch.float32).to(torch.bfloat16).cuda()
        T = torch.tensor(g.uniform(-1, 1, (a.rows, 2)), dtype=torch.float32).cuda()
        V = torch.tensor(g.integers(1, 5, a.rows), dtype=torch.uint8).cuda()

        def tstep():
            rtw.rtw_mlp_grad(mlp, 0, X, T, V)
            rtw.rtw_mlp_adam(mlp, 0, 1e-3)

        ms = _timed(torch, tstep, a.reps)
        flops = 3 * 2.0 * a.rows * (16 * 128 + 2 * 128 * 128 + 128 * 16)
        print(f"mlp_train rows={a.rows}: {ms:.3f} ms per step, {flops / ms / 1e9:.1f} TFLOP/s")
    elif a.case == "caustic":
        # the physical optics at the caustics of the ellipsoid's 512 x 1024 field (default widths and tiles)
        spec, cfg = W.ELLIPSOID, W.ELLIPSOID_GRID
        obj = rtw.Object([rtw.ObjectSpec(**spec, jones=(1.0, 0.0))])
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=cfg["p_max"], n_rays=a.rays, flags=rtw.RTW_TRACE_APERTURE)
        rays = rtw.rtw_trace(obj, tp)
        nd = cfg["n_theta"] * cfg["n_phi"]
        out = torch.empty((nd, 1, 2), dtype=torch.complex128, device="cuda")
        d = rtw.dirs_grid(cfg["n_theta"], cfg["n_phi"])
        cp = rtw.caustic_params()
        ms = _timed(torch, lambda: rtw.rtw_field_caustic(rays, d, cp, out), a.reps)
        print(f"caustic rays={a.rays}: field with the caustic correction {ms:.3f} ms")
    elif a.case == "batch":
        specs, rays = W.batch_objects(a.objects)
        obj = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
        cfg = W.BATCH
        out = torch.empty((a.objects, cfg["n_theta"] * cfg["n_phi"], 1, 2), dtype=torch.complex128, device="cuda")
        bp = rtw.batch_params(rays, p_max=cfg["p_max"], precision=prec)
        b = rtw.Batch()
        ms = _timed(torch, lambda: rtw.rtw_far_field_batch(obj, bp, rtw.dirs_grid(cfg["n_theta"], cfg["n_phi"]), out,
                                                           batch=b), a.reps)
        print(f"batch objects={a.objects} rays={int(np.sum(rays))} {pname}: {ms:.3f} ms")
    elif a.case == "learned":
        cfg = W.LEARNED
        specs, _ = W.batch_objects(a.objects, stream=W.STREAM_EVAL)
        obj = rtw.Object([rtw.ObjectSpec(**s) for s in specs])
        mlp = rtw.MLP(cfg["p_max"] + 1, learned.init_params(cfg["p_max"] + 1))
        nd = cfg["n_theta"] * cfg["n_phi"]
        out = torch.empty((a.objects, nd, 1, 2), dtype=torch.complex128, device="cuda")
        lp = rtw.learned_params(cfg["p_max"])
        ms = _timed(torch, lambda: rtw.rtw_field_learned(obj, mlp, lp, rtw.dirs_grid(cfg["n_theta"], cfg["n_phi"]),
                                                         out), a.reps)
        print(f"learned objects={a.objects}: {ms:.3f} ms")
    elif a.case == "pattern":
        # the side-lit spheroid's whole pattern at --res degrees (0.01 with 4e6 rays is the benchmark;
        # 0.05 with 1.6e5 rays keeps the same directions per triangle)
        obj = rtw.Object([rtw.ObjectSpec(**W.SPHEROID_SIDE, jones=(0.0, 1.0))])
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=5, n_rays=a.rays)
        rays = rtw.rtw_trace(obj, tp)
        nt = int(round(180.0 / a.res))
        out = torch.empty((nt * 2 * nt, 1, 2), dtype=torch.complex128, device="cuda")
        dirs = rtw.dirs_grid(nt, 2 * nt)
        ms = _timed(torch, lambda: rtw.rtw_field(rays, dirs, out), a.reps)
        print(f"pattern rays={a.rays} res={a.res} deg ({nt}x{2 * nt}): field {ms:.3f} ms")
    elif a.case == "po2d":
        import math

        sa = a.sphere
        obj = rtw.Object([rtw.ObjectSpec(a=sa, b=sa, c=sa, quat=(1.0, 0.0, 0.0, 0.0), m=W.WATER, wavelength=W.HE_NE,
                                         jones=(0.0, 1.0))])
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=2, spacing=a.spacing, flags=rtw.RTW_TRACE_APERTURE)
        rays = rtw.rtw_trace(obj, tp)
        _, nx, ny = obj.grid(0, tp)
        aw, fw = (W.HE_NE / sa) ** (2.0 / 3.0), 1.0 / math.sqrt(2.0 * math.pi / W.HE_NE * sa)
        thc = math.radians(137.922)
        tg, pg = torch.meshgrid(thc + torch.linspace(-0.4 * aw, 1.5 * aw, 64, dtype=torch.float64),
                                torch.linspace(-0.035, 0.035, 64, dtype=torch.float64), indexing="ij")
        dirs = torch.stack([tg.reshape(-1), pg.reshape(-1)], 1).cuda()
        out = torch.empty((dirs.shape[0], 2), dtype=torch.complex128, device="cuda")
        pp = rtw.po2d_params(2, [0, nx // 2, 0, ny - 1], (thc, 0.0), (3 * aw + 3 * fw, 3 * aw + 6 * fw))
        used = rtw.rtw_field_po2d(rays, pp, dirs, out, count=True)
        ms = _timed(torch, lambda: rtw.rtw_field_po2d(rays, pp, dirs, out), a.reps)
        print(f"po2d sphere={sa} grid={nx}x{ny} rays={used} dirs={dirs.shape[0]}: {ms:.3f} ms, "
              f"{used * dirs.shape[0] / ms / 1e6:.3f} Gterms/s")
    else:
        spec, cfg = W.ELLIPSOID, W.ELLIPSOID_GRID
        if a.case == "superellipsoid":
            spec = dict(W.SUPERELLIPSOID, shape_e=a.shape_e)
        obj = rtw.Object([rtw.ObjectSpec(**spec)])
        tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=cfg["p_max"], n_rays=a.rays,
                              precision=prec)
        rays = rtw.rtw_trace(obj, tp)
        out = torch.empty((cfg["n_theta"] * cfg["n_phi"], 1, 2), dtype=torch.complex128, device="cuda")

        def step():
            rtw.rtw_trace(obj, tp, rays)
            rtw.rtw_field(rays, rtw.dirs_grid(cfg["n_theta"], cfg["n_phi"]), out)

        ms = _timed(torch, step, a.reps)
        mt = _timed(torch, lambda: rtw.rtw_trace(obj, tp, rays), a.reps)
        print(f"{a.case} rays={a.rays} {pname}: trace + field {ms:.3f} ms, trace {mt:.3f} ms")
    rtw.rtw_sync_status()


if __name__ == "__main__":
    main()
