"""Operation count of the oracle's trace (the algorithmic flops of one ray interaction).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Builds the counting form of the oracle (opcount.cpp: the
oracle's sources compiled as C++ with every double counting the operations it executes), traces a
sample of a workload's rays with it and reports the counts per interaction.  Run as a script it
writes the stored count the benchmark divides by:

    python -m oracle.opcount            # writes tests/golden/oracle_flops_per_interaction.json

Only the test suite runs this module; the benchmark reads the JSON file it writes.
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_LIB = os.path.join(_HERE, "libopcount.so")
_SRCS = [os.path.join(_HERE, f) for f in ("opcount.cpp", "opcount.h", "rtw_oracle.c", "rtw_oracle.h", "mlp_oracle.c",
                                          "mlp_oracle.h")]
GOLDEN = os.path.join(_ROOT, "tests", "golden", "oracle_flops_per_interaction.json")
KINDS = ("add", "mul", "div", "sqrt", "fn")
_lib = None


def build(force: bool = False) -> str:
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(s) > os.path.getmtime(_LIB) for s in _SRCS)
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp,
               os.path.join(_HERE, "opcount.cpp")]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.or_opcount_trace.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p]
        L.or_opcount_trace.restype = ctypes.c_int64
        _lib = L
    return _lib


def count_trace(params, xy, pmax, records=False):
    """Counts of the oracle's trace of the impact points xy (n x 2) of the object with parameter
    vector params (oracle.Object.params): (interactions of the rays that hit, counts by kind,
    records (n x (pmax+1) x NFIELD) or None)."""
    from . import NFIELD

    params = np.ascontiguousarray(params, dtype=np.float64)
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((xy.shape[0], pmax + 1, NFIELD)) if records else None
    cnt = (ctypes.c_ulonglong * len(KINDS))()
    inter = lib().or_opcount_trace(params.ctypes.data, xy.ctypes.data, xy.shape[0], int(pmax),
                                   None if out is None else out.ctypes.data, cnt)
    if inter < 0:
        raise ValueError("invalid object parameters")
    return int(inter), dict(zip(KINDS, (int(c) for c in cnt))), out


def ellipsoid_sample(stride: int = 40):
    """The benchmark ellipsoid (120, 100, 80) um tilted 20 deg about x, orders 0..5: every
    stride-th row and column of its 4e6-ray square grid, the grid points whose rays hit."""
    from . import Object
    from paper_2403_13856_gb300 import workloads as W

    spec, cfg = W.ELLIPSOID, W.ELLIPSOID_GRID
    o = Object(spec["a"], spec["b"], spec["c"], quat=spec["quat"], m=spec["m"], wavelength=spec["wavelength"],
               jones=(1.0, 0.0))
    h, nx, ny, xc, yc = o.square_grid(cfg["n_rays"])
    xs = xc + (np.arange(nx) + 0.5 - nx / 2) * h
    ys = yc + (np.arange(ny) + 0.5 - ny / 2) * h
    X, Y = np.meshgrid(xs[::stride], ys[::stride])
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    hit = np.array([o.trace_ray(x, y, 0)[2] for x, y in xy])
    return o, xy[hit], cfg["p_max"]


def measure(stride: int = 40):
    o, xy, pmax = ellipsoid_sample(stride)
    inter, cnt, _ = count_trace(o.params, xy, pmax)
    return {"workload": "ellipsoid (120,100,80) um tilt 20 deg about x, m=1.333, lambda=0.6328 um, x-pol, p=0..5",
            "sample": f"every {stride}th row and column of the 4e6-ray grid, rays that hit: {xy.shape[0]}",
            "interactions": inter, "counts": cnt,
            "flops_per_interaction": sum(cnt.values()) / inter,
            "per_interaction": {k: v / inter for k, v in cnt.items()},
            "definition": "operations executed by the oracle's trace (or_trace_ray, all orders and far-field "
                          "records): additions, multiplications, divisions, square roots and elementary "
                          "functions, one each"}


if __name__ == "__main__":
    sys.path.insert(0, _ROOT)
    res = measure()
    with open(GOLDEN, "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")
    print(json.dumps(res, indent=1))
