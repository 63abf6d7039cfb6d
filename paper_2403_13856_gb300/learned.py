"""Training driver of the learned entry-point proposal (host orchestration only).

Every numerical step runs in the library's kernels: rtw_mlp_samples traces the rays and builds
features and targets, rtw_mlp_grad runs the forward, loss and backward kernels, rtw_mlp_adam the
optimiser.  This module draws the seeded inputs (entry points uniform on the unit disk of each
object, initial weights), slices batches and keeps checkpoints.
"""
from __future__ import annotations

import json
import os
from typing import Optional, Sequence

import numpy as np

from . import rtw
from . import workloads as W

NPARAM = rtw.RTW_MLP_NPARAM
LAYERS = ((128, 16), (128, 128), (128, 128), (16, 128))  # (out, in)


def init_params(n_orders: int, stream: int = W.STREAM_TRAIN, scale: float = 1.0) -> np.ndarray:
    """He-scaled normal weights and zero biases, drawn from the seeded generator (float32); the
    last layer is scaled down so that the first proposals start near the disk centre."""
    g = W.philox(stream + 1000)
    th = np.zeros((n_orders, NPARAM), dtype=np.float32)
    for p in range(n_orders):
        k = 0
        for li, (nout, nin) in enumerate(LAYERS):
            s = scale * np.sqrt(2.0 / nin) * (0.1 if li == 3 else 1.0)
            th[p, k:k + nout * nin] = g.standard_normal(nout * nin) * s
            k += nout * nin + nout
    return th


def disk_points(g, n: int) -> np.ndarray:
    r, a = np.sqrt(g.random(n)), 2 * np.pi * g.random(n)
    return np.stack([r * np.cos(a), r * np.sin(a)], 1)


class Samples:
    """Traced training rows of one batch of objects: X[p], T[p], valid[p] per order."""

    def __init__(self, obj: rtw.Object, n_rays: int, p_max: int, stream: int = W.STREAM_TRAIN, seed_offset: int = 0):
        import torch

        g = W.philox(stream + 100 * seed_offset)
        uv = torch.tensor(disk_points(g, n_rays)).cuda()
        oi = torch.tensor(g.integers(0, obj.count, n_rays).astype(np.int32)).cuda()
        np_ = p_max + 1
        self.n = n_rays
        self.p_max = p_max
        self.X = torch.empty((np_ * n_rays, 16), dtype=torch.bfloat16, device="cuda")
        self.T = torch.empty((np_ * n_rays, 2), dtype=torch.float32, device="cuda")
        self.valid = torch.empty(np_ * n_rays, dtype=torch.uint8, device="cuda")
        rtw.rtw_mlp_samples(obj, uv, oi, p_max, self.X, self.T, self.valid)

    def order(self, p: int):
        sl = slice(p * self.n, (p + 1) * self.n)
        return self.X[sl], self.T[sl], self.valid[sl]


def train(mlp: rtw.MLP, samples: Sequence[Samples], orders: Sequence[int], steps: int, batch: int = 8192,
          lr: float = 2e-3, lr_end: float = 1e-4, beta: float = 0.1, log_every: int = 0):
    """Adam on batches cycling through the samples, learning rate decayed geometrically from lr to
    lr_end; returns the mean loss of the last 50 steps per order."""
    import torch

    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = {}
    for p in orders:
        hist = []
        pos = 0
        si = 0
        for k in range(steps):
            X, T, V = samples[si].order(p)
            if pos + batch > X.shape[0]:
                pos = 0
                si = (si + 1) % len(samples)
                X, T, V = samples[si].order(p)
            sl = slice(pos, pos + batch)
            pos += batch
            rtw.rtw_mlp_grad(mlp, p, X[sl], T[sl], V[sl], beta=beta, loss=loss)
            rate = lr * (lr_end / lr) ** (k / max(1, steps - 1))
            rtw.rtw_mlp_adam(mlp, p, rate)
            if k >= steps - 50 or (log_every and k % log_every == 0):
                hist.append(loss.item())
        out[p] = float(np.mean(hist[-50:]))
    return out


def save(mlp: rtw.MLP, path: str, meta: Optional[dict] = None) -> None:
    """Checkpoint: a flat float32 binary (theta, m, v per order) and a JSON header."""
    arrs, steps = [], []
    for p in range(mlp.n_orders):
        th, m, v, st = mlp.get(p)
        arrs += [th, m, v]
        steps.append(st)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.concatenate(arrs).astype(np.float32).tofile(path + ".bin")
    with open(path + ".json", "w") as f:
        json.dump({"n_orders": mlp.n_orders, "nparam": NPARAM, "steps": steps, **(meta or {})}, f, indent=1)


def load(path: str) -> rtw.MLP:
    with open(path + ".json") as f:
        head = json.load(f)
    n = head["n_orders"]
    data = np.fromfile(path + ".bin", dtype=np.float32).reshape(n, 3, NPARAM)
    mlp = rtw.MLP(n)
    for p in range(n):
        mlp.set(p, data[p, 0], data[p, 1], data[p, 2], head["steps"][p])
    return mlp
