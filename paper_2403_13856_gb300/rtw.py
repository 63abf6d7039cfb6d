"""Thin ctypes binding of librtw.so (include/rtw.h), the GB300 Ray Theory of Waves library.

Argument marshalling only: every step of the path runs in the CUDA kernels behind the C ABI.
Device buffers are torch tensors (PyTorch provides device memory and streams).  There is no
CPU fallback: if the library or a CUDA device is missing, every call raises RTWError.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "librtw.so")

RTW_OK = 0
RTW_GRID_FAN, RTW_GRID_SQUARE = 0, 1
RTW_FP64, RTW_MIXED, RTW_DFLOAT = 0, 1, 2
RTW_DENSE, RTW_NEWTON = 0, 1
RTW_DIRS_PLANE, RTW_DIRS_GRID, RTW_DIRS_LIST = 0, 1, 2
RTW_FIELD_PER_ORDER, RTW_FIELD_PO, RTW_FIELD_NEAR_FOLDS = 1, 2, 4
RTW_TRACE_APERTURE = 1
RTW_MASK_CAUSTIC, RTW_MASK_AXIAL, RTW_MASK_PO = 1, 2, 4
FLAG_VALID, FLAG_ORIENT, FLAG_CAUSTIC = 1, 2, 4


class RTWError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rtw error {code}: {msg}")
        self.code = code


class rtw_object_desc(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("quat", ctypes.c_double * 4), ("center", ctypes.c_double * 3),
                ("m_re", ctypes.c_double), ("m_im", ctypes.c_double), ("shape_e", ctypes.c_double)]


class rtw_incident(ctypes.Structure):
    _fields_ = [("wavelength_um", ctypes.c_double), ("dir", ctypes.c_double * 3),
                ("jones_re", ctypes.c_double * 2), ("jones_im", ctypes.c_double * 2), ("kind", ctypes.c_int),
                ("source", ctypes.c_double * 3)]


class rtw_trace_params(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int), ("p_max", ctypes.c_int), ("precision", ctypes.c_int),
                ("flags", ctypes.c_int), ("n_rays", ctypes.c_int64), ("spacing", ctypes.c_double),
                ("fan_phi", ctypes.c_double), ("observe_radius", ctypes.c_double)]


class rtw_dirs(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("alpha0", ctypes.c_double), ("dalpha", ctypes.c_double), ("cell_window", ctypes.c_int64 * 4),
                ("list", ctypes.c_void_p), ("n_list", ctypes.c_int64)]


class rtw_batch_params(ctypes.Structure):
    _fields_ = [("p_max", ctypes.c_int), ("precision", ctypes.c_int), ("n_rays", ctypes.c_void_p),
                ("chunk_ray_orders", ctypes.c_int64), ("trace_variant", ctypes.c_int),
                ("trace_ctas_per_sm", ctypes.c_int), ("classify_block", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("timing", ctypes.c_int), ("mode", ctypes.c_int)]


TRACE_VARIANTS = 5

_lib = None


def lib():
    """Loads librtw.so; raises RTWError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RTWError(-3, f"{LIB_PATH} is missing: build it with paper_2403_13856_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        p, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        sig = {
            "rtw_create_object": ([p, i, p, p], i),
            "rtw_destroy_object": ([p], None),
            "rtw_object_grid": ([p, i, p, p, p, p], i),
            "rtw_trace": ([p, p, p, p], i),
            "rtw_rays_info": ([p, p, p, p], i),
            "rtw_rays_export": ([p, i, i64, i64, p, p, p, p, p], i),
            "rtw_destroy_rays": ([p], None),
            "rtw_trace_points": ([p, i, p, i64, i, p, p, p, p, p], i),
            "rtw_field": ([p, p, i, i, p, p, p], i),
            "rtw_field_po2d": ([p, p, p, i64, p, p, p], i),
            "rtw_field_caustic": ([p, p, p, i, p, p, p, p], i),
            "rtw_far_field_batch": ([p, p, p, i, p, p, p, p], i),
            "rtw_batch_info": ([p, p, p, p], i),
            "rtw_batch_times": ([p, p, p], i),
            "rtw_destroy_batch": ([p], None),
            "rtw_mlp_create": ([i, p, p], i),
            "rtw_mlp_destroy": ([p], None),
            "rtw_mlp_get": ([p, i, p, p, p, p], i),
            "rtw_mlp_set": ([p, i, p, p, p, i64], i),
            "rtw_mlp_samples": ([p, p, p, i64, i, p, p, p, p], i),
            "rtw_mlp_forward": ([p, i, p, i64, p, p], i),
            "rtw_mlp_activation_eval": ([p, p, i64, p], i),
            "rtw_mlp_grad": ([p, i, p, p, p, i64, ctypes.c_float, p, p], i),
            "rtw_mlp_grad_get": ([p, i, p, p], i),
            "rtw_mlp_adam": ([p, i, ctypes.c_float, p, p], i),
            "rtw_field_learned": ([p, p, p, p, i, p, p, p, p], i),
            "rtw_pipe_peak": ([i, i64, i, p, p, p], i),
            "rtw_sync_status": ([p], i),
            "rtw_newton_failures": ([p, p], i),
            "rtw_status_string": ([i], ctypes.c_char_p),
            "rtw_last_error": ([], ctypes.c_char_p),
            "rtw_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != RTW_OK:
        raise RTWError(rc, lib().rtw_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


@dataclass
class ObjectSpec:
    a: float
    b: float
    c: float
    quat: Sequence[float] = (1.0, 0.0, 0.0, 0.0)
    center: Sequence[float] = (0.0, 0.0, 0.0)
    m: float = 1.333
    wavelength: float = 0.6328
    jones: Sequence[complex] = (1.0, 0.0)
    source: Optional[Sequence[float]] = None  # point source position (um), else a plane wave along +z
    shape_e: float = 1.0  # superellipsoid exponent e >= 1 (sum |u_i|^(2e) = 1); 1: the ellipsoid


class Object:
    """rtw_object handle (one or many ellipsoids with their incident waves)."""

    def __init__(self, specs: Sequence[ObjectSpec]):
        n = len(specs)
        descs = (rtw_object_desc * n)()
        incs = (rtw_incident * n)()
        for k, s in enumerate(specs):
            d = descs[k]
            d.a, d.b, d.c = s.a, s.b, s.c
            d.quat[:] = list(s.quat)
            d.center[:] = list(s.center)
            d.m_re, d.m_im = s.m, 0.0
            d.shape_e = s.shape_e
            w = incs[k]
            w.wavelength_um = s.wavelength
            w.dir[:] = [0.0, 0.0, 1.0]
            j = [complex(x) for x in s.jones]
            w.jones_re[:] = [j[0].real, j[1].real]
            w.jones_im[:] = [j[0].imag, j[1].imag]
            w.kind = 0 if s.source is None else 1
            w.source[:] = [0.0, 0.0, 0.0] if s.source is None else [float(v) for v in s.source]
        h = ctypes.c_void_p()
        _check(lib().rtw_create_object(ctypes.byref(descs), n, ctypes.byref(incs), ctypes.byref(h)))
        self.handle = h
        self.count = n
        self.specs = list(specs)

    def grid(self, index: int, params: "rtw_trace_params"):
        h = ctypes.c_double()
        nx, ny = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().rtw_object_grid(self.handle, index, ctypes.byref(params), ctypes.byref(h), ctypes.byref(nx),
                                     ctypes.byref(ny)))
        return h.value, nx.value, ny.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.rtw_destroy_object(self.handle)
            self.handle = None


def trace_params(grid=RTW_GRID_SQUARE, p_max=5, precision=RTW_FP64, flags=0, n_rays=0, spacing=0.0, fan_phi=0.0,
                 observe_radius=0.0):
    tp = rtw_trace_params()
    tp.grid, tp.p_max, tp.precision, tp.flags = grid, p_max, precision, flags
    tp.n_rays, tp.spacing, tp.fan_phi = int(n_rays), float(spacing), float(fan_phi)
    tp.observe_radius = float(observe_radius)
    return tp


class Rays:
    """rtw_rays handle: the traced ray state, owned by the library."""

    def __init__(self):
        self.handle = ctypes.c_void_p()

    def info(self):
        R, npo, nob = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _check(lib().rtw_rays_info(self.handle, ctypes.byref(R), ctypes.byref(npo), ctypes.byref(nob)))
        return R.value, npo.value, nob.value

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.rtw_destroy_rays(self.handle)
            self.handle = ctypes.c_void_p()


def rtw_trace(obj: Object, params: rtw_trace_params, rays: Optional[Rays] = None, stream=None) -> Rays:
    rays = rays or Rays()
    _check(lib().rtw_trace(obj.handle, ctypes.byref(params), _stream_ptr(stream), ctypes.byref(rays.handle)))
    return rays


def rtw_rays_export(rays: Rays, order: int, first: int, count: int, s=None, F=None, psi=None, flags=None,
                    stream=None):
    _check(lib().rtw_rays_export(rays.handle, order, first, count, _ptr(s), _ptr(F), _ptr(psi), _ptr(flags),
                                 _stream_ptr(stream)))


def rtw_trace_points(obj: Object, index: int, xy, p_max: int, s=None, F=None, psi=None, flags=None, stream=None):
    n = xy.shape[0]
    _check(lib().rtw_trace_points(obj.handle, index, _ptr(xy), n, p_max, _ptr(s), _ptr(F), _ptr(psi), _ptr(flags),
                                  _stream_ptr(stream)))


def dirs_plane(n: int, alpha0: float, dalpha: float) -> rtw_dirs:
    d = rtw_dirs()
    d.kind, d.n_theta, d.n_phi, d.alpha0, d.dalpha = RTW_DIRS_PLANE, n, 0, alpha0, dalpha
    d.cell_window[:] = [-1, -1, -1, -1]
    return d


def dirs_grid(n_theta: int, n_phi: int, cell_window=None) -> rtw_dirs:
    d = rtw_dirs()
    d.kind, d.n_theta, d.n_phi = RTW_DIRS_GRID, n_theta, n_phi
    d.cell_window[:] = list(cell_window) if cell_window is not None else [-1, -1, -1, -1]
    return d


def dirs_list(theta_phi) -> rtw_dirs:
    """Directions from a device tensor of (theta, phi) pairs (float64, n x 2), kept alive on the
    returned structure."""
    d = rtw_dirs()
    d.kind, d.n_theta, d.n_phi, d.alpha0, d.dalpha = RTW_DIRS_LIST, 0, 0, 0.0, 0.0
    d.cell_window[:] = [-1, -1, -1, -1]
    d._keep = theta_phi
    d.list = theta_phi.data_ptr()
    d.n_list = theta_phi.shape[0]
    return d


class rtw_po2d_params(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("window", ctypes.c_int64 * 4), ("axis_theta", ctypes.c_double),
                ("axis_phi", ctypes.c_double), ("cone_full", ctypes.c_double), ("cone_end", ctypes.c_double)]


def po2d_params(order, window, axis, cone) -> rtw_po2d_params:
    pp = rtw_po2d_params()
    pp.order = int(order)
    pp.window[:] = [int(v) for v in window]
    pp.axis_theta, pp.axis_phi = float(axis[0]), float(axis[1])
    pp.cone_full, pp.cone_end = float(cone[0]), float(cone[1])
    return pp


def rtw_field_po2d(rays: Rays, pp: rtw_po2d_params, dirs, out, count=False, stream=None):
    """dirs: (n, 2) float64 (theta, phi) on the device; out: (n, 2) complex128 on the device.
    count=True returns the number of rays in the sum (the call then synchronises the stream)."""
    n = ctypes.c_int64(-1)
    _check(lib().rtw_field_po2d(rays.handle, ctypes.byref(pp), _ptr(dirs), dirs.shape[0], _ptr(out),
                                ctypes.byref(n) if count else None, _stream_ptr(stream)))
    return n.value if count else None


class rtw_caustic_params(ctypes.Structure):
    _fields_ = [("tile_theta", ctypes.c_int), ("tile_phi", ctypes.c_int), ("po_full", ctypes.c_double),
                ("po_end", ctypes.c_double), ("cone_full", ctypes.c_double), ("cone_end", ctypes.c_double),
                ("p_min", ctypes.c_int)]


def caustic_params(tile=(0, 0), po=(0.0, 0.0), cone=(0.0, 0.0), p_min=0) -> rtw_caustic_params:
    """Parameters of rtw_field_caustic; zeros take the library's defaults."""
    cp = rtw_caustic_params()
    cp.tile_theta, cp.tile_phi = int(tile[0]), int(tile[1])
    cp.po_full, cp.po_end = float(po[0]), float(po[1])
    cp.cone_full, cp.cone_end = float(cone[0]), float(cone[1])
    cp.p_min = int(p_min)
    return cp


def rtw_field_caustic(rays: Rays, dirs: rtw_dirs, cp: rtw_caustic_params, out, mask=None, weights=None, flags=0,
                      stream=None):
    """Square-grid far field with the 2-D physical optics of the caustics blended in (device tensors:
    out as rtw_field, mask (directions,) uint8, weights (directions, orders) float64)."""
    _check(lib().rtw_field_caustic(rays.handle, ctypes.byref(dirs), ctypes.byref(cp), flags, _ptr(out), _ptr(mask),
                                   _ptr(weights), _stream_ptr(stream)))


def rtw_field(rays: Rays, dirs: rtw_dirs, out, mask=None, mode=RTW_DENSE, flags=0, stream=None):
    _check(lib().rtw_field(rays.handle, ctypes.byref(dirs), mode, flags, _ptr(out), _ptr(mask), _stream_ptr(stream)))


class Batch:
    """rtw_batch handle: ray state, workspace and recorded graph of rtw_far_field_batch."""

    def __init__(self):
        self.handle = ctypes.c_void_p()

    def info(self):
        R, nc, rep = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _check(lib().rtw_batch_info(self.handle, ctypes.byref(R), ctypes.byref(nc), ctypes.byref(rep)))
        return R.value, nc.value, bool(rep.value)

    def times(self):
        t, f = ctypes.c_double(), ctypes.c_double()
        _check(lib().rtw_batch_times(self.handle, ctypes.byref(t), ctypes.byref(f)))
        return t.value, f.value

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.rtw_destroy_batch(self.handle)
            self.handle = ctypes.c_void_p()


def batch_params(n_rays, p_max=4, precision=RTW_FP64, chunk_ray_orders=0, trace_variant=0, trace_ctas_per_sm=0,
                 classify_block=0, use_graph=0, timing=0, mode=RTW_DENSE):
    """Options of rtw_far_field_batch; n_rays is kept alive on the returned structure."""
    bp = rtw_batch_params()
    arr = (ctypes.c_int64 * len(n_rays))(*[int(x) for x in n_rays])
    bp._n_rays = arr
    bp.n_rays = ctypes.cast(arr, ctypes.c_void_p)
    bp.p_max, bp.precision, bp.chunk_ray_orders = p_max, precision, int(chunk_ray_orders)
    bp.trace_variant, bp.trace_ctas_per_sm, bp.classify_block = trace_variant, trace_ctas_per_sm, classify_block
    bp.use_graph, bp.timing, bp.mode = int(use_graph), int(timing), int(mode)
    return bp


def rtw_far_field_batch(obj: Object, params: rtw_batch_params, dirs: rtw_dirs, out, mask=None, flags=0,
                        batch: Optional[Batch] = None, stream=None) -> Batch:
    batch = batch or Batch()
    _check(lib().rtw_far_field_batch(obj.handle, ctypes.byref(params), ctypes.byref(dirs), flags, _ptr(out),
                                     _ptr(mask), ctypes.byref(batch.handle), _stream_ptr(stream)))
    return batch


def rtw_sync_status(stream=None):
    _check(lib().rtw_sync_status(_stream_ptr(stream)))


RTW_MLP_NPARAM = 37264


class MLP:
    """rtw_mlp handle: one network per order (learned entry-point proposal)."""

    def __init__(self, n_orders: int, init=None):
        import numpy as np

        self.handle = ctypes.c_void_p()
        self.n_orders = n_orders
        buf = None
        if init is not None:
            buf = np.ascontiguousarray(init, dtype=np.float32).reshape(n_orders, RTW_MLP_NPARAM)
        _check(lib().rtw_mlp_create(n_orders, None if buf is None else buf.ctypes.data_as(ctypes.c_void_p),
                                    ctypes.byref(self.handle)))

    def get(self, order: int):
        import numpy as np

        th, m, v = (np.zeros(RTW_MLP_NPARAM, dtype=np.float32) for _ in range(3))
        step = ctypes.c_int64()
        _check(lib().rtw_mlp_get(self.handle, order, th.ctypes.data_as(ctypes.c_void_p),
                                 m.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(step)))
        return th, m, v, step.value

    def set(self, order: int, theta, m=None, v=None, step: int = 0):
        import numpy as np

        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (theta, m, v)]
        ptrs = [None if a is None else a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
        _check(lib().rtw_mlp_set(self.handle, order, *ptrs, int(step)))

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.rtw_mlp_destroy(self.handle)
            self.handle = ctypes.c_void_p()


def rtw_mlp_samples(obj: Object, uv, obj_index, p_max, X, T, valid, stream=None):
    _check(lib().rtw_mlp_samples(obj.handle, _ptr(uv), _ptr(obj_index), uv.shape[0], p_max, _ptr(X), _ptr(T),
                                 _ptr(valid), _stream_ptr(stream)))


def rtw_mlp_forward(mlp: MLP, order, X, Y, stream=None):
    _check(lib().rtw_mlp_forward(mlp.handle, order, _ptr(X), X.shape[0], _ptr(Y), _stream_ptr(stream)))


def rtw_mlp_activation_eval(x, y, stream=None):
    """The inference kernel's GELU on a float32 device tensor x into y."""
    _check(lib().rtw_mlp_activation_eval(_ptr(x), _ptr(y), x.numel(), _stream_ptr(stream)))


def rtw_mlp_grad(mlp: MLP, order, X, T, valid, beta=0.1, loss=None, stream=None):
    _check(lib().rtw_mlp_grad(mlp.handle, order, _ptr(X), _ptr(T), _ptr(valid), X.shape[0], float(beta), _ptr(loss),
                              _stream_ptr(stream)))


def rtw_mlp_grad_get(mlp: MLP, order, grad, stream=None):
    _check(lib().rtw_mlp_grad_get(mlp.handle, order, _ptr(grad), _stream_ptr(stream)))


def rtw_mlp_adam(mlp: MLP, order, lr, grad=None, stream=None):
    _check(lib().rtw_mlp_adam(mlp.handle, order, float(lr), _ptr(grad), _stream_ptr(stream)))


class rtw_learned_params(ctypes.Structure):
    _fields_ = [("p_max", ctypes.c_int), ("p_min", ctypes.c_float), ("max_steps", ctypes.c_int),
                ("tol", ctypes.c_double), ("chunk_rows", ctypes.c_int64), ("max_halvings", ctypes.c_int),
                ("precision", ctypes.c_int), ("fallback_rays", ctypes.c_void_p)]


def learned_params(p_max, p_min=0.0, max_steps=0, tol=0.0, chunk_rows=0, max_halvings=0, precision=0,
                   fallback_rays=None):
    """fallback_rays: per-object ray counts of the dense fallback (kept alive in the returned
    structure), or None."""
    lp = rtw_learned_params()
    lp.p_max, lp.p_min, lp.max_steps, lp.tol, lp.chunk_rows = p_max, p_min, max_steps, tol, int(chunk_rows)
    lp.max_halvings = int(max_halvings)
    lp.precision = int(precision)
    if fallback_rays is not None:
        lp._fallback = (ctypes.c_int64 * len(fallback_rays))(*[int(n) for n in fallback_rays])
        lp.fallback_rays = ctypes.cast(lp._fallback, ctypes.c_void_p)
    return lp


def rtw_field_learned(obj: Object, mlp: MLP, params: rtw_learned_params, dirs: rtw_dirs, out, mask=None, roots=None,
                      flags=0, stream=None):
    _check(lib().rtw_field_learned(obj.handle, mlp.handle, ctypes.byref(params), ctypes.byref(dirs), flags, _ptr(out),
                                   _ptr(mask), _ptr(roots), _stream_ptr(stream)))


RTW_PEAK_FP64, RTW_PEAK_FP32, RTW_PEAK_FP32X2 = 0, 1, 2


def rtw_pipe_peak(kind, iters, blocks_per_sm, sink, stream=None) -> float:
    """Launches the pipe-throughput kernel of `kind` on `stream`; returns the launch's flops."""
    flops = ctypes.c_double()
    _check(lib().rtw_pipe_peak(int(kind), int(iters), int(blocks_per_sm), _ptr(sink), ctypes.byref(flops),
                               _stream_ptr(stream)))
    return flops.value


def rtw_newton_failures(stream=None) -> int:
    n = ctypes.c_int64()
    _check(lib().rtw_newton_failures(_stream_ptr(stream), ctypes.byref(n)))
    return n.value


def rtw_version() -> str:
    return lib().rtw_version().decode()


def n_dirs(dirs: rtw_dirs) -> int:
    if dirs.kind == RTW_DIRS_LIST:
        return dirs.n_list
    return dirs.n_theta if dirs.kind == RTW_DIRS_PLANE else dirs.n_theta * dirs.n_phi


def plane_angles(dirs: rtw_dirs):
    """The in-plane angles alpha_k = alpha0 + k dalpha of a plane direction set (host numbers)."""
    return [dirs.alpha0 + k * dirs.dalpha for k in range(dirs.n_theta)]


def grid_angles(n_theta: int, n_phi: int):
    th = [(i + 0.5) * math.pi / n_theta for i in range(n_theta)]
    ph = [-math.pi + (j + 0.5) * 2 * math.pi / n_phi for j in range(n_phi)]
    return th, ph
