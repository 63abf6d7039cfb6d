"""Plain FP64 CPU oracle of the Ray Theory of Waves far field (ctypes binding).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` import this package.  The CUDA library under
``paper_2403_13856_gb300/`` never imports it, and the two share no code.

The C source ``rtw_oracle.c`` cites, per function, the passage of Ren et al., "Ray Theory of
Waves" (arXiv:2403.13856) it follows: Eqs. (SnellVec), (Fres), (WavefrontEqVec), (Theta-r),
(IntVCRM), (DivFactVCRM), (epsilon_VCRM), (PhasePath), (PhaseTotal) and the "Strategy of Ray
Theory of Waves" / "Diffraction effect correction" sections.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# record layout (mirrors the enum in rtw_oracle.h)
VALID, NF, ORIENT, NREFL, S, F, PSI, D, DGEO, J = 0, 1, 2, 3, 4, 7, 13, 14, 15, 16
V1, V2, REXIT, Q, E, DLEGS, NFLEGS, PATH, POWER, COSPROD, CAUSTIC = 20, 23, 26, 29, 33, 37, 38, 39, 40, 41, 42
NFIELD = 48
MASK_CAUSTIC, MASK_AXIAL, MASK_PO = 1, 2, 4
FIELD_PO, FIELD_EXACT, FIELD_EXACT_FOLDS = 1, 2, 4


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/liboracle.so`` (plain C, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rtw_oracle.h"))
    ):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.or_object_size.restype = i
        L.or_make_object.argtypes = [p, p]
        L.or_make_object.restype = i
        L.or_fan_halfwidth.argtypes = [p, d]
        L.or_fan_halfwidth.restype = d
        L.or_square_grid.argtypes = [p, i64, d, p, p, p, p, p]
        L.or_caustic_cap.argtypes = [p]
        L.or_caustic_cap.restype = d
        L.or_trace_ray.argtypes = [p, d, d, i, p, p]
        L.or_trace_ray.restype = i
        L.or_trace_rays.argtypes = [p, p, i64, i, p, i]
        L.or_field_fan.argtypes = [p, i64, d, i, p, i64, i, p, p]
        L.or_field_fan.restype = i
        L.or_field_grid.argtypes = [p, i64, d, i, i, i, p, i, p, p, i, p]
        L.or_field_grid.restype = i64
        L.or_newton.argtypes = [p, i, p, p, d, p]
        L.or_newton.restype = i
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Object:
    """One ellipsoid in a plane wave along +z (host medium index 1)."""

    def __init__(self, a, b, c, quat=(1.0, 0.0, 0.0, 0.0), center=(0.0, 0.0, 0.0), m=1.333,
                 wavelength=0.6328, jones=(1.0, 0.0)):
        L = lib()
        j = [complex(x) for x in jones]
        self.params = np.array([a, b, c, *quat, *center, m, wavelength,
                                j[0].real, j[0].imag, j[1].real, j[1].imag], dtype=np.float64)
        self._buf = ctypes.create_string_buffer(L.or_object_size())
        if L.or_make_object(_ptr(self.params), self._buf) != 0:
            raise ValueError("invalid object parameters")
        self.a, self.b, self.c = float(a), float(b), float(c)
        self.m, self.wavelength = float(m), float(wavelength)
        self.center = np.array(center, dtype=np.float64)
        self.k0 = 2 * np.pi / self.wavelength

    @property
    def handle(self):
        return ctypes.cast(self._buf, ctypes.c_void_p)

    def trace_ray(self, x, y, pmax):
        out = np.zeros((pmax + 1, NFIELD))
        pin = np.zeros(1)
        hit = lib().or_trace_ray(self.handle, float(x), float(y), int(pmax), _ptr(out), _ptr(pin))
        return out, float(pin[0]), bool(hit)

    def trace_rays(self, xy, pmax, threads=0):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        out = np.zeros((xy.shape[0], pmax + 1, NFIELD))
        lib().or_trace_rays(self.handle, _ptr(xy), xy.shape[0], int(pmax), _ptr(out), int(threads))
        return out

    def fan_halfwidth(self, fan_phi=0.0):
        return lib().or_fan_halfwidth(self.handle, float(fan_phi))

    def fan_impacts(self, nrays, fan_phi=0.0):
        w = self.fan_halfwidth(fan_phi)
        b = -w + (np.arange(nrays) + 0.5) * (2 * w / nrays)
        return b, self.center[0] + b * np.cos(fan_phi), self.center[1] + b * np.sin(fan_phi)

    def square_grid(self, n_target=0, h=0.0):
        hh, xc, yc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        nx, ny = ctypes.c_int64(), ctypes.c_int64()
        lib().or_square_grid(self.handle, int(n_target), float(h), ctypes.byref(hh), ctypes.byref(nx),
                             ctypes.byref(ny), ctypes.byref(xc), ctypes.byref(yc))
        return hh.value, nx.value, ny.value, xc.value, yc.value

    def caustic_cap(self):
        return lib().or_caustic_cap(self.handle)

    def field_fan(self, nrays, alpha, pmax, fan_phi=0.0, flags=0):
        alpha = np.ascontiguousarray(alpha, dtype=np.float64)
        out = np.zeros((alpha.size, pmax + 1, 4))
        mask = np.zeros(alpha.size, dtype=np.uint8)
        rc = lib().or_field_fan(self.handle, int(nrays), float(fan_phi), int(pmax), _ptr(alpha), alpha.size,
                                int(flags), _ptr(out), _ptr(mask))
        if rc != 0:
            raise RuntimeError("or_field_fan failed")
        return out, mask

    def field_grid(self, pmax, ntheta, nphi, n_target=0, h=0.0, window=None, flags=0, threads=0):
        out = np.zeros((ntheta * nphi, pmax + 1, 4))
        mask = np.zeros(ntheta * nphi, dtype=np.uint8)
        nfail = ctypes.c_int64(0)
        win = None if window is None else np.ascontiguousarray(window, dtype=np.int64)
        hits = lib().or_field_grid(self.handle, int(n_target), float(h), int(pmax), int(ntheta), int(nphi),
                                   None if win is None else _ptr(win), int(flags), _ptr(out), _ptr(mask),
                                   int(threads), ctypes.byref(nfail))
        if hits < 0:
            raise RuntimeError("or_field_grid failed")
        return out, mask, int(hits), int(nfail.value)

    def newton(self, p, target, xy, rmax=0.0):
        target = np.ascontiguousarray(target, dtype=np.float64)
        xy = np.array(xy, dtype=np.float64)
        rec = np.zeros(NFIELD)
        it = lib().or_newton(self.handle, int(p), _ptr(target), _ptr(xy), float(rmax), _ptr(rec))
        return it, xy, rec


def complex_field(out):
    """(..., 4) -> complex (..., 2) = (F_theta, F_phi)."""
    return out[..., 0::2] + 1j * out[..., 1::2]
