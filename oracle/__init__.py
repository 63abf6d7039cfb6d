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
_SRCS = [_SRC, os.path.join(_HERE, "mlp_oracle.c")]
_HDRS = [os.path.join(_HERE, "rtw_oracle.h"), os.path.join(_HERE, "mlp_oracle.h")]
_LIB = os.path.join(_HERE, "liboracle.so")

# record layout (mirrors the enum in rtw_oracle.h)
VALID, NF, ORIENT, NREFL, S, F, PSI, D, DGEO, J = 0, 1, 2, 3, 4, 7, 13, 14, 15, 16
V1, V2, REXIT, Q, E, DLEGS, NFLEGS, PATH, POWER, COSPROD, CAUSTIC = 20, 23, 26, 29, 33, 37, 38, 39, 40, 41, 42
NFIELD = 48
MASK_CAUSTIC, MASK_AXIAL, MASK_PO = 1, 2, 4
FIELD_PO, FIELD_EXACT, FIELD_EXACT_FOLDS = 1, 2, 4


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/liboracle.so`` (plain C, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS + _HDRS):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-fopenmp", "-o", tmp, *_SRCS, "-lm"]
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
        L.or_field_grid_counts.argtypes = [p, i64, d, i, i, i, i, p, p, p, i, p]
        L.or_field_grid_counts.restype = i64
        L.or_field_dirs.argtypes = [p, i64, d, i, p, i64, i, p, p, i, p]
        L.or_field_dirs.restype = i64
        L.or_near_record.argtypes = [p, p, d, p]
        L.or_near_record.restype = i
        L.or_field_sphere.argtypes = [p, i64, d, i, i, i, d, p, p, i]
        L.or_field_sphere.restype = i64
        L.or_field_po2d.argtypes = [p, i64, d, i, p, d, d, d, d, p, i64, p]
        L.or_field_po2d.restype = i64
        L.or_field_grid_caustic.argtypes = [p, i64, d, i, i, i, p, p, p, p, p, p, i]
        L.or_field_grid_caustic.restype = i64
        L.or_newton.argtypes = [p, i, p, p, d, p]
        L.or_newton.restype = i
        L.om_gelu.argtypes = [d]
        L.om_gelu.restype = d
        L.om_gelu_grad.argtypes = [d]
        L.om_gelu_grad.restype = d
        L.om_round_bf16.argtypes = [d]
        L.om_round_bf16.restype = d
        L.om_features.argtypes = [p, p, p]
        L.om_xy_to_uv.argtypes = [p, d, d, p]
        L.om_uv_to_xy.argtypes = [p, p, p, p]
        L.om_forward.argtypes = [p, p, i64, i, p]
        L.om_loss_grad.argtypes = [p, p, p, p, i64, d, i, p]
        L.om_loss_grad.restype = d
        L.om_adam.argtypes = [p, p, p, p, i64, i, d, d, d, d]
        L.or_field_learned.argtypes = [p, p, i, i, i, d, i, d, i, p, p, p]
        L.or_field_learned.restype = i64
        L.or_field_learned_dirs.argtypes = [p, p, i, p, i64, d, i, d, i, p, p, p]
        L.or_field_learned_dirs.restype = i64
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Object:
    """One ellipsoid in a plane wave along +z (host medium index 1)."""

    def __init__(self, a, b, c, quat=(1.0, 0.0, 0.0, 0.0), center=(0.0, 0.0, 0.0), m=1.333,
                 wavelength=0.6328, jones=(1.0, 0.0), source=None, shape_e=1.0):
        """source: None for a plane wave along +z, else the point source's position (um).
        shape_e: superellipsoid exponent e >= 1 (surface sum |u_i|^(2e) = 1), 1 for the ellipsoid."""
        L = lib()
        j = [complex(x) for x in jones]
        src = (0.0, 0.0, 0.0, 0.0) if source is None else (1.0, *source)
        self.params = np.array([a, b, c, *quat, *center, m, wavelength,
                                j[0].real, j[0].imag, j[1].real, j[1].imag, *src, shape_e], dtype=np.float64)
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

    def field_po2d(self, p, window, dirs, aperture_dir, cone, n_target=0, h=0.0):
        """2-D physical-optics field of order p over the rays of a vertex window of the square grid:
        aperture plane through the centre with normal aperture_dir = (theta, phi), rays weighted by
        the angle of their exit direction to that normal (1 up to cone[0], 0 from cone[1]);
        dirs: (n, 2) (theta, phi).  Returns (n, 2) complex (F_theta, F_phi) and the rays summed."""
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 2)
        win = np.ascontiguousarray(window, dtype=np.int64)
        out = np.zeros((dirs.shape[0], 4))
        used = lib().or_field_po2d(self.handle, int(n_target), float(h), int(p), _ptr(win), float(aperture_dir[0]),
                                   float(aperture_dir[1]), float(cone[0]), float(cone[1]), _ptr(dirs),
                                   dirs.shape[0], _ptr(out))
        if used < 0:
            raise ValueError("invalid aperture window or cone")
        return complex_field(out), int(used)

    def caustic_defaults(self):
        """Widths of the caustic correction of an object of largest semi-axis L: the Airy width
        Aw = (lambda / L)^(2/3) and the Fresnel width Fw = 1 / sqrt(k0 L) set po_full = 1.5 Aw,
        po_end = 3 Aw, cone_full = 3 Aw + 3 Fw and cone_end = 3 Aw + 6 Fw (the fan's constants)."""
        L = max(self.a, self.b, self.c)
        aw = (self.wavelength / L) ** (2.0 / 3.0)
        fw = 1.0 / np.sqrt(self.k0 * L)
        return dict(po_full=1.5 * aw, po_end=3.0 * aw, cone_full=3.0 * aw + 3.0 * fw, cone_end=3.0 * aw + 6.0 * fw)

    def field_grid_caustic(self, pmax, ntheta, nphi, tile=(16, 16), po_full=None, po_end=None, cone_full=None,
                           cone_end=None, p_min=1, n_target=0, h=0.0, threads=0):
        """or_field_grid_caustic: the square-grid field with the 2-D physical optics of the caustics
        blended in.  Widths left None take caustic_defaults().  Returns (out (ndir, pmax+1, 4), mask,
        weights (ndir, pmax+1), caustic orders (ndir uint32, bit p), l1 (ndir, pmax+1), hits)."""
        dflt = self.caustic_defaults()
        w = [dflt[k] if v is None else v for k, v in (("po_full", po_full), ("po_end", po_end),
                                                       ("cone_full", cone_full), ("cone_end", cone_end))]
        cp = np.array([tile[0], tile[1], *w, p_min], dtype=np.float64)
        nd = ntheta * nphi
        out = np.zeros((nd, pmax + 1, 4))
        mask = np.zeros(nd, dtype=np.uint8)
        weights = np.zeros((nd, pmax + 1))
        corders = np.zeros(nd, dtype=np.uint32)
        l1 = np.zeros((nd, pmax + 1))
        hits = lib().or_field_grid_caustic(self.handle, int(n_target), float(h), int(pmax), int(ntheta), int(nphi),
                                           _ptr(cp), _ptr(out), _ptr(mask), _ptr(weights), _ptr(corders), _ptr(l1),
                                           int(threads))
        if hits == -2:
            raise ValueError("a tile's cone reaches 90 degrees from its aperture normal")
        if hits < 0:
            raise RuntimeError("or_field_grid_caustic failed")
        return out, mask, weights, corders, l1, int(hits)

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

    def field_grid_counts(self, pmax, ntheta, nphi, n_target=0, h=0.0, flags=0, threads=0):
        """or_field_grid over every cell, with the number of hits per (direction, order): with
        FIELD_EXACT, the exact branches found (bit 0x80: a hit whose Newton step failed)."""
        out = np.zeros((ntheta * nphi, pmax + 1, 4))
        mask = np.zeros(ntheta * nphi, dtype=np.uint8)
        counts = np.zeros((ntheta * nphi, pmax + 1), dtype=np.uint8)
        nfail = ctypes.c_int64(0)
        hits = lib().or_field_grid_counts(self.handle, int(n_target), float(h), int(pmax), int(ntheta), int(nphi),
                                          int(flags), _ptr(out), _ptr(mask), _ptr(counts), int(threads),
                                          ctypes.byref(nfail))
        if hits < 0:
            raise RuntimeError("or_field_grid_counts failed")
        return out, mask, counts, int(nfail.value)

    def field_learned(self, theta, pmax, ntheta, nphi, p_min=0.05, max_steps=5, tol=0.0, max_halvings=3):
        """theta: (pmax+1) x MLP_NPARAM network parameters; each head's Newton steps are halved at
        most max_halvings times; returns out, mask, root counts."""
        theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(pmax + 1, -1)
        ndir = ntheta * nphi
        out = np.zeros((ndir, pmax + 1, 4))
        mask = np.zeros(ndir, dtype=np.uint8)
        roots = np.zeros((ndir, pmax + 1), dtype=np.uint8)
        lib().or_field_learned(self.handle, _ptr(theta), int(pmax), int(ntheta), int(nphi), float(p_min),
                               int(max_steps), float(tol), int(max_halvings), _ptr(out), _ptr(mask), _ptr(roots))
        return out, mask, roots

    def field_learned_dirs(self, theta, pmax, dirs, p_min=0.05, max_steps=5, tol=0.0, max_halvings=3):
        """The learned field on a list of directions dirs (n x 2: theta, phi)."""
        theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(pmax + 1, -1)
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 2)
        ndir = dirs.shape[0]
        out = np.zeros((ndir, pmax + 1, 4))
        mask = np.zeros(ndir, dtype=np.uint8)
        roots = np.zeros((ndir, pmax + 1), dtype=np.uint8)
        lib().or_field_learned_dirs(self.handle, _ptr(theta), int(pmax), _ptr(dirs), ndir, float(p_min),
                                    int(max_steps), float(tol), int(max_halvings), _ptr(out), _ptr(mask), _ptr(roots))
        return out, mask, roots

    def near_record(self, rec, R):
        """One order's record (NFIELD doubles) at the ray's crossing with the sphere |M| = R."""
        rec = np.ascontiguousarray(rec, dtype=np.float64)
        out = np.zeros(NFIELD)
        ok = lib().or_near_record(self.handle, _ptr(rec), float(R), _ptr(out))
        return out, bool(ok)

    def field_sphere(self, pmax, ntheta, nphi, R, n_target=0, h=0.0, threads=0):
        """The field on the sphere of radius R at the cell-centred (theta, phi) grid points:
        out is ndir x (pmax+1) x 6 (E_r, E_theta, E_phi as re, im), dimensionless."""
        out = np.zeros((ntheta * nphi, pmax + 1, 6))
        mask = np.zeros(ntheta * nphi, dtype=np.uint8)
        hits = lib().or_field_sphere(self.handle, int(n_target), float(h), int(pmax), int(ntheta), int(nphi),
                                     float(R), _ptr(out), _ptr(mask), int(threads))
        if hits < 0:
            raise ValueError("or_field_sphere: R must enclose the object")
        return out, mask, int(hits)

    def field_dirs(self, pmax, dirs, n_target=0, h=0.0, flags=0, threads=0):
        """The square-grid field on a list of directions dirs (n x 2: theta, phi)."""
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 2)
        out = np.zeros((dirs.shape[0], pmax + 1, 4))
        mask = np.zeros(dirs.shape[0], dtype=np.uint8)
        nfail = ctypes.c_int64(0)
        hits = lib().or_field_dirs(self.handle, int(n_target), float(h), int(pmax), _ptr(dirs), dirs.shape[0],
                                   int(flags), _ptr(out), _ptr(mask), int(threads), ctypes.byref(nfail))
        if hits < 0:
            raise RuntimeError("or_field_dirs failed")
        return out, mask, int(hits), int(nfail.value)

    def newton(self, p, target, xy, rmax=0.0):
        target = np.ascontiguousarray(target, dtype=np.float64)
        xy = np.array(xy, dtype=np.float64)
        rec = np.zeros(NFIELD)
        it = lib().or_newton(self.handle, int(p), _ptr(target), _ptr(xy), float(rmax), _ptr(rec))
        return it, xy, rec


def complex_field(out):
    """(..., 2k) -> complex (..., k): (F_theta, F_phi), or (E_r, E_theta, E_phi) on a sphere."""
    return out[..., 0::2] + 1j * out[..., 1::2]


# ------------------------------------------------------------------------------------------------
# learned inverse-map proposal (mlp_oracle.c)
# ------------------------------------------------------------------------------------------------
MLP_IN, MLP_H, MLP_OUT, MLP_HEADS = 16, 128, 16, 4
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_OUT * MLP_H + MLP_OUT


def mlp_features(obj: Object, s):
    s = np.ascontiguousarray(np.atleast_2d(s), dtype=np.float64)
    out = np.zeros((s.shape[0], MLP_IN))
    for i in range(s.shape[0]):
        lib().om_features(obj.handle, _ptr(s[i]), _ptr(out[i]))
    return out


def xy_to_uv(obj: Object, x, y):
    uv = np.zeros(2)
    lib().om_xy_to_uv(obj.handle, float(x), float(y), _ptr(uv))
    return uv


def uv_to_xy(obj: Object, uv):
    uv = np.ascontiguousarray(uv, dtype=np.float64)
    x, y = ctypes.c_double(), ctypes.c_double()
    lib().om_uv_to_xy(obj.handle, _ptr(uv), ctypes.byref(x), ctypes.byref(y))
    return x.value, y.value


def mlp_forward(theta, x, bf16=False):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    y = np.zeros((x.shape[0], MLP_OUT))
    lib().om_forward(_ptr(theta), _ptr(x), x.shape[0], int(bf16), _ptr(y))
    return y


def mlp_loss_grad(theta, x, target, valid, beta=0.1, bf16=False):
    """valid: per-row label, 0 = ignored, 1..4 = head label - 1 carries the target."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    target = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 2)
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    g = np.zeros(MLP_NPARAM)
    loss = lib().om_loss_grad(_ptr(theta), _ptr(x), _ptr(target), _ptr(valid), x.shape[0], float(beta), int(bf16),
                              _ptr(g))
    return loss, g


def mlp_adam(theta, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on theta, m, v (float64 arrays)."""
    lib().om_adam(_ptr(theta), _ptr(m), _ptr(v), _ptr(np.ascontiguousarray(grad, dtype=np.float64)), theta.size,
                  int(t), float(lr), float(b1), float(b2), float(eps))


def gelu(z):
    return lib().om_gelu(float(z))


def gelu_grad(z):
    return lib().om_gelu_grad(float(z))


def round_bf16(v):
    return lib().om_round_bf16(float(v))
