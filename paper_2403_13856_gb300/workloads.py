"""Synthetic inputs of the RTW workloads: object descriptions, ray and direction grids, seeds.

This module holds input parameters only (no step of the method).  Both the CUDA path and the
FP64 oracle read their inputs from here.  The objects follow the scattering configurations of the
paper (water drops, lambda = 0.6328 um, Figs. 3-4 and Table 1) at the sizes of the benchmark.
"""
from __future__ import annotations

import math

WATER = 1.333
HE_NE = 0.6328  # um


def quat_about_x(deg: float):
    """Unit quaternion (w, x, y, z) of an active rotation by `deg` degrees about +x."""
    h = math.radians(deg) / 2.0
    return (math.cos(h), math.sin(h), 0.0, 0.0)


# Sphere, radius 10 um: fan of 1e4 rays uniform in impact parameter, orders 0..3, 1801 scattering
# angles 0..180 deg (0.1 deg) in the plane phi = 0, s (E along y) and p (E along x) polarisation.
SPHERE10 = dict(a=10.0, b=10.0, c=10.0, quat=(1.0, 0.0, 0.0, 0.0), m=WATER, wavelength=HE_NE)
SPHERE10_FAN = dict(n_rays=10_000, p_max=3, n_dirs=1801, alpha0=0.0, dalpha=math.radians(0.1))

# Ellipsoidal drop (120, 100, 80) um tilted 20 deg about x, x polarisation, orders 0..5, about
# 4e6 rays on a square grid over the projected cross-section, 512 x 1024 (theta, phi) directions.
ELLIPSOID = dict(a=120.0, b=100.0, c=80.0, quat=quat_about_x(20.0), m=WATER, wavelength=HE_NE)
ELLIPSOID_GRID = dict(n_rays=4_000_000, p_max=5, n_theta=512, n_phi=1024)


# Oblate spheroid a = b = 100, c = 90 um lit along its x axis (the spheroid of the paper's Fig. 3
# setting): the incident wave travels along +z, so the body is turned by -90 deg about y, which
# carries its x axis onto z.
SPHEROID_SIDE = dict(a=100.0, b=100.0, c=90.0, quat=(math.cos(math.radians(-45.0)), 0.0, math.sin(math.radians(-45.0)), 0.0),
                     m=WATER, wavelength=HE_NE)
# its 3-D pattern at 0.01 deg over the whole sphere of directions: 4e6 rays, orders 0..5
SPHEROID_PATTERN = dict(n_rays=4_000_000, p_max=5, n_theta=18_000, n_phi=36_000)


def unit_quat(w: float, x: float, y: float, z: float):
    n = math.sqrt(w * w + x * x + y * y + z * z)
    return (w / n, x / n, y / n, z / n)


# Superellipsoid |u|^4 + |v|^4 + |w|^4 = 1 (e = 2) on the drop's semi-axes (120, 100, 80) um,
# turned about all three axes; the same grid sizes as the ellipsoid (the ray count is taken
# inside the silhouette of the bounding ellipsoid, 3^(1/4) times the semi-axes).
SUPERELLIPSOID = dict(a=120.0, b=100.0, c=80.0, quat=unit_quat(0.9, 0.25, -0.3, 0.15), m=WATER,
                      wavelength=HE_NE, shape_e=2.0)

# Table 1 of the paper: spheres of radius 50 and 500 um, order p = 2, perpendicular polarisation.
TABLE1_SPHERES = (50.0, 500.0)

# ------------------------------------------------------------------------------------------------
# Batched drops: seed-drawn ellipsoids of uneven size, shape, orientation, index and wavelength.
# Counter-based Philox generator keyed by (master seed, stream), one stream per purpose.
# ------------------------------------------------------------------------------------------------
MASTER_SEED = 2403138560
STREAM_BATCH = 1
STREAM_TRAIN = 2
STREAM_EVAL = 3

# 4096 ellipsoids: r0 ~ U[20, 500] um, b, c = r0 U[0.8, 1.2], uniform orientation, m ~ U[1.33, 1.55],
# lambda ~ U[0.4, 0.8] um, x polarisation, rays clamp(1e6 (r0 / 500)^2, 1e3, 1e6), orders 0..4,
# 128 x 256 (theta, phi) directions per object.
BATCH = dict(n_objects=4096, r0=(20.0, 500.0), aspect=(0.8, 1.2), m=(1.33, 1.55), wavelength=(0.4, 0.8),
             rays_ref=(1e6, 500.0), rays_clamp=(1_000, 1_000_000), p_max=4, n_theta=128, n_phi=256)


def philox(stream: int):
    """numpy Generator on the Philox-4x64 bit generator keyed by (MASTER_SEED, stream)."""
    import numpy as np

    return np.random.Generator(np.random.Philox(key=np.array([MASTER_SEED, stream], dtype=np.uint64)))


def shoemake_quaternions(u):
    """Uniform random unit quaternions (w, x, y, z) from uniforms u (n x 3) (Shoemake's method)."""
    import numpy as np

    u1, u2, u3 = u[:, 0], u[:, 1], u[:, 2]
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3),
                  b * np.cos(2 * np.pi * u3)], axis=1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def batch_objects(n_objects=None, stream=STREAM_BATCH, r0=None, rays_ref=None, rays_clamp=None):
    """Object specs (dicts of a, b, c, quat, m, wavelength) and ray counts of the batched workload.
    r0, rays_ref = (rays, at radius) and rays_clamp override the size recipe (small test batches)."""
    import numpy as np

    n = BATCH["n_objects"] if n_objects is None else int(n_objects)
    lo, hi = BATCH["r0"] if r0 is None else r0
    nref, rref = BATCH["rays_ref"] if rays_ref is None else rays_ref
    cmin, cmax = BATCH["rays_clamp"] if rays_clamp is None else rays_clamp
    g = philox(stream)
    u = g.random((n, 9))
    r = lo + (hi - lo) * u[:, 0]
    b = r * (BATCH["aspect"][0] + (BATCH["aspect"][1] - BATCH["aspect"][0]) * u[:, 1])
    c = r * (BATCH["aspect"][0] + (BATCH["aspect"][1] - BATCH["aspect"][0]) * u[:, 2])
    q = shoemake_quaternions(u[:, 3:6])
    m = BATCH["m"][0] + (BATCH["m"][1] - BATCH["m"][0]) * u[:, 6]
    lam = BATCH["wavelength"][0] + (BATCH["wavelength"][1] - BATCH["wavelength"][0]) * u[:, 7]
    rays = np.clip(np.rint(nref * (r / rref) ** 2), cmin, cmax).astype(np.int64)
    specs = [dict(a=float(r[i]), b=float(b[i]), c=float(c[i]), quat=tuple(float(x) for x in q[i]), m=float(m[i]),
                  wavelength=float(lam[i])) for i in range(n)]
    return specs, rays

# Learned proposal: networks for orders 0..4 trained on 2e7 rays traced through drops of the
# batched recipe (stream 2, entry points uniform on each projected section), evaluated on 1024
# further drops (stream 3) at 256 x 512 (theta, phi) directions each.
LEARNED = dict(n_objects=1024, n_theta=256, n_phi=512, p_max=4, train_objects=16384, train_rays=20_000_000,
               train_steps=20000, batch=8192)
