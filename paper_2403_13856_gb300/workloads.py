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

# Table 1 of the paper: spheres of radius 50 and 500 um, order p = 2, perpendicular polarisation.
TABLE1_SPHERES = (50.0, 500.0)
