"""Pins of the oracle's 2-D physical-optics aperture integral (or_field_po2d).

Near a caustic the ray sum fails and the paper replaces it by a diffraction integral of the complex
amplitudes the rays carry ("Diffraction effect correction based on VCRM").  The oracle's 1-D form
(a fan through a symmetry plane, the sagittal direction integrated by stationary phase) is pinned by
Table 1; the 2-D form integrates both directions numerically over a plane.  Its pins:

* the sphere's rainbow (order 2, perpendicular polarisation): the 2-D integral reproduces the 1-D PO
  field and the main bow of Table 1 (a = 50 and 500 um);
* away from caustics, stationary phase reduces it to the exact ray field (order 1 of a tilted
  ellipsoid, polarisation mixed).
"""
import math
import os

import numpy as np
import pytest

M_WATER = 1.333
LAM = 0.6328


def table1_main_bow(a):
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_rainbow_peaks.txt")
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            at, k, th = line.split()
            if float(at) == a and int(k) == 0:
                return float(th)
    raise KeyError(a)


def peak_positions(th, I):
    out = []
    for i in range(1, len(I) - 1):
        if I[i] > I[i - 1] and I[i] >= I[i + 1]:
            y0, y1, y2 = I[i - 1], I[i], I[i + 1]
            out.append(th[i] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * (th[1] - th[0]))
    return np.array(out)


@pytest.mark.parametrize("a,h,nfan", [(50.0, 0.1, 8000), (500.0, 0.25, 40000)])
def test_po2d_rainbow_matches_fan_po_and_table1(oracle_mod, a, h, nfan):
    """Order 2 of a sphere in the plane phi = 0, from 0.4 Airy widths inside the rainbow to 1.5
    outside (where the 1-D PO is used alone): the 2-D aperture over the left half of the ray grid,
    plane normal along the rainbow ray, rays tapered like the 1-D window (3 Airy + 3 Fresnel
    widths, to zero at + 6 Fresnel widths), against the 1-D PO intensity within 1e-2 (L2) and the
    main bow of Table 1 within 0.02 deg."""
    o = oracle_mod.Object(a, a, a, m=M_WATER, wavelength=LAM, jones=(0.0, 1.0))
    Aw, Fw = (LAM / a) ** (2.0 / 3.0), 1.0 / math.sqrt(o.k0 * a)
    thc = math.radians(137.922)  # the rainbow ray of m = 1.333 (minimum deviation)
    th = thc + np.linspace(-0.4 * Aw, 1.5 * Aw, 200)
    fan, _ = o.field_fan(nfan, th, 2, flags=oracle_mod.FIELD_PO)
    Ifan = np.abs(oracle_mod.complex_field(fan[:, 2, :])[:, 1]) ** 2
    _, nx, ny, _, _ = o.square_grid(h=h)
    dirs = np.stack([th, np.zeros_like(th)], 1)
    F, used = o.field_po2d(2, [0, nx // 2, 0, ny - 1], dirs, (thc, 0.0), (3 * Aw + 3 * Fw, 3 * Aw + 6 * Fw), h=h)
    assert used > 100_000
    I = np.abs(F[:, 1]) ** 2
    assert np.abs(F[:, 0]).max() < 1e-6 * np.abs(F[:, 1]).max()  # perpendicular polarisation stays so
    rel = np.linalg.norm(I - Ifan) / np.linalg.norm(Ifan)
    assert rel < 1e-2, rel
    pk = np.degrees(peak_positions(th, I))
    assert pk[0] == pytest.approx(table1_main_bow(a), abs=0.02)


def test_po2d_go_limit(oracle_mod):
    """Order 1 of a tilted ellipsoid, nine directions around one ray's exit direction: with an
    aperture of several Fresnel zones the integral equals the exact ray field within 1e-2, and a
    narrower aperture is visibly worse (the integral converges to the ray, it is not the ray)."""
    o = oracle_mod.Object(50.0, 40.0, 30.0, quat=(0.9, 0.25, -0.3, 0.15), m=M_WATER, wavelength=LAM,
                          jones=(0.6, 0.8j))
    h = 0.1
    _, nx, ny, _, _ = o.square_grid(h=h)
    rec, _, hit = o.trace_ray(10.0, 5.0, 1)
    assert hit
    s0 = rec[1, oracle_mod.S:oracle_mod.S + 3]
    th0, ph0 = math.acos(s0[2]), math.atan2(s0[1], s0[0])
    dirs = np.array([[th0 + dt, ph0 + dp] for dt in (-0.01, 0.0, 0.01) for dp in (-0.01, 0.0, 0.01)])
    out, _, _, nfail = o.field_dirs(1, dirs, h=h, flags=oracle_mod.FIELD_EXACT)
    assert nfail == 0
    G = oracle_mod.complex_field(out[:, 1, :])
    win = [0, nx - 1, 0, ny - 1]
    F, _ = o.field_po2d(1, win, dirs, (th0, ph0), (0.2, 0.35), h=h)
    err = np.abs(F - G).max() / np.abs(G).max()
    assert err < 1e-2, err
    Fn, _ = o.field_po2d(1, win, dirs, (th0, ph0), (0.05, 0.1), h=h)
    assert np.abs(Fn - G).max() / np.abs(G).max() > 5 * err


def test_po2d_arguments(oracle_mod):
    o = oracle_mod.Object(10.0, 10.0, 10.0, m=M_WATER, wavelength=LAM)
    _, nx, ny, _, _ = o.square_grid(h=0.5)
    d = np.array([[2.4, 0.0]])
    with pytest.raises(ValueError):  # beyond the grid
        o.field_po2d(2, [0, nx, 0, ny - 1], d, (2.4, 0.0), (0.1, 0.2), h=0.5)
    with pytest.raises(ValueError):  # cone_end must exceed cone_full
        o.field_po2d(2, [0, nx - 1, 0, ny - 1], d, (2.4, 0.0), (0.2, 0.1), h=0.5)
