"""Pins of the oracle's physical optics at the 3-D caustics of a square-grid field
(or_field_grid_caustic).

The paper corrects the ray sum near caustics by a diffraction integral of the rays' complex amplitudes
("Diffraction effect correction based on VCRM") and leaves the 3-D form "under study"; the oracle's
reading blends a plane-aperture integral into each order's ray sum with a taper of the angle to the
directions that order's fold cells cover.  Its pins:

* the weights are that taper of the brute-force nearest caustic direction (all caustic directions,
  no pruning of rows);
* the blended field is (1 - s) F_rays + s F_PO, with F_rays from or_field_grid and F_PO from a call
  whose widths make the integral the whole field (s = 1);
* the masks: the caustic bit only where an order's caustic direction keeps s < 1, the PO bit where
  any s > 0;
* the sphere's rainbow (order 2, perpendicular polarisation, a = 50 um): in the plane phi = 0 the 3-D
  field reproduces the 1-D PO of the fan (which Table 1 pins) within 1.5e-2 in intensity from 0.4
  Airy widths inside the bow to 1.5 outside, and puts the main bow of Table 1 within 0.02 deg.
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


def unit(nt, nph):
    th = (np.arange(nt) + 0.5) * np.pi / nt
    ph = -np.pi + (np.arange(nph) + 0.5) * 2 * np.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)


def ramp(x, x0, x1):
    c = np.cos(0.5 * np.pi * (x - x0) / (x1 - x0)) ** 2
    return np.where(x <= x0, 1.0, np.where(x >= x1, 0.0, c))


@pytest.fixture(scope="module")
def small(oracle_mod):
    """A tilted ellipsoid, orders 0..3, a coarse (theta, phi) grid: the default widths and 8 x 4 tiles."""
    o = oracle_mod.Object(14.0, 11.0, 9.0, quat=(0.9, 0.25, -0.3, 0.15), m=M_WATER, wavelength=LAM, jones=(0.6, 0.8j))
    nt, nph = 90, 60
    res = o.field_grid_caustic(3, nt, nph, tile=(8, 4), h=0.12)
    return o, nt, nph, res


def test_weights_are_the_taper_of_the_nearest_caustic_direction(oracle_mod, small):
    o, nt, nph, (out, mask, w, corders, l1, hits) = small
    d = o.caustic_defaults()
    u = unit(nt, nph)
    assert hits > 0
    ncaustic = 0
    for p in range(4):
        c = np.nonzero((corders >> p) & 1)[0]
        if p == 0:
            assert np.all(w[:, 0] == 0.0)
            continue
        ncaustic += c.size
        if c.size == 0:
            assert np.all(w[:, p] == 0.0)
            continue
        ang = np.arccos(np.clip(u @ u[c].T, -1.0, 1.0)).min(1)
        want = np.where(ang < d["po_end"], ramp(ang, d["po_full"], d["po_end"]), 0.0)
        np.testing.assert_allclose(w[:, p], want, atol=1e-9)
    assert ncaustic > 0


def test_masks_follow_the_weights(oracle_mod, small):
    o, nt, nph, (out, mask, w, corders, l1, hits) = small
    left = corders.copy()
    for p in range(1, 4):
        left &= ~np.where(w[:, p] == 1.0, np.uint32(1 << p), np.uint32(0))
    assert np.array_equal((mask & oracle_mod.MASK_CAUSTIC) != 0, left != 0)
    assert np.array_equal((mask & oracle_mod.MASK_PO) != 0, (w > 0).any(1))
    # every caustic direction of a corrected order is covered with weight 1
    for p in range(1, 4):
        c = ((corders >> p) & 1) != 0
        assert np.all(w[c, p] == 1.0)


def test_blend_is_the_weighted_sum_of_rays_and_aperture(oracle_mod, small):
    """(1 - s) F_rays + s F_PO: F_rays from or_field_grid, F_PO from a call whose po widths cover every
    direction (s = 1), the same tiles and cones."""
    o, nt, nph, (out, mask, w, corders, l1, hits) = small
    d = o.caustic_defaults()
    rays, _, _, _ = o.field_grid(3, nt, nph, h=0.12)
    po, _, w1, _, _, _ = o.field_grid_caustic(3, nt, nph, tile=(8, 4), h=0.12, po_full=3.5, po_end=3.6)
    assert np.all(w1[:, 1:] == 1.0)
    want = rays.copy()
    for p in range(1, 4):
        s = w[:, p][:, None]
        want[:, p] = (1.0 - s) * rays[:, p] + s * po[:, p]
    scale = np.abs(rays).max()
    assert np.abs(out - want).max() <= 1e-12 * scale
    assert np.abs(out[:, 0] - rays[:, 0]).max() == 0.0  # order 0 untouched


def test_sphere_rainbow_matches_fan_po_and_table1(oracle_mod):
    """Order 2 of a 50 um sphere, perpendicular polarisation, the plane phi = 0 (the middle column of an
    odd phi grid), tiles one column wide so that the aperture normals lie in that plane."""
    a = 50.0
    o = oracle_mod.Object(a, a, a, m=M_WATER, wavelength=LAM, jones=(0.0, 1.0))
    nt, nph = 1800, 5
    out, mask, w, corders, l1, hits = o.field_grid_caustic(2, nt, nph, tile=(16, 1), h=0.1)
    th = (np.arange(nt) + 0.5) * np.pi / nt
    Aw = (LAM / a) ** (2.0 / 3.0)
    thc = math.radians(137.922)  # the rainbow ray of m = 1.333 (minimum deviation)
    sel = (th > thc - 0.4 * Aw) & (th < thc + 1.5 * Aw)
    col = nph // 2
    F = oracle_mod.complex_field(out.reshape(nt, nph, 3, 4)[:, col, 2])[sel]
    assert np.all(w.reshape(nt, nph, 3)[sel, col, 2] == 1.0)  # the PO alone
    fan, _ = o.field_fan(8000, th[sel], 2, flags=oracle_mod.FIELD_PO)
    Ffan = oracle_mod.complex_field(fan[:, 2, :])
    assert np.abs(F[:, 0]).max() < 1e-6 * np.abs(F[:, 1]).max()  # perpendicular polarisation stays so
    I, Ifan = np.abs(F[:, 1]) ** 2, np.abs(Ffan[:, 1]) ** 2
    rel = np.linalg.norm(I - Ifan) / np.linalg.norm(Ifan)
    assert rel < 1.5e-2, rel
    pk = np.degrees(peak_positions(th[sel], I))
    assert pk[0] == pytest.approx(table1_main_bow(a), abs=0.02)
    # the rainbow row is caustic for order 2 and no longer masked
    assert ((corders >> 2) & 1).sum() > 0
    assert not np.any(mask & oracle_mod.MASK_CAUSTIC & (((corders >> 2) & 1) != 0))


def test_caustic_arguments(oracle_mod):
    o = oracle_mod.Object(10.0, 10.0, 10.0, m=M_WATER, wavelength=LAM)
    with pytest.raises(RuntimeError):
        o.field_grid_caustic(2, 30, 20, tile=(0, 4), h=0.5)
    with pytest.raises(RuntimeError):
        o.field_grid_caustic(2, 30, 20, po_full=0.2, po_end=0.1, h=0.5)
    with pytest.raises(ValueError):  # a cone reaching 90 deg from its tile's normal
        o.field_grid_caustic(2, 30, 20, cone_full=1.2, cone_end=1.6, h=0.5)
    src = oracle_mod.Object(10.0, 10.0, 10.0, m=M_WATER, wavelength=LAM, source=(0.0, 0.0, -100.0))
    with pytest.raises(RuntimeError):
        src.field_grid_caustic(2, 30, 20, h=0.5)
