"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (``oracle/``) against something other than itself: a closed form,
an identity of physics, the paper's printed equations in their special case, brute-force finite
differences of the bare geometry, or the numbers printed in Table 1 of Ren et al., "Ray Theory
of Waves" (arXiv:2403.13856).  No GPU is needed.
"""
import math
import os

import numpy as np
import pytest

M_WATER = 1.333
LAM = 0.6328


def sphere(oracle_mod, a=10.0, m=M_WATER, jones=(0.0, 1.0), lam=LAM):
    return oracle_mod.Object(a, a, a, m=m, wavelength=lam, jones=jones)


def tilted_ellipsoid(oracle_mod, jones=(1.0, 0.0), scale=1.0):
    # semi-axes (120, 100, 80) um, active rotation of 20 degrees about x
    h = math.radians(20.0) / 2
    return oracle_mod.Object(120.0 * scale, 100.0 * scale, 80.0 * scale, quat=(math.cos(h), math.sin(h), 0, 0),
                             m=M_WATER, wavelength=LAM, jones=jones)


def rec_at(oracle_mod, obj, b, pmax=3):
    rec, pin, hit = obj.trace_ray(b, 0.0, pmax)
    assert hit
    return rec, pin


def fresnel_closed(i, m):
    """Textbook (Born & Wolf) amplitude coefficients from the angles, for the closed-form pins."""
    r = math.asin(math.sin(i) / m)
    ci, cr = math.cos(i), math.cos(r)
    rs = (ci - m * cr) / (ci + m * cr)
    return rs, r


# --------------------------------------------------------------------------------------------
# P1: Fresnel coefficients (Eq. Fres) -- energy, Brewster, normal incidence, TIR, Stokes
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("deg", [0.5, 30.0, 53.12, 60.0, 80.0, 89.0])
@pytest.mark.parametrize("jones", [(1.0, 0.0), (0.0, 1.0), (0.6, 0.8j)])
def test_single_interface_energy(oracle_mod, deg, jones):
    """R + T = 1 at the first interface: reflected power plus transmitted power (with its
    n cos(theta_t) / cos(theta_i) factor) equals the incident power."""
    o = sphere(oracle_mod, jones=jones)
    b = 10.0 * math.sin(math.radians(deg))
    rec, pin = rec_at(oracle_mod, o, b, pmax=0)
    total = rec[0, oracle_mod.POWER] + pin
    assert abs(total - 1.0) < 1e-14


def test_brewster_zero(oracle_mod):
    """r_par vanishes at tan(i_B) = m (the phase jump the paper attributes to Airy's failure)."""
    iB = math.atan(M_WATER)
    b = 10.0 * math.sin(iB)
    rec_par, _ = rec_at(oracle_mod, sphere(oracle_mod, jones=(1.0, 0.0)), b, pmax=0)
    rec_perp, _ = rec_at(oracle_mod, sphere(oracle_mod, jones=(0.0, 1.0)), b, pmax=0)
    assert rec_par[0, oracle_mod.POWER] < 1e-28
    assert rec_perp[0, oracle_mod.POWER] > 1e-2
    # sign change of r_par across Brewster: the reflected x-field flips sign
    f = []
    for d in (-1.0, 1.0):
        rec, _ = rec_at(oracle_mod, sphere(oracle_mod, jones=(1.0, 0.0)), 10.0 * math.sin(iB + d * 0.02), pmax=0)
        F = rec[0, oracle_mod.F:oracle_mod.F + 6:2]
        s = rec[0, oracle_mod.S:oracle_mod.S + 3]
        eth = np.array([s[2], 0.0, -s[0]])  # in-plane unit vector perpendicular to s
        f.append(float(F @ eth))
    assert f[0] * f[1] < 0


@pytest.mark.parametrize("jones", [(1.0, 0.0), (0.0, 1.0)])
def test_normal_incidence_isotropic(oracle_mod, jones):
    """At normal incidence the reflected field is r E_inc with r = (1-m)/(1+m) for any
    polarisation (r_par = -r_perp in the paper's convention, Eq. Fres)."""
    o = sphere(oracle_mod, jones=jones)
    rec, _ = rec_at(oracle_mod, o, 1e-9, pmax=0)
    F = rec[0, oracle_mod.F:oracle_mod.F + 6:2] + 1j * rec[0, oracle_mod.F + 1:oracle_mod.F + 6:2]
    r = (1 - M_WATER) / (1 + M_WATER)
    expect = r * math.sqrt(rec[0, oracle_mod.D]) * np.array([jones[0], jones[1], 0.0])
    assert np.allclose(F, expect, atol=1e-9, rtol=0)


def test_total_internal_reflection(oracle_mod):
    """An air bubble in water (m < 1): beyond the critical angle |r| = 1 for both polarisations
    and no transmitted ray exists."""
    for jones in [(1.0, 0.0), (0.0, 1.0), (0.6, 0.8)]:
        o = sphere(oracle_mod, m=1.0 / M_WATER, jones=jones)
        b = 10.0 * math.sin(math.radians(60.0))
        rec, pin, hit = o.trace_ray(b, 0.0, 3)
        assert abs(rec[0, oracle_mod.POWER] - 1.0) < 1e-14
        assert pin == 0.0
        assert np.all(rec[1:, oracle_mod.VALID] == 0)


@pytest.mark.parametrize("deg", [15.0, 45.0, 70.0])
def test_stokes_relations(oracle_mod, deg):
    """Time reversal fixes t t' = 1 - r^2 and r' = -r.  For a sphere the internal angle of every
    internal interaction equals the refraction angle, so the perpendicular Fresnel factors of
    Eq. (epsilon_VCRM) are eps_1 = 1 - r^2, eps_2 = -r (1 - r^2), eps_3 = r^2 (1 - r^2), with r
    read off the p = 0 ray."""
    o = sphere(oracle_mod, jones=(0.0, 1.0))
    b = 10.0 * math.sin(math.radians(deg))
    rec, _ = rec_at(oracle_mod, o, b, pmax=3)

    def eps(p):
        Fy = rec[p, oracle_mod.F + 2] + 1j * rec[p, oracle_mod.F + 3]
        nf = int(rec[p, oracle_mod.NF])
        return Fy / (math.sqrt(rec[p, oracle_mod.D]) * (-1j) ** nf)

    r = eps(0)
    assert abs(r.imag) < 1e-15
    rs, _ = fresnel_closed(math.radians(deg), M_WATER)
    assert abs(r.real - rs) < 1e-14
    assert abs(eps(1) - (1 - r * r)) < 1e-14
    assert abs(eps(2) - (-r * (1 - r * r))) < 1e-14
    assert abs(eps(3) - (r * r * (1 - r * r))) < 1e-14


# --------------------------------------------------------------------------------------------
# P2: the wavefront equation reduces to Synge's relations, Eqs. (1)-(2), in a symmetric plane
# --------------------------------------------------------------------------------------------

def synge_chain(i, m, a, pmax):
    """Principal WFC of the exit wave of each order, from Eqs. (1)-(2) of the paper with the
    sphere's data (rho_1 = rho_2 = a, outward normal, signed normal components) and free
    propagation 1/R -> 1/(R + d) along the chords.  Returns [(1/R_1, 1/R_2)] per order."""
    r = math.asin(math.sin(i) / m)
    ci, cr = math.cos(i), math.cos(r)
    k0 = 1.0
    out = []
    # p = 0: reflection outside, k_in = -k0 ci, k_ln = +k0 ci
    kin, kln = -k0 * ci, k0 * ci
    out.append(((kln - kin) / a / k0, (kln - kin) / a * k0 / (kln * kln)))
    # entry refraction: k_i = k0, k_r = m k0, k_rn = -m k0 cr
    kin, krn, ki, kr = -k0 * ci, -m * k0 * cr, k0, m * k0
    q1 = (krn - kin) / a / kr
    q2 = (krn - kin) / a * kr / (krn * krn)
    d = 2 * a * cr
    for p in range(1, pmax + 1):
        q1, q2 = q1 / (1 + d * q1), q2 / (1 + d * q2)
        # exit refraction: k_i = m k0 with k_in = m k0 cr (outward), k_r = k0 with k_rn = k0 ci
        kin, ki = m * k0 * cr, m * k0
        krn, kr = k0 * ci, k0
        e1 = (ki * q1 + (krn - kin) / a) / kr
        e2 = (kin * kin / ki * q2 + (krn - kin) / a) * kr / (krn * krn)
        out.append((e1, e2))
        # internal reflection: k_ln = -m k0 cr
        kln = -m * k0 * cr
        q1 = (ki * q1 + (kln - kin) / a) / ki
        q2 = (kin * kin / ki * q2 + (kln - kin) / a) * ki / (kln * kln)
    return out


@pytest.mark.parametrize("deg", [10.0, 45.0, 62.0, 80.0])
def test_synge_reduction(oracle_mod, deg):
    a = 10.0
    o = sphere(oracle_mod, a=a)
    b = a * math.sin(math.radians(deg))
    rec, _ = rec_at(oracle_mod, o, b, pmax=3)
    ref = synge_chain(math.radians(deg), M_WATER, a, 3)
    for p in range(4):
        Q = rec[p, oracle_mod.Q:oracle_mod.Q + 4].reshape(2, 2)
        # basis v1 is the normal of the incident plane (Synge index 1), v2 lies in it (index 2)
        assert abs(Q[0, 1]) < 1e-13 and abs(Q[1, 0]) < 1e-13
        assert Q[0, 0] == pytest.approx(ref[p][0], rel=1e-11, abs=1e-14)
        assert Q[1, 1] == pytest.approx(ref[p][1], rel=1e-11, abs=1e-14)


# --------------------------------------------------------------------------------------------
# P3/P4: sphere closed forms of geometric optics
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("deg", [5.0, 30.0, 60.0, 85.0])
def test_sphere_reflection_cross_section(oracle_mod, deg):
    """p = 0: R_1 R_2 = (a/(2 cos i)) (a cos i / 2) = a^2/4 for every incidence."""
    a = 10.0
    rec, _ = rec_at(oracle_mod, sphere(oracle_mod, a=a), a * math.sin(math.radians(deg)), pmax=0)
    assert rec[0, oracle_mod.D] == pytest.approx(a * a / 4, rel=1e-12)
    assert rec[0, oracle_mod.NF] == 0


@pytest.mark.parametrize("m", [1.333, 1.55])
@pytest.mark.parametrize("deg", [12.0, 45.0, 70.0])
def test_sphere_closed_forms(oracle_mod, m, deg):
    """Deviation 2i - 2p r + (p-1) pi, divergence a^2 sin i cos i / (sin th |dTheta/di|) and
    path phase 2 k a (p m cos r - cos i) (van de Hulst's geometric optics of the sphere)."""
    a = 10.0
    o = sphere(oracle_mod, a=a, m=m)
    i = math.radians(deg)
    r = math.asin(math.sin(i) / m)
    rec, _ = rec_at(oracle_mod, o, a * math.sin(i), pmax=4)
    for p in range(1, 5):
        Theta = 2 * i - 2 * p * r + (p - 1) * math.pi
        th = math.acos(math.cos(Theta))
        s = rec[p, oracle_mod.S:oracle_mod.S + 3]
        assert math.acos(max(-1.0, min(1.0, s[2]))) == pytest.approx(th, abs=1e-12)
        dTdi = 2 - 2 * p * math.cos(i) / (m * math.cos(r))
        D = a * a * math.sin(i) * math.cos(i) / (math.sin(th) * abs(dTdi))
        assert rec[p, oracle_mod.D] == pytest.approx(D, rel=1e-11)
        psi = 2 * o.k0 * a * (p * m * math.cos(r) - math.cos(i))
        assert rec[p, oracle_mod.PSI] == pytest.approx(psi, abs=1e-10)
    # p = 0 phase: -2 k a cos i
    assert rec[0, oracle_mod.PSI] == pytest.approx(-2 * o.k0 * a * math.cos(i), abs=1e-11)


def test_sphere_worked_values(oracle_mod):
    """a = 10 um, m = 1.333, i = 45 deg: the sphere's closed forms of the test above (deviation,
    divergence factor a^2 sin i cos i / (sin theta |d theta / d i|), optical path), evaluated by hand
    to six figures, as a fixed cross-check of the oracle's orders 1..3."""
    a = 10.0
    o = sphere(oracle_mod, a=a)
    rec, _ = rec_at(oracle_mod, o, a * math.sin(math.radians(45.0)), pmax=3)
    want = {1: (25.927, 152.789, 8.45777), 2: (141.853, 160.917, 31.0577), 3: (102.220, 29.158, 53.6576)}
    for p, (th, D, psik) in want.items():
        s = rec[p, oracle_mod.S:oracle_mod.S + 3]
        assert math.degrees(math.acos(s[2])) == pytest.approx(th, abs=1e-3)
        assert rec[p, oracle_mod.D] == pytest.approx(D, abs=1e-3)
        assert rec[p, oracle_mod.PSI] / o.k0 == pytest.approx(psik, abs=1e-4)


# --------------------------------------------------------------------------------------------
# P5: Descartes rainbow angles (folds of the in-plane map)
# --------------------------------------------------------------------------------------------

def dalpha_db(oracle_mod, o, b, p):
    rec, _, _ = o.trace_ray(b, 0.0, p)
    r = rec[p]
    J = r[oracle_mod.J:oracle_mod.J + 4].reshape(2, 2)
    ds = J[0, 0] * r[oracle_mod.V1:oracle_mod.V1 + 3] + J[1, 0] * r[oracle_mod.V2:oracle_mod.V2 + 3]
    s = r[oracle_mod.S:oracle_mod.S + 3]
    al = math.atan2(s[0], s[2])
    ea = np.array([math.cos(al), 0.0, -math.sin(al)])
    return float(ds @ ea), r


@pytest.mark.parametrize("m,p", [(1.333, 2), (1.333, 3), (1.333, 4), (1.333, 5), (1.33, 2), (1.33, 3),
                                 (1.55, 2), (1.55, 3)])
def test_descartes_angles(oracle_mod, m, p):
    a = 10.0
    o = sphere(oracle_mod, a=a, m=m)
    ic = math.acos(math.sqrt((m * m - 1) / (p * p - 1)))
    rc = math.asin(math.sin(ic) / m)
    th_c = math.acos(math.cos(2 * ic - 2 * p * rc + (p - 1) * math.pi))
    lo, hi = a * math.sin(ic - 0.1), a * math.sin(min(ic + 0.1, math.pi / 2 - 1e-3))
    flo = dalpha_db(oracle_mod, o, lo, p)[0]
    fhi, rhi = dalpha_db(oracle_mod, o, hi, p)
    assert flo * fhi < 0
    orient_lo = dalpha_db(oracle_mod, o, lo, p)[1][oracle_mod.ORIENT]
    assert orient_lo != rhi[oracle_mod.ORIENT]  # the fold flips the orientation of the map
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        fm, rm = dalpha_db(oracle_mod, o, mid, p)
        if rm[oracle_mod.VALID] == 0:
            break  # exactly on the fold: det Q' = 0, the ray record is (rightly) invalid
        if fm * flo > 0:
            lo, flo = mid, fm
        else:
            hi = mid
    rec, _, _ = o.trace_ray(lo, 0.0, p)
    s = rec[p, oracle_mod.S:oracle_mod.S + 3]
    assert math.acos(s[2]) == pytest.approx(th_c, abs=1e-9)


def test_descartes_values_print(oracle_mod):
    """The classical numbers: primary 137.92 deg, secondary 129.11 deg for m = 1.333."""
    for p, want in [(2, 137.922), (3, 129.109)]:
        m = 1.333
        ic = math.acos(math.sqrt((m * m - 1) / (p * p - 1)))
        rc = math.asin(math.sin(ic) / m)
        th = math.degrees(math.acos(math.cos(2 * ic - 2 * p * rc + (p - 1) * math.pi)))
        assert th == pytest.approx(want, abs=1e-3)


# --------------------------------------------------------------------------------------------
# P6: brute-force ray tube of a tilted ellipsoid (no curvature used)
# --------------------------------------------------------------------------------------------

def test_tube_jacobian_bruteforce(oracle_mod):
    """dOmega/dA from central differences of the traced exit directions against the curvature
    chain: J (in the exit basis), D_geo = 1/|det J|, the orientation sign and energy
    |F|^2 = P dA/dOmega with P the order's power fraction.  This checks Eq. (WavefrontEqVec),
    the projections P and the free propagation of Q against the bare geometry."""
    o = tilted_ellipsoid(oracle_mod, jones=(0.6, 0.8j), scale=0.1)
    h_fd = 1e-5 * 12.0
    hh, nx, ny, xc, yc = o.square_grid(h=1.0)
    checked = 0
    rng = np.random.default_rng(7)
    for _ in range(64):
        while True:
            u, v = rng.uniform(-1, 1, size=2)
            if u * u + v * v < 0.8:
                break
        # a point of the projected ellipse
        x = xc + u * 11.0
        y = yc + v * 9.5
        rec0, _, hit = o.trace_ray(x, y, 5)
        if not hit:
            continue
        # central differences at h and h/2, Richardson-extrapolated to O(h^4)
        offs = (-h_fd, -h_fd / 2, h_fd / 2, h_fd)
        sx = [o.trace_ray(x + d, y, 5)[0] for d in offs]
        sy = [o.trace_ray(x, y + d, 5)[0] for d in offs]
        for p in range(6):
            r = rec0[p]
            recs = [q[p] for q in sx + sy]
            if r[oracle_mod.VALID] == 0 or any(q[oracle_mod.VALID] == 0 for q in recs):
                continue
            S = lambda q: q[oracle_mod.S:oracle_mod.S + 3]

            def rich(q):
                d1 = (S(q[3]) - S(q[0])) / (2 * h_fd)
                d2 = (S(q[2]) - S(q[1])) / h_fd
                return (4 * d2 - d1) / 3

            dsx = rich(recs[0:4])
            dsy = rich(recs[4:8])
            s = S(r)
            vol = float(s @ np.cross(dsx, dsy))
            J = r[oracle_mod.J:oracle_mod.J + 4].reshape(2, 2)
            v1, v2 = r[oracle_mod.V1:oracle_mod.V1 + 3], r[oracle_mod.V2:oracle_mod.V2 + 3]
            Jfd = np.array([[v1 @ dsx, v1 @ dsy], [v2 @ dsx, v2 @ dsy]])
            scale = np.abs(J).max()
            if abs(np.linalg.det(J)) < 1e-3 * scale * scale:
                continue  # too close to a caustic for finite differences
            assert np.allclose(Jfd, J, rtol=0, atol=2e-6 * scale)
            assert r[oracle_mod.DGEO] == pytest.approx(1.0 / abs(vol), rel=2e-5)
            assert np.sign(vol) == r[oracle_mod.ORIENT]
            F = r[oracle_mod.F:oracle_mod.F + 6]
            assert float(F @ F) == pytest.approx(r[oracle_mod.POWER] * r[oracle_mod.DGEO], rel=1e-10)
            checked += 1
    assert checked > 100


# --------------------------------------------------------------------------------------------
# P7: mirror symmetry of an axis-aligned ellipsoid
# --------------------------------------------------------------------------------------------

def test_mirror_symmetry_rays(oracle_mod):
    """Mirror y -> -y maps the object onto itself: the ray at (x, -y) is the mirror image of the
    ray at (x, y); an x-polarised field is even, a y-polarised one odd."""
    for jones, sign in [((1.0, 0.0), 1.0), ((0.0, 1.0), -1.0)]:
        o = oracle_mod.Object(12.0, 10.0, 8.0, m=M_WATER, wavelength=LAM, jones=jones)
        M = np.diag([1.0, -1.0, 1.0])
        rng = np.random.default_rng(3)
        for _ in range(20):
            x, y = rng.uniform(-8, 8), rng.uniform(-6, 6)
            ra, _, ha = o.trace_ray(x, y, 4)
            rb, _, hb = o.trace_ray(x, -y, 4)
            assert ha == hb
            for p in range(5):
                assert ra[p, oracle_mod.VALID] == rb[p, oracle_mod.VALID]
                if ra[p, oracle_mod.VALID] == 0:
                    continue
                assert np.allclose(M @ ra[p, oracle_mod.S:oracle_mod.S + 3], rb[p, oracle_mod.S:oracle_mod.S + 3], atol=1e-14)
                Fa = ra[p, oracle_mod.F:oracle_mod.F + 6:2] + 1j * ra[p, oracle_mod.F + 1:oracle_mod.F + 6:2]
                Fb = rb[p, oracle_mod.F:oracle_mod.F + 6:2] + 1j * rb[p, oracle_mod.F + 1:oracle_mod.F + 6:2]
                assert np.allclose(sign * (M @ Fa), Fb, atol=1e-12 * max(1.0, np.abs(Fa).max()))
                assert ra[p, oracle_mod.PSI] == pytest.approx(rb[p, oracle_mod.PSI], abs=1e-11)
                assert ra[p, oracle_mod.NF] == rb[p, oracle_mod.NF]


def test_mirror_symmetry_field_exact(oracle_mod):
    """The exact branch sum (O3) over the cell-centred (theta, phi) grid is mirror symmetric:
    |F_p(theta, phi)| = |F_p(theta, -phi)| per order for an axis-aligned ellipsoid and x
    polarisation.  Directions whose branch comes from a triangle at the rim of the valid region
    of the ray grid can miss it on one side (the diagonal split of the cells is not mirror
    symmetric there); those one-sided misses are bounded, everything else agrees to 1e-8."""
    o = oracle_mod.Object(12.0, 10.0, 8.0, m=M_WATER, wavelength=LAM, jones=(1.0, 0.0))
    nt, nph = 24, 48
    # orders 0 and 1 have no fold; near a fold the gap left by the skipped fold triangles also
    # depends on the diagonal split (the per-ray test covers the higher orders)
    out, mask, hits, nfail = o.field_grid(1, nt, nph, h=0.25, flags=oracle_mod.FIELD_EXACT)
    assert hits > 1000 and nfail == 0
    F = oracle_mod.complex_field(out).reshape(nt, nph, 2, 2)
    mk = mask.reshape(nt, nph)
    A = np.abs(F)
    B = A[:, ::-1]
    ok = (mk == 0) & (mk[:, ::-1] == 0)
    both = ok[:, :, None] & (A.max(axis=3) > 0) & (B.max(axis=3) > 0)
    one = ok[:, :, None] & ((A.max(axis=3) > 0) != (B.max(axis=3) > 0))
    scale = A.max()
    assert np.allclose(A[both], B[both], rtol=1e-8, atol=1e-8 * scale)
    assert one.sum() < 0.06 * both.sum(), (one.sum(), both.sum())


# --------------------------------------------------------------------------------------------
# P8: energy bookkeeping over all orders
# --------------------------------------------------------------------------------------------

def test_energy_all_orders(oracle_mod):
    o = tilted_ellipsoid(oracle_mod, jones=(0.3, 0.9 + 0.3j), scale=0.1)
    inc = abs(0.3) ** 2 + abs(0.9 + 0.3j) ** 2
    rng = np.random.default_rng(11)
    n = 0
    for _ in range(200):
        x, y = rng.uniform(-12, 12), rng.uniform(-12, 12)
        rec, pin, hit = o.trace_ray(x, y, 12)
        if not hit or np.any(rec[:, oracle_mod.VALID] == 0):
            continue
        total = rec[:, oracle_mod.POWER].sum() + pin
        assert total == pytest.approx(inc, rel=1e-12)
        n += 1
    assert n > 50


# --------------------------------------------------------------------------------------------
# P9: Table 1 of the paper (supernumerary bows of a sphere)
# --------------------------------------------------------------------------------------------

def load_table1():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_rainbow_peaks.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            a, k, th = line.split()
            rows.append((float(a), int(k), float(th)))
    return rows


def peak_positions(th, I):
    out = []
    for i in range(1, len(I) - 1):
        if I[i] > I[i - 1] and I[i] >= I[i + 1]:
            y0, y1, y2 = I[i - 1], I[i], I[i + 1]
            out.append(th[i] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * (th[1] - th[0]))
    return np.array(out)


@pytest.mark.parametrize("a,nrays", [(50.0, 8000), (500.0, 40000)])
def test_table1_rainbow_peaks(oracle_mod, a, nrays):
    """Order p = 2, perpendicular polarisation, 1-D fan in the plane phi = 0; ray sum (O2) with
    the physical-optics integral (O4) around the fold.  Every RTW entry of Table 1 within
    0.02 deg (the table prints 0.01 deg)."""
    o = sphere(oracle_mod, a=a, jones=(0.0, 1.0))
    th = np.radians(np.arange(137.5, 161.0, 0.002))
    out, mask = o.field_fan(nrays, th, 2, flags=oracle_mod.FIELD_PO)
    I = np.abs(oracle_mod.complex_field(out[:, 2, :])[:, 1]) ** 2
    pk = np.degrees(peak_positions(th, I))
    for a_t, K, want in load_table1():
        if a_t != a:
            continue
        assert pk[K] == pytest.approx(want, abs=0.02), (a, K, pk[K], want)


def test_po_matches_rays_outside_caustic(oracle_mod):
    """Between 1.5 and 3 Airy widths the PO integral is blended with the ray sum; both must agree
    there, and the blended field must follow the exact branch sum (O3) within a few percent."""
    a = 500.0
    o = sphere(oracle_mod, a=a, jones=(0.0, 1.0))
    Aw = (LAM / a) ** (2 / 3)
    thc = math.radians(137.922)
    th = thc + np.linspace(1.6 * Aw, 2.9 * Aw, 200)
    po, _ = o.field_fan(40000, th, 2, flags=oracle_mod.FIELD_PO)
    ex, _ = o.field_fan(40000, th, 2, flags=oracle_mod.FIELD_EXACT)
    Ip = np.abs(oracle_mod.complex_field(po[:, 2, :])[:, 1]) ** 2
    Ie = np.abs(oracle_mod.complex_field(ex[:, 2, :])[:, 1]) ** 2
    rel = np.linalg.norm(Ip - Ie) / np.linalg.norm(Ie)
    assert rel < 0.05


# --------------------------------------------------------------------------------------------
# P10: the interpolation (O2) converges to the exact branch sum (O3) as O(h^2)
# --------------------------------------------------------------------------------------------

def test_fan_interpolation_converges(oracle_mod):
    o = sphere(oracle_mod, a=10.0, jones=(0.0, 1.0))
    th = np.radians(np.arange(10.0, 60.0, 0.1))
    errs = []
    for n in (1000, 2000, 4000):
        o2, _ = o.field_fan(n, th, 1)
        o3, _ = o.field_fan(n, th, 1, flags=oracle_mod.FIELD_EXACT)
        F2 = oracle_mod.complex_field(o2[:, 1, :])
        F3 = oracle_mod.complex_field(o3[:, 1, :])
        errs.append(np.linalg.norm(F2 - F3) / np.linalg.norm(F3))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.2 < r1 < 4.8 and 3.2 < r2 < 4.8, errs


def test_grid_interpolation_converges(oracle_mod):
    o = oracle_mod.Object(12.0, 10.0, 8.0, quat=(math.cos(0.1), math.sin(0.1), 0, 0), m=M_WATER,
                          wavelength=LAM, jones=(1.0, 0.0))
    errs = []
    for h in (0.1, 0.05, 0.025):
        o2, m2, hits, _ = o.field_grid(1, 32, 64, h=h)
        o3, m3, _, nf = o.field_grid(1, 32, 64, h=h, flags=oracle_mod.FIELD_EXACT)
        ok = (m2 == 0)
        F2 = oracle_mod.complex_field(o2).sum(axis=1)[ok]
        F3 = oracle_mod.complex_field(o3).sum(axis=1)[ok]
        errs.append(np.linalg.norm(F2 - F3) / np.linalg.norm(F3))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs


def test_grid_matches_fan_in_symmetry_plane(oracle_mod):
    """A sphere's 2-D field in the plane phi ~ 0 agrees with the fan field there: both are
    interpolations of the same exact branch sum (checked with O3 on both)."""
    o = sphere(oracle_mod, a=10.0, jones=(0.0, 1.0))
    nt, nph = 90, 64
    out, mask, hits, nfail = o.field_grid(1, nt, nph, h=0.1, flags=oracle_mod.FIELD_EXACT)
    F = oracle_mod.complex_field(out).sum(axis=1).reshape(nt, nph, 2)
    j = nph // 2  # phi = +pi/nph (closest to 0)
    phi = -math.pi + (j + 0.5) * 2 * math.pi / nph
    th = (np.arange(nt) + 0.5) * math.pi / nt
    o1, m1 = o.field_fan(4000, th, 1, fan_phi=phi, flags=oracle_mod.FIELD_EXACT)
    F1 = oracle_mod.complex_field(o1).sum(axis=1)
    ok = (mask.reshape(nt, nph)[:, j] == 0) & (m1 == 0) & (th > 0.2) & (th < 1.2)
    assert ok.sum() > 20
    assert np.allclose(F[ok, j, :], F1[ok], rtol=1e-7, atol=1e-7 * np.abs(F1[ok]).max())


def test_direction_list_matches_grid(oracle_mod):
    """The field on a list of directions equals the grid field on the same directions (the grid's
    own directions in shuffled order), including the masks."""
    o = oracle_mod.Object(6.0, 5.0, 4.0, quat=(0.9659258262890683, 0.2588190451025207, 0.0, 0.0), m=1.333,
                          wavelength=0.6328)
    nt, nph = 24, 48
    ref, rm, hits, _ = o.field_grid(2, nt, nph, n_target=20_000)
    th = (np.arange(nt) + 0.5) * np.pi / nt
    ph = -np.pi + (np.arange(nph) + 0.5) * 2 * np.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    dirs = np.stack([T.ravel(), P.ravel()], 1)
    perm = np.random.default_rng(3).permutation(dirs.shape[0])
    out, m, h2, _ = o.field_dirs(2, dirs[perm], n_target=20_000)
    assert h2 == hits
    assert np.array_equal(m, rm[perm])
    # the same contributions, added in another thread order
    assert np.abs(out - ref[perm]).max() <= 1e-13 * np.abs(ref).max()


# --------------------------------------------------------------------------------------------
# Fields at finite points M (Eqs. IntVCRM, DivFactVCRM with kappa_GM, PhasePath to r_M)
# --------------------------------------------------------------------------------------------

def sphere_crossing(r, s, R):
    """t > 0 with |r + t s| = R, from the quadratic in t."""
    sr, rr = float(np.dot(s, r)), float(np.dot(r, r))
    return -sr + math.sqrt(sr * sr - rr + R * R)


@pytest.mark.parametrize("deg", [5.0, 30.0, 60.0, 85.0])
@pytest.mark.parametrize("R", [20.0, 50.0, 400.0])
def test_near_field_convex_mirror(oracle_mod, deg, R):
    """p = 0 on a sphere of radius a, seen at the point M where the reflected ray meets the sphere
    |M| = R: a convex mirror's reflected wave diverges from the focal lines a cos(i)/2 and
    a/(2 cos i) behind the surface (Coddington's equations for a plane wave), so
    |E(M)|^2 = |r_perp|^2 / ((1 + 2t/(a cos i)) (1 + 2t cos(i)/a)); the phase is k (z_1 + t) with
    z_1 = -a cos i the incidence point, M lies on the mirror-reflected ray, no focal line is met."""
    a = 10.0
    o = sphere(oracle_mod, a=a)
    i = math.radians(deg)
    rec, _ = rec_at(oracle_mod, o, a * math.sin(i), pmax=0)
    near, ok = o.near_record(rec[0], R)
    assert ok
    r1 = np.array([a * math.sin(i), 0.0, -a * math.cos(i)])
    n = r1 / a
    s = np.array([0.0, 0.0, 1.0]) - 2 * n[2] * n  # law of reflection for k = z
    t = sphere_crossing(r1, s, R)
    rs, _ = fresnel_closed(i, M_WATER)
    I_closed = rs * rs / ((1 + 2 * t / (a * math.cos(i))) * (1 + 2 * t * math.cos(i) / a))
    F = near[oracle_mod.F:oracle_mod.F + 6]
    assert F[0::2] @ F[0::2] + F[1::2] @ F[1::2] == pytest.approx(I_closed, rel=1e-12)
    assert near[oracle_mod.PSI] == pytest.approx(o.k0 * (-a * math.cos(i) + t), rel=1e-14)
    assert np.allclose(near[oracle_mod.S:oracle_mod.S + 3], (r1 + t * s) / R, atol=1e-14)
    assert near[oracle_mod.NF] == 0 and near[oracle_mod.ORIENT] == rec[0, oracle_mod.ORIENT]


def test_near_field_tends_to_far_field(oracle_mod):
    """Far from the object, R E(R u) e^{-ikR} tends to the far-field amplitude F(s), M/R to s,
    and the phase of E(M) to k R + Psi plus k (R + s.r - t), the end-point term; checked on every
    order 0..3 of rays of the tilted ellipsoid at R = 1e8 um.  The amplitude's deviation is
    bounded by (|tr Q'^-1| + |r_exit|) / R (the wavefront's radii and the exit point against R),
    the direction's by |r_exit| / R, the phase's by the rounding of k R = 1e9 rad."""
    o = tilted_ellipsoid(oracle_mod)
    R = 1e8
    for b in (-70.0, -20.0, 5.0, 45.0, 90.0):
        rec, _, hit = o.trace_ray(b, 0.3 * b, 3)
        assert hit
        for p in range(4):
            if rec[p, oracle_mod.VALID] == 0.0:
                continue
            near, ok = o.near_record(rec[p], R)
            assert ok
            s = rec[p, oracle_mod.S:oracle_mod.S + 3]
            r = rec[p, oracle_mod.REXIT:oracle_mod.REXIT + 3]
            Q = rec[p, oracle_mod.Q:oracle_mod.Q + 4].reshape(2, 2)
            Ff = rec[p, oracle_mod.F:oracle_mod.F + 6]
            Fn = near[oracle_mod.F:oracle_mod.F + 6] * R
            bound = (abs(np.trace(np.linalg.inv(Q))) + np.linalg.norm(r)) / R
            assert np.abs(Fn - Ff).max() <= bound * np.abs(Ff).max()
            assert np.abs(near[oracle_mod.S:oracle_mod.S + 3] - s).max() <= np.linalg.norm(r) / R
            sr, rr = float(s @ r), float(r @ r)
            geo = (sr * sr - rr) / (math.sqrt(sr * sr - rr + R * R) + R)
            expect = rec[p, oracle_mod.PSI] + o.k0 * R + o.k0 * geo
            assert near[oracle_mod.PSI] == pytest.approx(expect, abs=1e-6)
            assert near[oracle_mod.NF] == rec[p, oracle_mod.NF]


def mirror_closed(a, m, R, theta):
    """Convex-mirror reflection (p = 0) seen on the sphere |M| = R at polar angle theta: the
    incidence angle i whose reflected ray reaches that M (bisection on the law of reflection),
    the last leg t and |r_perp|, |r_par| (Born & Wolf)."""
    def geo(i):
        r1 = np.array([a * math.sin(i), 0.0, -a * math.cos(i)])
        s = np.array([0.0, 0.0, 1.0]) - 2 * (r1[2] / a) * (r1 / a)
        t = sphere_crossing(r1, s, R)
        M = r1 + t * s
        return math.atan2(M[0], M[2]), t
    lo, hi = 1e-9, math.pi / 2 - 1e-9
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (geo(lo)[0] - theta) * (geo(mid)[0] - theta) <= 0:
            hi = mid
        else:
            lo = mid
    i = 0.5 * (lo + hi)
    t = geo(i)[1]
    r_ = math.asin(math.sin(i) / m)
    ci, cr = math.cos(i), math.cos(r_)
    return i, t, (ci - m * cr) / (ci + m * cr), (m * ci - cr) / (m * ci + cr)


def test_near_field_sphere_grid_matches_mirror(oracle_mod):
    """The dense-ray field on the sphere |M| = 40 um around a reflecting sphere of radius 10 um
    (p = 0, x-polarised light) against the convex-mirror closed form: the plane of incidence at
    azimuth phi carries r_par cos(phi) and r_perp sin(phi), so
    |E|^2 = (r_par^2 cos^2 phi + r_perp^2 sin^2 phi) / ((1 + 2t/(a cos i)) (1 + 2t cos(i)/a)),
    counted over all three components (the ray through M is not radial).  The error falls like
    the square of the ray spacing."""
    a, R = 10.0, 40.0
    o = sphere(oracle_mod, a=a, jones=(1.0, 0.0))
    nt, nph = 24, 48
    th = (np.arange(nt) + 0.5) * math.pi / nt
    ph = -math.pi + (np.arange(nph) + 0.5) * 2 * math.pi / nph
    closed = {it: mirror_closed(a, M_WATER, R, th[it]) for it in range(6, nt - 2)}
    errs = []
    for n_target in (4_000, 16_000, 64_000):
        out, mask, hits = o.field_sphere(0, nt, nph, R, n_target=n_target)
        assert hits > 0
        E = oracle_mod.complex_field(out)[:, 0]
        I_grid = (np.abs(E) ** 2).sum(axis=-1)
        e = 0.0
        for it, (i, t, rs, rp) in closed.items():
            for jp in range(nph):
                k = it * nph + jp
                if mask[k]:
                    continue
                c2 = math.cos(ph[jp]) ** 2
                Ic = (rp * rp * c2 + rs * rs * (1 - c2)) / ((1 + 2 * t / (a * math.cos(i))) * (1 + 2 * t * math.cos(i) / a))
                e = max(e, abs(I_grid[k] / Ic - 1))
        errs.append(e)
    print("near-field sphere: max relative intensity error per ray density", errs)
    assert errs[1] < 0.4 * errs[0] and errs[2] < 0.4 * errs[1] and errs[2] < 3e-3


# --------------------------------------------------------------------------------------------
# Incident waves that are not plane: a point source (Eq. PhaseTotal's Phi_i, Q_i of
# Eq. WavefrontEqVec at the first point, A_0 of Eq. IntVCRM)
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("zs", [30.0, 100.0, 1000.0])
@pytest.mark.parametrize("x", [0.5, 3.0, 6.0, 9.0])
def test_point_source_convex_mirror(oracle_mod, zs, x):
    """A point source on the axis at distance zs below a sphere of radius a: a ray leaving it
    toward the point (x, 0) of the plane through the centre meets the sphere at r_1, at distance
    rho, with incidence angle i.  A convex mirror images a source at distance rho into virtual
    focal lines of curvature 1/rho + 2/(a cos i) and 1/rho + 2 cos(i)/a (Coddington's equations),
    so the reflected far field of the spherical wave e^{ik rho}/rho is
    |F|^2 = |r_perp|^2 / (rho^2 (1/rho + 2/(a cos i)) (1/rho + 2 cos(i)/a)) with phase
    k (rho - s.r_1), s the mirror-reflected direction (y-polarised source: perpendicular to the
    plane of incidence)."""
    a = 10.0
    o = oracle_mod.Object(a, a, a, m=M_WATER, wavelength=LAM, jones=(0.0, 1.0), source=(0.0, 0.0, -zs))
    rec, _, hit = o.trace_ray(x, 0.0, 0)
    assert hit
    S = np.array([0.0, 0.0, -zs])
    k = np.array([x, 0.0, zs]) / math.hypot(x, zs)
    # entry point: |S + rho k| = a, smaller root
    b = float(k @ S)
    rho = -b - math.sqrt(b * b - (S @ S - a * a))
    r1 = S + rho * k
    n = r1 / a
    ci = -float(k @ n)
    s = k - 2 * float(k @ n) * n
    i = math.acos(ci)
    rs, _ = fresnel_closed(i, M_WATER)
    I_closed = rs * rs / (rho * rho * (1 / rho + 2 / (a * ci)) * (1 / rho + 2 * ci / a))
    F = rec[0, oracle_mod.F:oracle_mod.F + 6]
    assert F[0::2] @ F[0::2] + F[1::2] @ F[1::2] == pytest.approx(I_closed, rel=1e-12)
    # r_1 = S + rho k cancels to about 1e-16 zs in this closed form
    assert np.allclose(rec[0, oracle_mod.S:oracle_mod.S + 3], s, atol=1e-14 * zs)
    assert rec[0, oracle_mod.PSI] == pytest.approx(o.k0 * (rho - s @ r1), abs=1e-12 * o.k0 * zs)
    assert rec[0, oracle_mod.NF] == 0


def test_point_source_tends_to_plane_wave(oracle_mod):
    """A source far below the tilted ellipsoid, at distance Z = 1e9 um: every order 0..3 of the
    ray through (x, y) approaches the plane wave's ray at (x, y): Z F -> F (within 1e-5, a hundred
    times L / Z), s -> s, and the phase exceeds the plane wave's by k (Z + (x^2 + y^2) /
    (2 Z)) up to the first-order change k r_exit . ds of the far-field phase with the direction and
    the rounding of k Z = 1e10 rad."""
    Z = 1e9
    plane = tilted_ellipsoid(oracle_mod, jones=(1.0, 0.3j))
    h = math.radians(20.0) / 2
    point = oracle_mod.Object(120.0, 100.0, 80.0, quat=(math.cos(h), math.sin(h), 0, 0), m=M_WATER, wavelength=LAM,
                              jones=(1.0, 0.3j), source=(0.0, 0.0, -Z))
    for x, y in ((-70.0, 10.0), (-20.0, -30.0), (5.0, 2.0), (45.0, 60.0), (90.0, -5.0)):
        rp, _, hp = plane.trace_ray(x, y, 3)
        rq, _, hq = point.trace_ray(x, y, 3)
        assert hp and hq
        for p in range(4):
            assert rq[p, oracle_mod.VALID] == rp[p, oracle_mod.VALID]
            if rp[p, oracle_mod.VALID] == 0.0:
                continue
            # corrections of order L / Z = 1e-7, magnified where F varies quickly with s: 1e-5
            Fp = rp[p, oracle_mod.F:oracle_mod.F + 6]
            assert np.abs(Z * rq[p, oracle_mod.F:oracle_mod.F + 6] - Fp).max() <= 1e-5 * np.abs(Fp).max()
            ds = np.linalg.norm(rq[p, oracle_mod.S:oracle_mod.S + 3] - rp[p, oracle_mod.S:oracle_mod.S + 3])
            assert ds < 1e-6
            # the far-field phase varies with the direction as dPsi/ds = -k r_exit: the direction's
            # O(L/Z) shift moves it by at most k |r_exit| |ds| (first order)
            d = rq[p, oracle_mod.PSI] - rp[p, oracle_mod.PSI] - plane.k0 * (Z + (x * x + y * y) / (2 * Z))
            rx = np.linalg.norm(rp[p, oracle_mod.REXIT:oracle_mod.REXIT + 3])
            assert abs(d) <= 1.5 * plane.k0 * rx * ds + 5e-6
            assert rq[p, oracle_mod.NF] == rp[p, oracle_mod.NF]
            assert rq[p, oracle_mod.ORIENT] == rp[p, oracle_mod.ORIENT]


def point_mirror_closed(a, m, zs, theta):
    """Reflection (p = 0) of the spherical wave from a source at distance zs below a sphere of
    radius a, reaching the far-field polar angle theta: the ray through (x, 0) of the centre plane
    found by bisection on x, its rho, incidence angle i and tilt alpha from the axis, and the two
    reflected curvatures 1/rho + 2/(a cos i), 1/rho + 2 cos(i)/a."""
    S = np.array([0.0, 0.0, -zs])
    def geo(x):
        k = np.array([x, 0.0, zs]) / math.hypot(x, zs)
        b = float(k @ S)
        rho = -b - math.sqrt(b * b - (S @ S - a * a))
        r1 = S + rho * k
        n = r1 / a
        s = k - 2 * float(k @ n) * n
        return math.atan2(s[0], s[2]), rho, -float(k @ n), k
    xmax = a * zs / math.sqrt(zs * zs - a * a) * (1 - 1e-9)  # the tangent ray
    lo, hi = 1e-9, xmax
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (geo(lo)[0] - theta) * (geo(mid)[0] - theta) <= 0:
            hi = mid
        else:
            lo = mid
    _, rho, ci, k = geo(0.5 * (lo + hi))
    r_ = math.asin(math.sqrt(1 - ci * ci) / m)
    cr = math.cos(r_)
    rs, rp = (ci - m * cr) / (ci + m * cr), (m * ci - cr) / (m * ci + cr)
    return rho, ci, float(k[2]), rs, rp


def test_point_source_grid_matches_mirror(oracle_mod):
    """The dense-ray far field of a sphere (radius 10 um, p = 0) lit by an x-polarised point
    source 40 um below its centre, against the mirror closed form: the source's field at the
    first point carries r_par with weight cos^2(phi) cos^2(alpha) and r_perp with sin^2(phi)
    (p = x made perpendicular to the ray of tilt alpha), so
    |F|^2 = (r_par^2 cos^2 phi cos^2 alpha + r_perp^2 sin^2 phi) /
            (rho^2 (1/rho + 2/(a cos i)) (1/rho + 2 cos(i)/a));
    the error falls with the ray spacing."""
    a, zs = 10.0, 40.0
    o = oracle_mod.Object(a, a, a, m=M_WATER, wavelength=LAM, jones=(1.0, 0.0), source=(0.0, 0.0, -zs))
    nt, nph = 24, 48
    th = (np.arange(nt) + 0.5) * math.pi / nt
    ph = -math.pi + (np.arange(nph) + 0.5) * 2 * math.pi / nph
    # away from the edge of the reflected cone (grazing rays end near theta = 14.5 deg), which the
    # outermost cells of a coarse grid need not reach
    closed = {it: point_mirror_closed(a, M_WATER, zs, th[it]) for it in range(6, nt - 2)}
    errs = []
    for n_target in (4_000, 16_000, 64_000):
        out, mask, hits, _ = o.field_grid(0, nt, nph, n_target=n_target)
        assert hits > 0
        I_grid = (np.abs(oracle_mod.complex_field(out)[:, 0]) ** 2).sum(axis=-1)
        e = 0.0
        for it, (rho, ci, ca, rs, rp) in closed.items():
            for jp in range(nph):
                k = it * nph + jp
                if mask[k]:
                    continue
                c2 = math.cos(ph[jp]) ** 2
                Ic = (rp * rp * c2 * ca * ca + rs * rs * (1 - c2)) / (
                    rho * rho * (1 / rho + 2 / (a * ci)) * (1 / rho + 2 * ci / a))
                e = max(e, abs(I_grid[k] / Ic - 1))
        errs.append(e)
    print("point source, sphere p = 0: max relative intensity error per ray density", errs)
    assert errs[1] < 0.4 * errs[0] and errs[2] < 0.4 * errs[1] and errs[2] < 5e-3
