"""Pins of the oracle's superellipsoid, sum_i |u_i|^(2e) = 1 in the body frame (u = R^T (x - c) / a).

The ray theory needs of the surface only, at each interaction point, its normal and its curvature
matrix (principle (iii) of the Introduction, Eq. (WavefrontEqVec)); the oracle takes both from the
gradient and Hessian of the implicit function.  Each test checks that against something other than
the oracle's own formulas:

* a brute-force tracer here (numpy and scipy only: roots of F along the line by sampling and
  Brent's method, the normal from central differences of F, the textbook vector Snell law) fixes
  the geometry, i.e. entry, chords, normals, exit directions and optical paths;
* central differences of the traced exit directions fix the Jacobian ds/d(x, y) and so the
  curvature chain of Eq. (WavefrontEqVec) with the Hessian of a genuine non-quadric;
* e -> 1 reduces to the ellipsoid's closed-form quadric path;
* energy is conserved over all orders, and a body with a = b is symmetric under a quarter turn.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.spatial.transform import Rotation

M_WATER = 1.333
LAM = 0.6328
QUAT = (0.9, 0.25, -0.3, 0.15)  # (w, x, y, z), not normalised: a generic tilt about all three axes


class Body:
    """Independent description of the superellipsoid for the brute-force tracer."""

    def __init__(self, semi, quat, center, e):
        w, x, y, z = quat
        self.R = Rotation.from_quat([x, y, z, w]).as_matrix()  # body -> world
        self.semi = np.asarray(semi, dtype=np.float64)
        self.c = np.asarray(center, dtype=np.float64)
        self.e = float(e)
        self.rb = self.semi.max() * math.sqrt(3.0)  # radius of a ball that holds the box |u_i| <= 1

    def F(self, x):
        u = (self.R.T @ (x - self.c)) / self.semi
        return float(np.sum(np.abs(u) ** (2 * self.e)))

    def normal(self, x):
        h = 1e-6 * self.semi.min()
        g = np.array([(self.F(x + h * d) - self.F(x - h * d)) / (2 * h) for d in np.eye(3)])
        return g / np.linalg.norm(g)

    def root(self, x, k, first):
        """First (entry, from outside) or last crossing (exit, from a surface point) of F = 1
        along x + t k, t > 0, by sampling and Brent's method; None where it is ambiguous."""
        T = 2.0 * self.rb + (np.linalg.norm(x - self.c) if first else 0.0)
        ts = np.linspace(0.0, T, 4001)[1:]
        phi = np.array([self.F(x + t * k) - 1.0 for t in ts])
        if first:
            idx = np.nonzero(phi < 0)[0]
            if idx.size == 0 or idx[0] == 0:
                return None
            a, b = ts[idx[0] - 1], ts[idx[0]]
        else:
            if phi[0] >= 0:
                return None
            idx = np.nonzero(phi >= 0)[0]
            if idx.size == 0:
                return None
            a, b = ts[idx[0] - 1], ts[idx[0]]
        return brentq(lambda t: self.F(x + t * k) - 1.0, a, b, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=200)


def refract(k, n, n1, n2):
    """Vector Snell law; n is the surface normal (either sign).  None for total internal reflection."""
    nn = n if k @ n < 0 else -n
    eta = n1 / n2
    c1 = -(k @ nn)
    c2sq = 1.0 - eta * eta * (1.0 - c1 * c1)
    if c2sq < 0:
        return None
    kt = eta * k + (eta * c1 - math.sqrt(c2sq)) * nn
    return kt / np.linalg.norm(kt)


def reflect(k, n):
    return k - 2.0 * (k @ n) * n


def brute_trace(body, m, x, y, zs, pmax):
    """Exit direction, exit point and optical path per order (None where the order does not leave)."""
    r0 = np.array([x, y, zs])
    kz = np.array([0.0, 0.0, 1.0])
    t = body.root(r0, kz, True)
    if t is None:
        return None
    r1 = r0 + t * kz
    n1 = body.normal(r1)
    out = [(reflect(kz, n1), r1.copy(), r1[2])]
    k = refract(kz, n1, 1.0, m)
    r, path = r1, r1[2]
    for p in range(1, pmax + 1):
        d = body.root(r, k, False)
        if d is None:
            return out
        r = r + d * k
        path += m * d
        n = body.normal(r)
        kt = refract(k, n, m, 1.0)
        out.append(None if kt is None else (kt, r.copy(), path))
        k = reflect(k, n)
    return out


@pytest.mark.parametrize("e", [1.5, 2.0, 3.0])
def test_super_geometry_bruteforce(oracle_mod, e):
    """Exit directions, exit points and optical paths of orders 0..3 against the brute-force tracer."""
    semi, center = (12.0, 10.0, 8.0), (0.7, -0.4, 0.3)
    o = oracle_mod.Object(*semi, quat=QUAT, center=center, m=M_WATER, wavelength=LAM, shape_e=e)
    body = Body(semi, QUAT, center, e)
    zs = center[2] - 2.0 * max(semi) - 1.0
    rng = np.random.default_rng(41)
    checked = 0
    for _ in range(70):
        x, y = center[0] + rng.uniform(-13, 13), center[1] + rng.uniform(-13, 13)
        rec, _, hit = o.trace_ray(x, y, 3)
        ref = brute_trace(body, M_WATER, x, y, zs, 3)
        assert hit == (ref is not None)
        if ref is None:
            continue
        for p, rp in enumerate(ref):
            r = rec[p]
            if rp is None:
                assert r[oracle_mod.VALID] == 0
                continue
            assert r[oracle_mod.VALID] == 1
            s, rx, path = rp
            assert np.allclose(r[oracle_mod.S:oracle_mod.S + 3], s, rtol=0, atol=1e-8)
            assert np.allclose(r[oracle_mod.REXIT:oracle_mod.REXIT + 3], rx, rtol=0, atol=1e-8 * max(semi))
            assert r[oracle_mod.PATH] == pytest.approx(path, abs=1e-8 * max(semi))
            checked += 1
    assert checked > 100


def test_super_tube_jacobian_bruteforce(oracle_mod):
    """J = ds/d(x, y) from the curvature chain (Hessian of F in the curvature matrix C) against
    central differences of the traced exit directions, D_geo = 1/|det J| and |F|^2 = P dA/dOmega,
    on a tilted superellipsoid with e = 2."""
    o = oracle_mod.Object(12.0, 10.0, 8.0, quat=QUAT, m=M_WATER, wavelength=LAM, jones=(0.6, 0.8j), shape_e=2.0)
    h_fd = 1.2e-4
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(80):
        x, y = rng.uniform(-12, 12), rng.uniform(-12, 12)
        rec0, _, hit = o.trace_ray(x, y, 4)
        if not hit:
            continue
        offs = (-h_fd, -h_fd / 2, h_fd / 2, h_fd)
        sx = [o.trace_ray(x + d, y, 4)[0] for d in offs]
        sy = [o.trace_ray(x, y + d, 4)[0] for d in offs]
        for p in range(5):
            r = rec0[p]
            recs = [q[p] for q in sx + sy]
            if r[oracle_mod.VALID] == 0 or any(q[oracle_mod.VALID] == 0 for q in recs):
                continue
            S = lambda q: q[oracle_mod.S:oracle_mod.S + 3]

            def rich(q):
                d1 = (S(q[3]) - S(q[0])) / (2 * h_fd)
                d2 = (S(q[2]) - S(q[1])) / h_fd
                return (4 * d2 - d1) / 3

            dsx, dsy = rich(recs[0:4]), rich(recs[4:8])
            vol = float(S(r) @ np.cross(dsx, dsy))
            J = r[oracle_mod.J:oracle_mod.J + 4].reshape(2, 2)
            v1, v2 = r[oracle_mod.V1:oracle_mod.V1 + 3], r[oracle_mod.V2:oracle_mod.V2 + 3]
            Jfd = np.array([[v1 @ dsx, v1 @ dsy], [v2 @ dsx, v2 @ dsy]])
            scale = np.abs(J).max()
            if abs(np.linalg.det(J)) < 1e-3 * scale * scale:
                continue  # too close to a caustic for finite differences
            assert np.allclose(Jfd, J, rtol=0, atol=2e-5 * scale), (p, J, Jfd)
            assert r[oracle_mod.DGEO] == pytest.approx(1.0 / abs(vol), rel=2e-4)
            assert np.sign(vol) == r[oracle_mod.ORIENT]
            F = r[oracle_mod.F:oracle_mod.F + 6]
            assert float(F @ F) == pytest.approx(r[oracle_mod.POWER] * r[oracle_mod.DGEO], rel=1e-10)
            checked += 1
    assert checked > 80


def test_super_e1_limit(oracle_mod):
    """e = 1 + 1e-12 takes the superellipsoid path (line roots, gradient and Hessian of F) and must
    reproduce the ellipsoid's closed-form quadric path to rounding."""
    kw = dict(quat=QUAT, m=M_WATER, wavelength=LAM, jones=(0.3, 0.9 + 0.3j))
    oq = oracle_mod.Object(12.0, 10.0, 8.0, **kw)
    os_ = oracle_mod.Object(12.0, 10.0, 8.0, shape_e=1.0 + 1e-12, **kw)
    rng = np.random.default_rng(2)
    n = 0
    for _ in range(60):
        x, y = rng.uniform(-11, 11), rng.uniform(-11, 11)
        ra, pa, ha = oq.trace_ray(x, y, 5)
        rb, pb, hb = os_.trace_ray(x, y, 5)
        assert ha == hb
        if not ha:
            continue
        assert np.array_equal(ra[:, oracle_mod.VALID], rb[:, oracle_mod.VALID])
        for p in range(6):
            if ra[p, oracle_mod.VALID] == 0:
                continue
            for f, w in [(oracle_mod.S, 3), (oracle_mod.REXIT, 3), (oracle_mod.J, 4), (oracle_mod.Q, 4), (oracle_mod.F, 6)]:
                a, b = ra[p, f:f + w], rb[p, f:f + w]
                assert np.allclose(a, b, rtol=0, atol=1e-8 * max(1.0, np.abs(a).max())), (p, f)
            assert ra[p, oracle_mod.PSI] == pytest.approx(rb[p, oracle_mod.PSI], abs=1e-7)
            assert ra[p, oracle_mod.NF] == rb[p, oracle_mod.NF]
            n += 1
        assert pa == pytest.approx(pb, rel=1e-8, abs=1e-14)
    assert n > 150


@pytest.mark.parametrize("e", [1.5, 4.0])
def test_super_energy_all_orders(oracle_mod, e):
    """The power fractions of all orders plus what stays inside add up to the incident power, also
    for rays that some flat part of the body holds by total internal reflection (invalid orders)."""
    jones = (0.3, 0.9 + 0.3j)
    o = oracle_mod.Object(12.0, 10.0, 8.0, quat=QUAT, m=M_WATER, wavelength=LAM, jones=jones, shape_e=e)
    inc = abs(jones[0]) ** 2 + abs(jones[1]) ** 2
    rng = np.random.default_rng(13)
    n = 0
    for _ in range(200):
        x, y = rng.uniform(-14, 14), rng.uniform(-14, 14)
        rec, pin, hit = o.trace_ray(x, y, 12)
        if not hit:
            continue
        assert rec[:, oracle_mod.POWER].sum() + pin == pytest.approx(inc, rel=1e-12)
        n += 1
    assert n > 100


def test_super_quarter_turn_field(oracle_mod):
    """A superellipsoid with a = b, axis along z, turned by a quarter about z is itself, and so is
    the square ray grid: the x-polarised field at (theta, phi) equals, up to the turn of the basis,
    the y-polarised field at (theta, phi + 90 degrees).  In the (e_theta, e_phi) basis that is
    F_y(theta, phi + 90) = F_x(theta, phi), on the exact branch sum (Newton on every triangle)."""
    nt, nph = 24, 48
    args = dict(m=M_WATER, wavelength=LAM, shape_e=2.5)
    ox = oracle_mod.Object(10.0, 10.0, 7.0, jones=(1.0, 0.0), **args)
    oy = oracle_mod.Object(10.0, 10.0, 7.0, jones=(0.0, 1.0), **args)
    _, nx, ny, _, _ = ox.square_grid(h=0.3)
    assert nx == ny
    outs = []
    for o in (ox, oy):
        out, mask, hits, nfail = o.field_grid(1, nt, nph, h=0.3, flags=oracle_mod.FIELD_EXACT)
        assert hits > 1000 and nfail == 0
        outs.append((oracle_mod.complex_field(out).reshape(nt, nph, 2, 2), mask.reshape(nt, nph)))
    (Fx, mx), (Fy, my) = outs
    q = nph // 4
    Fy_back = np.roll(Fy, -q, axis=1)  # Fy_back[:, j] = Fy[:, j + q]
    my_back = np.roll(my, -q, axis=1)
    ok = (mx == 0) & (my_back == 0)
    A, B = np.abs(Fx), np.abs(Fy_back)
    both = ok[:, :, None] & (A.max(axis=3) > 0) & (B.max(axis=3) > 0)
    one = ok[:, :, None] & ((A.max(axis=3) > 0) != (B.max(axis=3) > 0))
    scale = A.max()
    assert both.sum() > 500
    assert np.allclose(Fx[both], Fy_back[both], rtol=1e-8, atol=1e-8 * scale)
    assert one.sum() < 0.06 * both.sum(), (one.sum(), both.sum())


def source_frame(c, src):
    """The grid plane's axes of a point source as the oracle's header defines them: a = (c - s)/|c - s|,
    e1 = x (y when a is within 26 deg of x) made perpendicular to a, e2 = a x e1."""
    a = np.asarray(c, float) - np.asarray(src, float)
    a /= np.linalg.norm(a)
    ref = np.array([0.0, 1.0, 0.0]) if abs(a[0]) > 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = ref - (ref @ a) * a
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(a, e1)


@pytest.mark.parametrize("e", [1.5, 3.0])
def test_super_point_source_geometry_bruteforce(oracle_mod, e):
    """A point source lighting a tilted superellipsoid: rays from the source through points of the
    grid plane, orders 0..3, exit directions, exit points and optical paths (from the source) against
    the brute-force tracer."""
    semi, center, src = (12.0, 10.0, 8.0), (0.7, -0.4, 0.3), (15.0, -10.0, -60.0)
    o = oracle_mod.Object(*semi, quat=QUAT, center=center, m=M_WATER, wavelength=LAM, shape_e=e, source=src)
    body = Body(semi, QUAT, center, e)
    e1, e2 = source_frame(center, src)
    rng = np.random.default_rng(17)
    checked = 0
    for _ in range(70):
        x, y = rng.uniform(-16, 16, 2)
        rec, _, hit = o.trace_ray(x, y, 3)
        v = np.asarray(center) + x * e1 + y * e2 - np.asarray(src)
        k = v / np.linalg.norm(v)
        t = body.root(np.asarray(src, float), k, True)
        assert hit == (t is not None)
        if t is None:
            continue
        r1 = np.asarray(src, float) + t * k
        n1 = body.normal(r1)
        ref = [(reflect(k, n1), r1.copy(), t)]
        kk = refract(k, n1, 1.0, M_WATER)
        r, path = r1, t
        for p in range(1, 4):
            d = body.root(r, kk, False)
            if d is None:
                break
            r = r + d * kk
            path += M_WATER * d
            n = body.normal(r)
            kt = refract(kk, n, M_WATER, 1.0)
            ref.append(None if kt is None else (kt, r.copy(), path))
            kk = reflect(kk, n)
        for p, rp in enumerate(ref):
            if rp is None:
                assert rec[p, oracle_mod.VALID] == 0
                continue
            assert rec[p, oracle_mod.VALID] == 1
            assert np.allclose(rec[p, oracle_mod.S:oracle_mod.S + 3], rp[0], rtol=0, atol=1e-8)
            assert np.allclose(rec[p, oracle_mod.REXIT:oracle_mod.REXIT + 3], rp[1], rtol=0, atol=1e-7)
            assert rec[p, oracle_mod.PATH] == pytest.approx(rp[2], abs=1e-7)
            checked += 1
    assert checked > 60


def test_super_point_source_e1_limit(oracle_mod):
    """e = 1 + 1e-12 with a point source reproduces the ellipsoid's closed-form entry from the
    source (and its lit ellipse on the grid plane)."""
    kw = dict(quat=QUAT, m=M_WATER, wavelength=LAM, jones=(0.3, 0.9 + 0.3j), source=(20.0, -5.0, -80.0))
    oq = oracle_mod.Object(12.0, 10.0, 8.0, **kw)
    os_ = oracle_mod.Object(12.0, 10.0, 8.0, shape_e=1.0 + 1e-12, **kw)
    assert np.allclose(oq.square_grid(n_target=5000), os_.square_grid(n_target=5000), rtol=1e-9, atol=1e-9)
    rng = np.random.default_rng(4)
    n = 0
    for _ in range(60):
        x, y = rng.uniform(-12, 12, 2)
        ra, _, ha = oq.trace_ray(x, y, 4)
        rb, _, hb = os_.trace_ray(x, y, 4)
        assert ha == hb
        if not ha:
            continue
        for p in range(5):
            if ra[p, oracle_mod.VALID] == 0:
                continue
            for f, w in [(oracle_mod.S, 3), (oracle_mod.REXIT, 3), (oracle_mod.F, 6)]:
                a, b = ra[p, f:f + w], rb[p, f:f + w]
                assert np.allclose(a, b, rtol=0, atol=1e-8 * max(1.0, np.abs(a).max())), (p, f)
            assert ra[p, oracle_mod.PSI] == pytest.approx(rb[p, oracle_mod.PSI], abs=1e-7)
            n += 1
    assert n > 100


def test_super_refusals(oracle_mod):
    """e < 1 (not convex) is refused, and so are a source inside the bounding ellipsoid and fans on a
    superellipsoid."""
    with pytest.raises(ValueError):
        oracle_mod.Object(10.0, 9.0, 8.0, shape_e=0.8)
    with pytest.raises(ValueError):  # outside the body (c = 8) but inside its bounding ellipsoid (8 x 3^(1/4))
        oracle_mod.Object(10.0, 9.0, 8.0, shape_e=2.0, source=(0.0, 0.0, -10.2))
    o = oracle_mod.Object(10.0, 9.0, 8.0, shape_e=2.0)
    with pytest.raises(RuntimeError):
        o.field_fan(100, np.linspace(0.1, 3.0, 8), 1)
