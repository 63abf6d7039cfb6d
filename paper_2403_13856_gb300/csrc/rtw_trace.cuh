// rtw_trace.cuh -- device code of the per-ray trace (the first half of the RTW hot path).
//
// One thread traces one incident ray of the plane wave through the ellipsoid.  At every
// interaction the wave is re-expressed in the local basis (e_perp, e_par) of the incident plane,
// where the projection matrices of the wavefront equation are diagonal:
//     P_i = diag(1, -n.k_i),   P' = diag(1, -n.k'),      (Eq. Theta-r with s = (e_perp, n x e_perp))
// so Eq. (WavefrontEqVec), k' P' Q' P'^T = k_i P_i Q_i P_i^T + C n.(k' - k_i), is solved entry by
// entry without a 2x2 inverse.  The wave carries
//     Q  (3 unique entries) in the basis (a, b = a x k), a = e_perp of the last interaction,
//     E  (2 complex) on the same basis: the product of the Fresnel coefficients (Eq. Fres) applied
//        step by step in each incident plane (Eq. epsilon_VCRM, "re-evaluated at each interaction"),
//     D_legs = prod 1/|det(I + d Q)| over the internal legs (Eq. DivFactVCRM),
//     N_f    = number of negative eigenvalues of (I + d Q) over the legs (focal lines),
//     the optical path from the plane z = 0 (Eq. PhasePath) and the sign of det T, T the transfer of
//     transverse offsets (orientation of the map t -> s).
#pragma once

#include <type_traits>

#include "rtw_df.cuh"
#include "rtw_internal.h"

namespace rtw {

struct ExitWave {
    double k[3];   // exit direction s
    double ep[3];  // first basis vector; the second is ep x k
    double q11, q12, q22;
    double e1r, e1i, e2r, e2i;
    double t11, t12, t21, t22;  // transfer of offsets (x, y) -> basis (only with kJ)
    double pdet;   // prod |det(I + d Q)| over the internal legs: D_legs = 1 / pdet
    double cosprod, path;
    double r[3];   // exit point
    int nf_legs;
    int sT;        // sign of det T
};

struct FarRecord {
    double s[3];
    double F[6];
    double psi;
    uint32_t flags;
};

// negative eigenvalues of a symmetric 2 x 2 matrix from its trace and determinant
__device__ __forceinline__ int neg_eigs_td(double tr, double det)
{
    if (det < 0.0) return 1;
    if (det > 0.0 && tr < 0.0) return 2;
    if (det == 0.0 && tr < 0.0) return 1;
    return 0;
}

__device__ __forceinline__ int neg_eigs_sym(double a11, double a12, double a22)
{
    return neg_eigs_td(a11 + a22, a11 * a22 - a12 * a12);
}

__device__ __forceinline__ void symv(const double* W, double x, double y, double z, double& ox, double& oy,
                                     double& oz)
{
    ox = W[0] * x + W[1] * y + W[2] * z;
    oy = W[1] * x + W[3] * y + W[4] * z;
    oz = W[2] * x + W[4] * y + W[5] * z;
}

// amp (-i)^nf (er + i ei): a quarter turn per focal line, by swaps and signs
__device__ __forceinline__ void focal_phase(int nf, double amp, double er, double ei, double& ar, double& ai)
{
    switch (nf & 3) {
    case 1: ar = amp * ei; ai = -amp * er; break;
    case 2: ar = -amp * er; ai = -amp * ei; break;
    case 3: ar = -amp * ei; ai = amp * er; break;
    default: ar = amp * er; ai = amp * ei; break;
    }
}

// Far-field record of an exit wave: F = E' sqrt(D_legs / |det Q'|) (-i)^{N_f}, Psi = k0 (L - s.r),
// with sqrt(D) = 1 / sqrt(|det Q'| prod |det(I + d Q)|).
__device__ __forceinline__ bool far_record(const ObjDev& o, const ExitWave& w, FarRecord& fr)
{
    double detQ = w.q11 * w.q22 - w.q12 * w.q12;
    if (!isfinite(detQ)) return false;
    // an exit wave flat in a principal direction (det Q' = 0, where a stretch of surface has no
    // curvature) sends its energy into a single direction: a caustic at infinity, kept as a valid
    // ray with the caustic flag and no amplitude
    const bool flat = !(fabs(detQ) > 0.0);
    const int nf = w.nf_legs + neg_eigs_td(w.q11 + w.q22, detQ);
    double amp = flat ? 0.0 : rsqrt(fabs(detQ) * w.pdet);
    double D = amp * amp;
    double a1r, a1i, a2r, a2i;
    focal_phase(nf, amp, w.e1r, w.e1i, a1r, a1i);
    focal_phase(nf, amp, w.e2r, w.e2i, a2r, a2i);
    double v2x = w.ep[1] * w.k[2] - w.ep[2] * w.k[1];
    double v2y = w.ep[2] * w.k[0] - w.ep[0] * w.k[2];
    double v2z = w.ep[0] * w.k[1] - w.ep[1] * w.k[0];
    fr.s[0] = w.k[0];
    fr.s[1] = w.k[1];
    fr.s[2] = w.k[2];
    fr.F[0] = a1r * w.ep[0] + a2r * v2x;
    fr.F[1] = a1i * w.ep[0] + a2i * v2x;
    fr.F[2] = a1r * w.ep[1] + a2r * v2y;
    fr.F[3] = a1i * w.ep[1] + a2i * v2y;
    fr.F[4] = a1r * w.ep[2] + a2r * v2z;
    fr.F[5] = a1i * w.ep[2] + a2i * v2z;
    fr.psi = o.k0 * (w.path - (w.k[0] * w.r[0] + w.k[1] * w.r[1] + w.k[2] * w.r[2]));
    // orientation of (x, y) -> s: sign(det J) sign(s . (v1 x v2)), det J = det Q' det T,
    // v1 x v2 = ep x (ep x s) = -s
    int orient = (detQ > 0.0 ? 1 : -1) * w.sT * -1;
    // caustic when dA/dOmega = D / cosprod exceeds the cap
    uint32_t f = kFlagValid | (orient > 0 ? kFlagOrient : 0u) | ((flat || D > o.cap * w.cosprod) ? kFlagCaustic : 0u);
    f |= (uint32_t)(nf > 255 ? 255 : nf) << 8;
    fr.flags = f;
    return true;
}

// Record of an exit wave at the point M where it crosses the sphere |M| = R (R beyond the exit
// point), following the divergence chain and the optical path to M (Eqs. DivFactVCRM with
// kappa_GM, PhasePath): the last leg of length t ends the chain with 1 / det(I + t Q') and adds
// its focal lines; F = E' sqrt(D_legs / |det(I + t Q')|) (-i)^{N_f} is the field at M for a unit
// incident wave, Psi = k0 (L + t), s = M / R.  Orientation of (x, y) -> M: sign det(I + t Q')
// sign det T (times the far-field convention's -1); caustic when t^2 D / cosprod exceeds the cap
// (dA/dOmega in the limit t -> infinity).
__device__ __forceinline__ bool near_record(const ObjDev& o, const ExitWave& w, double R, FarRecord& fr)
{
    const double sr = w.k[0] * w.r[0] + w.k[1] * w.r[1] + w.k[2] * w.r[2];
    const double rr = w.r[0] * w.r[0] + w.r[1] * w.r[1] + w.r[2] * w.r[2];
    const double disc = sr * sr - rr + R * R;
    if (!(R * R > rr) || !(disc >= 0.0)) return false;
    const double t = sqrt(disc) - sr;
    const double a11 = 1.0 + t * w.q11, a12 = t * w.q12, a22 = 1.0 + t * w.q22;
    const double detA = a11 * a22 - a12 * a12;
    if (!(fabs(detA) > 0.0) || !isfinite(detA)) return false;
    const int nf = w.nf_legs + neg_eigs_td(a11 + a22, detA);
    const double amp = rsqrt(fabs(detA) * w.pdet);
    const double D = amp * amp;
    double a1r, a1i, a2r, a2i;
    focal_phase(nf, amp, w.e1r, w.e1i, a1r, a1i);
    focal_phase(nf, amp, w.e2r, w.e2i, a2r, a2i);
    const double v2x = w.ep[1] * w.k[2] - w.ep[2] * w.k[1];
    const double v2y = w.ep[2] * w.k[0] - w.ep[0] * w.k[2];
    const double v2z = w.ep[0] * w.k[1] - w.ep[1] * w.k[0];
    const double iR = 1.0 / R;
    fr.s[0] = (w.r[0] + t * w.k[0]) * iR;
    fr.s[1] = (w.r[1] + t * w.k[1]) * iR;
    fr.s[2] = (w.r[2] + t * w.k[2]) * iR;
    fr.F[0] = a1r * w.ep[0] + a2r * v2x;
    fr.F[1] = a1i * w.ep[0] + a2i * v2x;
    fr.F[2] = a1r * w.ep[1] + a2r * v2y;
    fr.F[3] = a1i * w.ep[1] + a2i * v2y;
    fr.F[4] = a1r * w.ep[2] + a2r * v2z;
    fr.F[5] = a1i * w.ep[2] + a2i * v2z;
    fr.psi = o.k0 * (w.path + t);
    const int orient = (detA > 0.0 ? 1 : -1) * w.sT * -1;
    uint32_t f = kFlagValid | (orient > 0 ? kFlagOrient : 0u) | (t * t * D > o.cap * w.cosprod ? kFlagCaustic : 0u);
    f |= (uint32_t)(nf > 255 ? 255 : nf) << 8;
    fr.flags = f;
    return true;
}

// Impact point of grid ray `local` of object o; false if it lies outside the projected section.
__device__ __forceinline__ bool ray_origin(const ObjDev& o, long long local, double& x, double& y)
{
    if (o.grid == kGridFan) {
        double b = -o.fan_w + ((double)local + 0.5) * o.h;
        x = o.c[0] + b * o.fan_ex;
        y = o.c[1] + b * o.fan_ey;
        return true;
    }
    long long ix = local % o.nx, iy = local / o.nx;
    x = o.gc[0] + ((double)ix + 0.5 - (double)(o.nx / 2)) * o.h;
    y = o.gc[1] + ((double)iy + 0.5 - (double)(o.ny / 2)) * o.h;
    double dx = x - o.gc[0], dy = y - o.gc[1];
    double qf = dx * (o.S[0] * dx + o.S[1] * dy) + dy * (o.S[1] * dx + o.S[2] * dy);
    return qf < 1.0;
}

template <typename T>
__device__ __forceinline__ void symvT(const T* W, T x, T y, T z, T& ox, T& oy, T& oz)
{
    ox = W[0] * x + W[1] * y + W[2] * z;
    oy = W[1] * x + W[3] * y + W[4] * z;
    oz = W[2] * x + W[4] * y + W[5] * z;
}

// Distance along k from r (double) to the surface: the root t of (r + t k - c)^T W (r + t k - c) = 1
// given by the quadratic formula in the working precision (sign selects the entry / far root).
// In single precision the root is then polished by one Newton step evaluated in double precision,
// so intersection points and optical paths keep double-precision accuracy (the quadric's residual
// after the step is of the order of the square of the single-precision error).
// wp, when given, is W (r - c) already formed in the working precision at this r (the normal's
// gradient), which the quadratic reuses; wk_out, when given, receives W k.
template <typename T>
__device__ __forceinline__ double chord_to_surface(const ObjDev& o, const T* Wt, const double r[3], const T k[3],
                                                   T sign, bool* ok, const T* wp = nullptr, T* wk_out = nullptr)
{
    const T px = (T)(r[0] - o.c[0]), py = (T)(r[1] - o.c[1]), pz = (T)(r[2] - o.c[2]);
    T wkx, wky, wkz, wpx, wpy, wpz;
    symvT(Wt, k[0], k[1], k[2], wkx, wky, wkz);
    if (wk_out) {
        wk_out[0] = wkx;
        wk_out[1] = wky;
        wk_out[2] = wkz;
    }
    if (wp) {
        wpx = wp[0];
        wpy = wp[1];
        wpz = wp[2];
    } else {
        symvT(Wt, px, py, pz, wpx, wpy, wpz);
    }
    const T Ak = k[0] * wkx + k[1] * wky + k[2] * wkz;
    const T Bk = k[0] * wpx + k[1] * wpy + k[2] * wpz;
    const T Ck = px * wpx + py * wpy + pz * wpz - T(1);
    T dk = Bk * Bk - Ak * Ck;
    *ok = true;
    if (sign < T(0)) {
        if (!(dk > T(0))) {
            *ok = false;
            return 0.0;
        }
    } else if (dk < T(0)) {
        dk = T(0);
    }
    double d = (double)((-Bk + sign * sqrt(dk)) / Ak);
    if (sizeof(T) == sizeof(float)) {
        const double kx = k[0], ky = k[1], kz = k[2];
        const double ux = r[0] - o.c[0] + d * kx, uy = r[1] - o.c[1] + d * ky, uz = r[2] - o.c[2] + d * kz;
        double gx, gy, gz;
        symv(o.W, ux, uy, uz, gx, gy, gz);
        const double f = ux * gx + uy * gy + uz * gz - 1.0;
        const double fp = 2.0 * (kx * gx + ky * gy + kz * gz);
        d -= (double)((float)f / (float)fp);
    }
    return d;
}

// Chord from the surface point r along the inward direction k (the far root of the quadric) with
// A = k^T W k and 1/A given (the reciprocal formed with the interaction's others) and wp = W (r - c),
// the gradient at r; double precision only (single precision takes chord_to_surface and its polish).
template <typename T>
__device__ __forceinline__ double chord_inside(const ObjDev& o, const double r[3], const T k[3], T Ak, T iAk,
                                               const T* wp)
{
    const T px = (T)(r[0] - o.c[0]), py = (T)(r[1] - o.c[1]), pz = (T)(r[2] - o.c[2]);
    const T Bk = k[0] * wp[0] + k[1] * wp[1] + k[2] * wp[2];
    const T Ck = px * wp[0] + py * wp[1] + pz * wp[2] - T(1);
    T dk = Bk * Bk - Ak * Ck;
    if (dk < T(0)) dk = T(0);
    const T sq = dk > T(0) ? dk * rsqrt(dk) : T(0);  // rsqrt: 1 ulp, no correctly rounded root needed
    return (double)((-Bk + sq) * iAk);
}

// ---- superellipsoid F(x) = sum_i |u_i|^(2e) = 1 (e > 1), u = diag(1/a) Rb^T (x - c) ----
// F is convex, so a line meets the surface at most twice, and phi(t) = F(r + t k) - 1 is convex
// along every line: Newton from a point beyond a root on the side where phi >= 0 moves
// monotonically to that root.  The brackets are the body box |u_i| <= 1 and the bounding
// ellipsoid sum u_i^2 = bound2, both of which contain the body (phi >= 0 on them).

// body coordinates of r and body rates of the direction k
__device__ __forceinline__ void super_line(const ObjDev& o, const double r[3], const double k[3], double u[3],
                                           double kap[3])
{
    const double dx = r[0] - o.c[0], dy = r[1] - o.c[1], dz = r[2] - o.c[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        u[i] = (o.Rb[i] * dx + o.Rb[3 + i] * dy + o.Rb[6 + i] * dz) * o.inv_a[i];
        kap[i] = (o.Rb[i] * k[0] + o.Rb[3 + i] * k[1] + o.Rb[6 + i] * k[2]) * o.inv_a[i];
    }
}

// |v|^(2e-2) for v >= 0 (0 at v = 0 for e > 1): n - 2 products when 2e is an integer n, else pow
__device__ __forceinline__ double super_pow(const ObjDev& o, double av)
{
    const int n = o.shape_n;
    if (n > 0) {
        double r = 1.0;
        for (int i = 2; i < n; ++i) r *= av;
        return r;
    }
    return pow(av, 2.0 * o.shape_e - 2.0);
}

// phi(t) and phi'(t) = 2e sum |v_i|^(2e-2) v_i kappa_i, v = u + t kappa
__device__ __forceinline__ double super_phi(const ObjDev& o, const double u[3], const double kap[3], double t,
                                            double& dphi)
{
    const double e2 = 2.0 * o.shape_e;
    double f = -1.0, df = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double v = fma(t, kap[i], u[i]), av = fabs(v);
        const double pw = super_pow(o, av);
        f = fma(pw * av, av, f);
        df = fma(pw * v, kap[i], df);
    }
    dphi = e2 * df;
    return f;
}

// parameters where the line u + t kappa crosses the bounding ellipsoid sum u_i^2 = bound2
__device__ __forceinline__ bool super_bound(const ObjDev& o, const double u[3], const double kap[3], double& t_in,
                                            double& t_out)
{
    const double A = kap[0] * kap[0] + kap[1] * kap[1] + kap[2] * kap[2];
    const double B = u[0] * kap[0] + u[1] * kap[1] + u[2] * kap[2];
    const double C = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] - o.bound2;
    const double disc = B * B - A * C;
    if (!(disc > 0.0)) return false;
    const double sq = sqrt(disc), iA = 1.0 / A;
    t_in = (-B - sq) * iA;
    t_out = (-B + sq) * iA;
    return true;
}

// reciprocals of the three body rates, from one division when none is zero (a bracket needs no
// more than their rounding)
__device__ __forceinline__ void super_inv_rates(const double kap[3], double inv[3])
{
    const double p01 = kap[0] * kap[1], pall = p01 * kap[2];
    if (pall != 0.0) {
        const double r = 1.0 / pall;
        inv[0] = r * kap[1] * kap[2];
        inv[1] = r * kap[0] * kap[2];
        inv[2] = r * p01;
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) inv[i] = kap[i] != 0.0 ? 1.0 / kap[i] : 0.0;
    }
}

// entry of the ray r0 + t k into the body: Newton from the entry of the bracket (box and bounding
// ellipsoid), where phi >= 0 and decreasing.  A point past the minimum of phi (phi' >= 0) with
// phi still positive, or past the bracket, means the line misses: a root would lie before it.
__device__ __forceinline__ bool super_entry(const ObjDev& o, const double r0[3], const double k[3], double& t_hit)
{
    double u[3], kap[3];
    super_line(o, r0, k, u, kap);
    double tin, tout;
    if (!super_bound(o, u, kap, tin, tout)) return false;
    double inv[3];
    super_inv_rates(kap, inv);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (kap[i] == 0.0) {
            if (!(fabs(u[i]) < 1.0)) return false;
        } else {
            const double ta = (-1.0 - u[i]) * inv[i], tb = (1.0 - u[i]) * inv[i];
            tin = fmax(tin, fmin(ta, tb));
            tout = fmin(tout, fmax(ta, tb));
        }
    }
    if (!(tin < tout)) return false;
    double t = tin, prev = INFINITY;
    for (int it = 0; it < 96; ++it) {
        double df;
        const double f = super_phi(o, u, kap, t, df);
        if (!(f > 0.0)) break;
        if (!(df < 0.0)) return false;
        const double step = -f / df;
        t += step;
        if (t > tout) return false;
        // converged: a rounding-sized step, or a small step after a quadratic contraction (the next
        // correction, about step^2 phi'' / 2 phi', is then below rounding)
        if (step <= 4e-16 * fabs(t) || (step <= 1e-9 * fabs(t) && step <= 1e-3 * prev)) break;
        prev = step;
    }
    t_hit = t;
    return true;
}

// chord from surface point r along the inward direction k: Newton from the nearer exit of the
// bracket, where phi >= 0 and increasing, down to the positive root
__device__ __forceinline__ double super_chord(const ObjDev& o, const double r[3], const double k[3])
{
    double u[3], kap[3];
    super_line(o, r, k, u, kap);
    double tin, t;
    if (!super_bound(o, u, kap, tin, t)) return 0.0;
    double inv[3];
    super_inv_rates(kap, inv);
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if (kap[i] != 0.0) t = fmin(t, (copysign(1.0, kap[i]) - u[i]) * inv[i]);
    if (!(t > 0.0)) return 0.0;
    double prev = INFINITY;
    for (int it = 0; it < 96; ++it) {
        double df;
        const double f = super_phi(o, u, kap, t, df);
        if (!(f > 0.0) || !(df > 0.0)) break;
        const double step = f / df;
        t -= step;
        if (step <= 4e-16 * t || (step <= 1e-9 * t && step <= 1e-3 * prev)) break;
        prev = step;
    }
    return t;
}

// g = grad F / 2 at surface point r (world frame) and the body-diagonal half Hessian
// hb_i = e (2e - 1) |u_i|^(2e-2) / a_i^2: the curvature form is sigma_a^T diag(hb) sigma_b / |g|
// with sigma = Rb^T s (body components of the surface vectors)
__device__ __forceinline__ void super_grad(const ObjDev& o, const double r[3], double g[3], double hb[3])
{
    const double dx = r[0] - o.c[0], dy = r[1] - o.c[1], dz = r[2] - o.c[2];
    const double e = o.shape_e;
    double gb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double ui = (o.Rb[i] * dx + o.Rb[3 + i] * dy + o.Rb[6 + i] * dz) * o.inv_a[i];
        const double pw = super_pow(o, fabs(ui));
        gb[i] = e * pw * ui * o.inv_a[i];
        hb[i] = e * (2.0 * e - 1.0) * pw * o.inv_a[i] * o.inv_a[i];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) g[j] = o.Rb[3 * j] * gb[0] + o.Rb[3 * j + 1] * gb[1] + o.Rb[3 * j + 2] * gb[2];
}

// A single-precision exit direction is unit only to 6e-8; the far-field phase s.r_exit and the
// stored direction take it normalised in double precision.
__device__ __forceinline__ void normalize_exit(ExitWave& w)
{
    const double il = rsqrt(w.k[0] * w.k[0] + w.k[1] * w.k[1] + w.k[2] * w.k[2]);
    w.k[0] *= il;
    w.k[1] *= il;
    w.k[2] *= il;
}

// Traces the incident ray at impact point (x, y) for orders 0..pmax; sink.emit(p, ExitWave) is
// called for every order that leaves the object.  T is the working precision of directions,
// bases, curvature, Fresnel and Jones arithmetic; positions and the optical path are double.
// kJ: also carry the transfer matrix T of transverse offsets.  kSuper: the object is a
// superellipsoid (double precision only): entry, chords, normal and curvature come from F above.
template <typename T, bool kJ, class Sink, bool kSuper = false>
__device__ void trace_ray(const ObjDev& o, double x, double y, int pmax, Sink& sink)
{
    static_assert(!kSuper || std::is_same<T, double>::value, "superellipsoids are traced in double precision");
    const T W[6] = {(T)o.W[0], (T)o.W[1], (T)o.W[2], (T)o.W[3], (T)o.W[4], (T)o.W[5]};
    // entry point of the incident ray (plane wave along +z), started below the object
    double r[3] = {x, y, o.zstart};
    T k0v = T(0), k1v = T(0), k2v = T(1);
    // incident wave: k = z, basis (a, b) = (x, -y) so that every basis has a x b = -k
    T a0 = T(1), a1 = T(0), a2 = T(0);
    T q11 = T(0), q12 = T(0), q22 = T(0);
    T E1r = (T)o.jre[0], E1i = (T)o.jim[0], E2r = -(T)o.jre[1], E2i = -(T)o.jim[1];
    T T11 = T(1), T12 = T(0), T21 = T(0), T22 = T(-1);
    int sT = -1;
    T pdet = T(1), cosprod = T(1);
    double path;
    if (!o.src_mode) {
        if constexpr (kSuper) {
            const double kz[3] = {0.0, 0.0, 1.0};
            double t;
            if (!super_entry(o, r, kz, t)) return;
            r[2] += t;
        } else {
            const T kz[3] = {T(0), T(0), T(1)};
            bool ok;
            const double t = chord_to_surface<T>(o, W, r, kz, T(-1), &ok);
            if (!ok) return;
            r[2] += t;
        }
        path = r[2];  // phase of the incident plane wave at the first point (zero at the origin)
    } else if constexpr (std::is_same<T, double>::value) {
        // point source s: the ray toward X = c + x e1 + y e2 meets the surface at distance rho with
        // the spherical wave's curvature I / rho, amplitude 1 / rho and phase k rho; the entry root
        // is solved from the ray's point of closest approach to the centre (no cancellation for a
        // distant source)
        double v[3], g[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            v[i] = o.c[i] + x * o.e1[i] + y * o.e2[i] - o.src[i];
            g[i] = o.src[i] - o.c[i];
        }
        const double dP = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), iP = 1.0 / dP;
        const double k[3] = {v[0] * iP, v[1] * iP, v[2] * iP};
        double rho;
        if constexpr (kSuper) {
            // superellipsoid: the smaller root of the line function from the source
            if (!super_entry(o, o.src, k, rho)) return;
#pragma unroll
            for (int i = 0; i < 3; ++i) r[i] = o.src[i] + rho * k[i];
        } else {
            const double t0 = -(k[0] * g[0] + k[1] * g[1] + k[2] * g[2]);
            const double f[3] = {g[0] + t0 * k[0], g[1] + t0 * k[1], g[2] + t0 * k[2]};
            double wkx, wky, wkz, wfx, wfy, wfz;
            symv(o.W, k[0], k[1], k[2], wkx, wky, wkz);
            symv(o.W, f[0], f[1], f[2], wfx, wfy, wfz);
            const double A = k[0] * wkx + k[1] * wky + k[2] * wkz, B = k[0] * wfx + k[1] * wfy + k[2] * wfz;
            const double Cq = f[0] * wfx + f[1] * wfy + f[2] * wfz - 1.0;
            const double disc = B * B - A * Cq;
            if (!(disc > 0.0)) return;
            const double u = (-B - sqrt(disc)) / A;
            rho = t0 + u;
            if (!(rho > 0.0)) return;
#pragma unroll
            for (int i = 0; i < 3; ++i) r[i] = o.c[i] + f[i] + u * k[i];
        }
        k0v = k[0];
        k1v = k[1];
        k2v = k[2];
        // basis a = e1 made perpendicular to k, b = a x k
        const double ek = o.e1[0] * k[0] + o.e1[1] * k[1] + o.e1[2] * k[2];
        double ax = o.e1[0] - ek * k[0], ay = o.e1[1] - ek * k[1], az = o.e1[2] - ek * k[2];
        const double ia = rsqrt(ax * ax + ay * ay + az * az);
        ax *= ia;
        ay *= ia;
        az *= ia;
        const double bx = ay * k[2] - az * k[1], by = az * k[0] - ax * k[2], bz = ax * k[1] - ay * k[0];
        a0 = ax;
        a1 = ay;
        a2 = az;
        const double irho = 1.0 / rho;
        q11 = irho;
        q22 = irho;
        // E = (p . a, p . b) / rho with p = jones_x e1 + jones_y e2 (its part along k drops out)
        const double a_e1 = ax * o.e1[0] + ay * o.e1[1] + az * o.e1[2], a_e2 = ax * o.e2[0] + ay * o.e2[1] + az * o.e2[2];
        const double b_e1 = bx * o.e1[0] + by * o.e1[1] + bz * o.e1[2], b_e2 = bx * o.e2[0] + by * o.e2[1] + bz * o.e2[2];
        E1r = (o.jre[0] * a_e1 + o.jre[1] * a_e2) * irho;
        E1i = (o.jim[0] * a_e1 + o.jim[1] * a_e2) * irho;
        E2r = (o.jre[0] * b_e1 + o.jre[1] * b_e2) * irho;
        E2i = (o.jim[0] * b_e1 + o.jim[1] * b_e2) * irho;
        // transverse offset at the surface per unit (x, y) of the grid's plane
        const double sc = rho * iP;
        T11 = sc * a_e1;
        T12 = sc * a_e2;
        T21 = sc * b_e1;
        T22 = sc * b_e2;
        const double dT = T11 * T22 - T12 * T21;
        sT = dT > 0.0 ? 1 : -1;
        cosprod = fabs(dT);  // dA/dOmega of the caustic test counts grid area: |det T| of the start
        path = rho;
    } else {
        return;  // point sources are traced in double precision (the entry points reject others)
    }
    int nf = 0;
    T n_in = T(1);
    double n_in_d = 1.0;  // the same index in double precision, for the optical path
    // reciprocal wave numbers of the two media, once per ray
    const T k0 = (T)o.k0, mo = (T)o.m;
    const T ik_host = T(1) / k0, ik_obj = T(1) / (k0 * mo), inv_mo = T(1) / mo;
    // in double precision the gradient at the next surface point is carried forward:
    // W (r + d k - c) = W (r - c) + d W k, with W k from the chord
    constexpr bool kCarryGrad = sizeof(T) == sizeof(double) && !kSuper;
    T gnext[3] = {T(0), T(0), T(0)};
    for (int q = 1; q <= pmax + 1; ++q) {
        const T n_out = (q == 1) ? mo : T(1);
        // outward normal n = W (r - c) / |W (r - c)|
        T gx, gy, gz;
        T hb[3] = {T(0), T(0), T(0)};
        if constexpr (kSuper) {
            double gs[3];
            super_grad(o, r, gs, hb);
            gx = gs[0];
            gy = gs[1];
            gz = gs[2];
        } else if (kCarryGrad && q > 1) {
            gx = gnext[0];
            gy = gnext[1];
            gz = gnext[2];
        } else {
            symvT(W, (T)(r[0] - o.c[0]), (T)(r[1] - o.c[1]), (T)(r[2] - o.c[2]), gx, gy, gz);
        }
        const T inv_gn = rsqrt(gx * gx + gy * gy + gz * gz);
        const T nx = gx * inv_gn, ny = gy * inv_gn, nz = gz * inv_gn;
        const T ci = k0v * nx + k1v * ny + k2v * nz;  // signed cosine of incidence
        if (fabs(ci) < T(1e-9)) return;               // grazing: P' singular
        // e_perp = k x n / |k x n| (normal of the incident plane)
        T ex = k1v * nz - k2v * ny, ey = k2v * nx - k0v * nz, ez = k0v * ny - k1v * nx;
        const T el2 = ex * ex + ey * ey + ez * ez;
        T il = T(0);
        if (el2 < T(1e-24)) {
            ex = a0; ey = a1; ez = a2;
        } else {
            il = rsqrt(el2);
            ex *= il; ey *= il; ez *= il;
        }
        // rotation of the incident basis (a, b = a x k) onto (e_perp, e_perp x k): cr = a.e_perp and
        // sr = b.e_perp = ((a.k) ci - a.n) / |k x n|, which is -(a.n) / |k x n| since a is normal to k
        // (0 where e_perp falls back to a); the other precisions, whose a.k is zero only to their
        // rounding, form b
        const T cr = a0 * ex + a1 * ey + a2 * ez;
        T sr;
        if constexpr (!std::is_same<T, double>::value) {
            const T b0 = a1 * k2v - a2 * k1v, b1 = a2 * k0v - a0 * k2v, b2 = a0 * k1v - a1 * k0v;
            sr = b0 * ex + b1 * ey + b2 * ez;
        } else {
            sr = -(a0 * nx + a1 * ny + a2 * nz) * il;
        }
        const T Ep_r = E1r * cr + E2r * sr, Ep_i = E1i * cr + E2i * sr;
        const T Eq_r = -E1r * sr + E2r * cr, Eq_i = -E1i * sr + E2i * cr;
        const T cc = cr * cr, ss = sr * sr, cs = cr * sr;
        const T Qe11 = cc * q11 + T(2) * cs * q12 + ss * q22;
        const T Qe12 = -cs * q11 + (cc - ss) * q12 + cs * q22;
        const T Qe22 = ss * q11 - T(2) * cs * q12 + cc * q22;
        T Te11 = T(0), Te12 = T(0), Te21 = T(0), Te22 = T(0);
        if (kJ) {
            Te11 = cr * T11 + sr * T21;
            Te12 = cr * T12 + sr * T22;
            Te21 = -sr * T11 + cr * T21;
            Te22 = -sr * T12 + cr * T22;
        }
        // surface curvature matrix in (s1, s2) = (e_perp, n x e_perp): C_ab = s_a^T W s_b / |grad|
        const T s2x = ny * ez - nz * ey, s2y = nz * ex - nx * ez, s2z = nx * ey - ny * ex;
        T C11, C12, C22;
        if constexpr (kSuper) {
            // C_ab = sigma_a^T diag(hb) sigma_b / |g|, sigma = Rb^T s
            C11 = C12 = C22 = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T p1 = o.Rb[i] * ex + o.Rb[3 + i] * ey + o.Rb[6 + i] * ez;
                const T p2 = o.Rb[i] * s2x + o.Rb[3 + i] * s2y + o.Rb[6 + i] * s2z;
                C11 += hb[i] * p1 * p1;
                C12 += hb[i] * p1 * p2;
                C22 += hb[i] * p2 * p2;
            }
            C11 *= inv_gn;
            C12 *= inv_gn;
            C22 *= inv_gn;
        } else {
            T wex, wey, wez, wsx, wsy, wsz;
            symvT(W, ex, ey, ez, wex, wey, wez);
            symvT(W, s2x, s2y, s2z, wsx, wsy, wsz);
            C11 = (ex * wex + ey * wey + ez * wez) * inv_gn;
            C12 = (ex * wsx + ey * wsy + ez * wsz) * inv_gn;
            C22 = (s2x * wsx + s2y * wsy + s2z * wsz) * inv_gn;
        }
        // Eq. (SnellVec): the common tangential wave vector tau = k_i k - k_in n has |tau|^2 =
        // k_i^2 - k_in^2 for a unit k; single precision, whose k is unit only to 6e-8, forms tau
        const T ki = k0 * n_in, kt = k0 * n_out;
        const T kin = ki * ci;
        constexpr bool kTau = std::is_same<T, float>::value;
        T tx = T(0), ty = T(0), tz = T(0), ktn2;
        if constexpr (kTau) {
            tx = ki * k0v - kin * nx;
            ty = ki * k1v - kin * ny;
            tz = ki * k2v - kin * nz;
            ktn2 = kt * kt - (tx * tx + ty * ty + tz * tz);
        } else {
            ktn2 = (kt * kt - ki * ki) + kin * kin;
        }
        const T mr = (q == 1) ? mo : inv_mo, mr2 = mr * mr;  // n_out / n_in
        const T inv_ki = (q == 1) ? ik_host : ik_obj, inv_kt = (q == 1) ? ik_obj : ik_host;
        const bool tok = ktn2 > T(0);
        T ktn = T(0);
        // double precision: |k_tn| and 1 / |k_tn| from one reciprocal square root (1 ulp)
        constexpr bool kRootRecip = std::is_same<T, double>::value;
        T rktn = T(0);
        if (tok) {
            if constexpr (kRootRecip) {
                rktn = rsqrt(ktn2);
                ktn = copysign(ktn2 * rktn, kin);
            } else {
                ktn = copysign(sqrt(ktn2), kin);
            }
        }
        // directions of the reflected wave, k_l = (tau - k_in n) / k_i = k - 2 ci n, and of the
        // transmitted one, k_t = (tau + k_tn n) / k_t (= rio k + g n, rio = k_i / k_t, g = (k_tn - k_in) / k_t)
        const T ci2 = T(2) * ci;
        const T lk0 = k0v - ci2 * nx, lk1 = k1v - ci2 * ny, lk2 = k2v - ci2 * nz;
        T tk0 = T(0), tk1 = T(0), tk2 = T(0), dn = T(0), rio = T(0), g = T(0);
        if (tok) {
            dn = ktn - kin;
            if constexpr (kTau) {
                tk0 = (tx + ktn * nx) * inv_kt;
                tk1 = (ty + ktn * ny) * inv_kt;
                tk2 = (tz + ktn * nz) * inv_kt;
            } else {
                rio = ki * inv_kt;
                g = dn * inv_kt;
                tk0 = rio * k0v + g * nx;
                tk1 = rio * k1v + g * ny;
                tk2 = rio * k2v + g * nz;
            }
        }
        // in double precision, W k and A = k^T W k of the chord that follows (along the transmitted
        // wave at the entry, the reflected one after it): its 1/A joins the reciprocal below
        constexpr bool kFoldA = std::is_same<T, double>::value && !kSuper;
        T cwk[3] = {T(0), T(0), T(0)}, cAk = T(1), iAk = T(1);
        if (kFoldA && q <= pmax && (q > 1 || tok)) {
            const T c0 = q == 1 ? tk0 : lk0, c1 = q == 1 ? tk1 : lk1, c2 = q == 1 ? tk2 : lk2;
            symvT(W, c0, c1, c2, cwk[0], cwk[1], cwk[2]);
            cAk = c0 * cwk[0] + c1 * cwk[1] + c2 * cwk[2];
        }
        // Eq. (Fres)
        T rp_r, rp_i, rq_r, rq_i, tp_r = T(0), tq_r = T(0);
        T inv_ci, inv_ktn = T(0);
        if (tok) {
            // one reciprocal serves 1/(k_in + k_tn), 1/(m^2 k_in + k_tn), 1/ci, 1/k_tn (and 1/A)
            const T den1 = kin + ktn, den2 = mr2 * kin + ktn;
            const T aa = den1 * den2, bb = ci * ktn, P = aa * bb;
            const T invA = T(1) / (P * cAk);
            const T inv = cAk * invA;
            iAk = P * invA;
            const T i1 = den2 * bb * inv, i2 = den1 * bb * inv;
            inv_ci = aa * ktn * inv;
            if constexpr (kRootRecip) inv_ktn = copysign(rktn, kin);
            else inv_ktn = aa * ci * inv;
            rp_r = (kin - ktn) * i1;
            rq_r = (mr2 * kin - ktn) * i2;
            tp_r = T(2) * kin * i1;
            tq_r = T(2) * mr * kin * i2;
            rp_i = T(0);
            rq_i = T(0);
        } else {
            // total internal reflection: k_tn = i sign(k_in) kappa
            const T kap = copysign(sqrt(-ktn2), kin);
            const T u = mr2 * kin;
            T d1, d2;
            if constexpr (kFoldA) {
                // one reciprocal for both denominators, 1/ci and 1/A
                const T D1 = kin * kin + kap * kap, D2 = u * u + kap * kap, P = D1 * D2 * ci;
                const T invA = T(1) / (P * cAk);
                const T inv = cAk * invA;
                iAk = P * invA;
                d1 = D2 * ci * inv;
                d2 = D1 * ci * inv;
                inv_ci = D1 * D2 * inv;
            } else {
                d1 = T(1) / (kin * kin + kap * kap);
                d2 = T(1) / (u * u + kap * kap);
                inv_ci = T(1) / ci;
            }
            rp_r = (kin * kin - kap * kap) * d1;
            rp_i = T(-2) * kin * kap * d1;
            rq_r = (u * u - kap * kap) * d2;
            rq_i = T(-2) * u * kap * d2;
        }
        // reflected wave: k_l = tau - k_in n, signed cosine -ci; Eq. (WavefrontEqVec) in the
        // diagonal bases with n.(k_l - k_i) = -2 k_in
        T lq11 = T(0), lq12 = T(0), lq22 = T(0);
        T le1r = T(0), le1i = T(0), le2r = T(0), le2i = T(0), lt21 = T(0), lt22 = T(0);
        // the wave reflected inside at the last interaction is never used
        if (q == 1 || q <= pmax) {
            // the entries of the general equation with k' = k_i and n.(k_l - k_i) = -2 k_in, the
            // factors k_i and ci cancelled exactly
            lq11 = Qe11 - ci2 * C11;
            lq12 = -Qe12 - T(2) * C12;
            lq22 = Qe22 - T(2) * C22 * inv_ci;
            if (std::is_same<T, double>::value && tok) {  // real coefficients
                le1r = rp_r * Ep_r;
                le1i = rp_r * Ep_i;
                le2r = rq_r * Eq_r;
                le2i = rq_r * Eq_i;
            } else {
                le1r = rp_r * Ep_r - rp_i * Ep_i;
                le1i = rp_r * Ep_i + rp_i * Ep_r;
                le2r = rq_r * Eq_r - rq_i * Eq_i;
                le2i = rq_r * Eq_i + rq_i * Eq_r;
            }
            if (kJ) {
                lt21 = -Te21;
                lt22 = -Te22;
            }
        }
        T tq11 = T(0), tq12 = T(0), tq22 = T(0);
        T te1r = T(0), te1i = T(0), te2r = T(0), te2i = T(0), tt21 = T(0), tt22 = T(0);
        T ct = T(0);
        if (tok) {
            const T inv_ct = kt * inv_ktn;
            ct = ktn * inv_kt;  // signed cosine of the transmitted wave
            tq12 = (kin * Qe12 - C12 * dn) * inv_ktn;  // inv_kt inv_ct = 1 / k_tn
            if constexpr (kTau) {
                tq11 = (ki * Qe11 + C11 * dn) * inv_kt;
                tq22 = (ki * ci * ci * Qe22 + C22 * dn) * inv_kt * inv_ct * inv_ct;
            } else {
                tq11 = rio * Qe11 + C11 * g;
                tq22 = (rio * ci * ci * Qe22 + C22 * g) * (inv_ct * inv_ct);
            }
            te1r = tp_r * Ep_r;
            te1i = tp_r * Ep_i;
            te2r = tq_r * Eq_r;
            te2i = tq_r * Eq_i;
            if (kJ) {
                const T f = ct * inv_ci;
                tt21 = f * Te21;
                tt22 = f * Te22;
            }
        }
        const T cos_ratio = tok ? fabs(ct * inv_ci) : T(0);
        ExitWave w;
        if (q == 1) {
            // order 0: external reflection (Eq. epsilon_VCRM, p = 0)
            w.k[0] = lk0; w.k[1] = lk1; w.k[2] = lk2;
            w.q11 = lq11; w.q12 = lq12; w.q22 = lq22;
            w.e1r = le1r; w.e1i = le1i; w.e2r = le2r; w.e2i = le2i;
            if (kJ) { w.t11 = Te11; w.t12 = Te12; w.t21 = lt21; w.t22 = lt22; }
            w.ep[0] = ex; w.ep[1] = ey; w.ep[2] = ez;
            w.pdet = 1.0;
            w.cosprod = cosprod;  // 1 for a plane wave; |det T| of the start for a point source
            w.path = path;
            w.r[0] = r[0]; w.r[1] = r[1]; w.r[2] = r[2];
            w.nf_legs = 0;
            w.sT = -sT;
            if (sizeof(T) == sizeof(float)) normalize_exit(w);
            sink.emit(0, w);
            if (!tok) return;
            k0v = tk0; k1v = tk1; k2v = tk2;
            q11 = tq11; q12 = tq12; q22 = tq22;
            E1r = te1r; E1i = te1i; E2r = te2r; E2i = te2i;
            if (kJ) { T11 = Te11; T12 = Te12; T21 = tt21; T22 = tt22; }
            cosprod *= cos_ratio;
            n_in = n_out;  // the transmitted wave continues inside
            n_in_d = o.m;
        } else {
            // order q-1 leaves by refraction; the reflected wave stays inside
            if (tok) {
                w.k[0] = tk0; w.k[1] = tk1; w.k[2] = tk2;
                w.q11 = tq11; w.q12 = tq12; w.q22 = tq22;
                w.e1r = te1r; w.e1i = te1i; w.e2r = te2r; w.e2i = te2i;
                if (kJ) { w.t11 = Te11; w.t12 = Te12; w.t21 = tt21; w.t22 = tt22; }
                w.ep[0] = ex; w.ep[1] = ey; w.ep[2] = ez;
                w.pdet = pdet;
                w.cosprod = cosprod * cos_ratio;
                w.path = path;
                w.r[0] = r[0]; w.r[1] = r[1]; w.r[2] = r[2];
                w.nf_legs = nf;
                w.sT = sT;
                if (sizeof(T) == sizeof(float)) normalize_exit(w);
                sink.emit(q - 1, w);
            }
            k0v = lk0; k1v = lk1; k2v = lk2;
            q11 = lq11; q12 = lq12; q22 = lq22;
            E1r = le1r; E1i = le1i; E2r = le2r; E2i = le2i;
            if (kJ) { T11 = Te11; T12 = Te12; T21 = lt21; T22 = lt22; }
            sT = -sT;
        }
        a0 = ex; a1 = ey; a2 = ez;
        if (q == pmax + 1) break;
        // chord to the next surface point along the inward direction
        const T kk[3] = {k0v, k1v, k2v};
        T wk[3] = {T(0), T(0), T(0)};
        double dd;
        if constexpr (kSuper) {
            dd = super_chord(o, r, kk);
        } else if constexpr (kFoldA) {
            const T wg[3] = {gx, gy, gz};
            dd = chord_inside<T>(o, r, kk, cAk, iAk, wg);
            wk[0] = cwk[0];
            wk[1] = cwk[1];
            wk[2] = cwk[2];
        } else {
            bool ok;
            const T wg[3] = {gx, gy, gz};
            dd = chord_to_surface<T>(o, W, r, kk, T(1), &ok, wg, wk);
        }
        if (!(dd > 0.0)) return;
        const T d = (T)dd;
        if constexpr (kCarryGrad) {
            gnext[0] = gx + d * wk[0];
            gnext[1] = gy + d * wk[1];
            gnext[2] = gz + d * wk[2];
        }
        // free propagation: Q(d) = Q (I + d Q)^{-1} = (Q + d det Q I) / det(I + d Q)
        const T A11 = T(1) + d * q11, A22 = T(1) + d * q22, A12 = d * q12;
        const T detA = A11 * A22 - A12 * A12;
        if (detA == T(0)) return;
        const T idet = T(1) / detA;
        const T dq = q11 * q22 - q12 * q12;
        q11 = (q11 + d * dq) * idet;
        q12 = q12 * idet;
        q22 = (q22 + d * dq) * idet;
        pdet *= fabs(detA);
        if constexpr (std::is_same<T, double>::value) nf += neg_eigs_td(A11 + A22, detA);
        else nf += neg_eigs_sym((double)A11, (double)A12, (double)A22);
        if (detA < T(0)) sT = -sT;
        if (kJ) {
            const T n11 = A11 * T11 + A12 * T21, n12 = A11 * T12 + A12 * T22;
            const T n21 = A12 * T11 + A22 * T21, n22 = A12 * T12 + A22 * T22;
            T11 = n11; T12 = n12; T21 = n21; T22 = n22;
        }
        // dd is the parameter along k; in single precision |k| = 1 only to 6e-8, so the optical
        // path takes the segment's true length dd |k|, evaluated in double precision
        double seg = dd;
        if (sizeof(T) == sizeof(float)) {
            const double kx = k0v, ky = k1v, kz = k2v;
            seg = dd * sqrt(kx * kx + ky * ky + kz * kz);
        }
        path += n_in_d * seg;
        r[0] += dd * (double)k0v;
        r[1] += dd * (double)k1v;
        r[2] += dd * (double)k2v;
    }
}

template <bool kJ, class Sink>
__device__ __forceinline__ void trace_ray_fp64(const ObjDev& o, double x, double y, int pmax, Sink& sink)
{
    trace_ray<double, kJ>(o, x, y, pmax, sink);
}

}  // namespace rtw
