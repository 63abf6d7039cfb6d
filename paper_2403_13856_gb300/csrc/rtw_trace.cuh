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

__device__ __forceinline__ int neg_eigs_sym(double a11, double a12, double a22)
{
    double det = a11 * a22 - a12 * a12, tr = a11 + a22;
    if (det < 0.0) return 1;
    if (det > 0.0 && tr < 0.0) return 2;
    if (det == 0.0 && tr < 0.0) return 1;
    return 0;
}

__device__ __forceinline__ void symv(const double* W, double x, double y, double z, double& ox, double& oy,
                                     double& oz)
{
    ox = W[0] * x + W[1] * y + W[2] * z;
    oy = W[1] * x + W[3] * y + W[4] * z;
    oz = W[2] * x + W[4] * y + W[5] * z;
}

// Far-field record of an exit wave: F = E' sqrt(D_legs / |det Q'|) (-i)^{N_f}, Psi = k0 (L - s.r),
// with sqrt(D) = 1 / sqrt(|det Q'| prod |det(I + d Q)|).
__device__ __forceinline__ bool far_record(const ObjDev& o, const ExitWave& w, FarRecord& fr)
{
    double detQ = w.q11 * w.q22 - w.q12 * w.q12;
    if (!(fabs(detQ) > 0.0) || !isfinite(detQ)) return false;
    int nf = w.nf_legs + neg_eigs_sym(w.q11, w.q12, w.q22);
    double amp = rsqrt(fabs(detQ) * w.pdet);
    double D = amp * amp;
    double pr = 1.0, pi = 0.0;  // (-i)^nf
    switch (nf & 3) {
    case 1: pr = 0.0; pi = -1.0; break;
    case 2: pr = -1.0; pi = 0.0; break;
    case 3: pr = 0.0; pi = 1.0; break;
    default: break;
    }
    double a1r = amp * (w.e1r * pr - w.e1i * pi), a1i = amp * (w.e1r * pi + w.e1i * pr);
    double a2r = amp * (w.e2r * pr - w.e2i * pi), a2i = amp * (w.e2r * pi + w.e2i * pr);
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
    uint32_t f = kFlagValid | (orient > 0 ? kFlagOrient : 0u) | (D > o.cap * w.cosprod ? kFlagCaustic : 0u);
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
    x = o.c[0] + ((double)ix + 0.5 - (double)(o.nx / 2)) * o.h;
    y = o.c[1] + ((double)iy + 0.5 - (double)(o.ny / 2)) * o.h;
    double dx = x - o.c[0], dy = y - o.c[1];
    double qf = dx * (o.S[0] * dx + o.S[1] * dy) + dy * (o.S[1] * dx + o.S[2] * dy);
    return qf < 1.0;
}

// Traces the incident ray at impact point (x, y) for orders 0..pmax; sink.emit(p, ExitWave) is
// called for every order that leaves the object.  kJ: also carry the transfer matrix T.
template <bool kJ, class Sink>
__device__ void trace_ray_fp64(const ObjDev& o, double x, double y, int pmax, Sink& sink)
{
    const double* W = o.W;
    // entry point of the incident ray (plane wave along +z), started below the object
    double ux = x - o.c[0], uy = y - o.c[1], uz = o.zstart - o.c[2];
    double wx, wy, wz;
    symv(W, ux, uy, uz, wx, wy, wz);
    double A = W[5], B = wz, Cq = ux * wx + uy * wy + uz * wz - 1.0;
    double disc = B * B - A * Cq;
    if (!(disc > 0.0)) return;
    double t = (-B - sqrt(disc)) / A;
    double r0 = x, r1 = y, r2 = o.zstart + t;
    // incident wave: k = z, basis (a, b) = (x, -y) so that every basis has a x b = -k
    double k0v = 0.0, k1v = 0.0, k2v = 1.0;
    double a0 = 1.0, a1 = 0.0, a2 = 0.0;
    double q11 = 0.0, q12 = 0.0, q22 = 0.0;
    double E1r = o.jre[0], E1i = o.jim[0], E2r = -o.jre[1], E2i = -o.jim[1];
    double T11 = 1.0, T12 = 0.0, T21 = 0.0, T22 = -1.0;
    int sT = -1;
    double path = r2;  // phase of the incident plane wave at the first point (zero at the origin)
    double pdet = 1.0, cosprod = 1.0;
    int nf = 0;
    double n_in = 1.0;
    // reciprocal wave numbers of the two media, once per ray
    const double ik_host = 1.0 / o.k0, ik_obj = 1.0 / (o.k0 * o.m);
    for (int q = 1; q <= pmax + 1; ++q) {
        const double n_out = (q == 1) ? o.m : 1.0;
        // outward normal n = W (r - c) / |W (r - c)|
        double gx, gy, gz;
        symv(W, r0 - o.c[0], r1 - o.c[1], r2 - o.c[2], gx, gy, gz);
        double inv_gn = rsqrt(gx * gx + gy * gy + gz * gz);
        double nx = gx * inv_gn, ny = gy * inv_gn, nz = gz * inv_gn;
        double ci = k0v * nx + k1v * ny + k2v * nz;  // signed cosine of incidence
        if (fabs(ci) < 1e-9) return;                 // grazing: P' singular
        // e_perp = k x n / |k x n| (normal of the incident plane)
        double ex = k1v * nz - k2v * ny, ey = k2v * nx - k0v * nz, ez = k0v * ny - k1v * nx;
        double el2 = ex * ex + ey * ey + ez * ez;
        if (el2 < 1e-24) {
            ex = a0; ey = a1; ez = a2;
        } else {
            double il = rsqrt(el2);
            ex *= il; ey *= il; ez *= il;
        }
        // rotation of the incident basis (a, b = a x k) onto (e_perp, e_perp x k)
        double b0 = a1 * k2v - a2 * k1v, b1 = a2 * k0v - a0 * k2v, b2 = a0 * k1v - a1 * k0v;
        double cr = a0 * ex + a1 * ey + a2 * ez, sr = b0 * ex + b1 * ey + b2 * ez;
        double Ep_r = E1r * cr + E2r * sr, Ep_i = E1i * cr + E2i * sr;
        double Eq_r = -E1r * sr + E2r * cr, Eq_i = -E1i * sr + E2i * cr;
        double cc = cr * cr, ss = sr * sr, cs = cr * sr;
        double Qe11 = cc * q11 + 2.0 * cs * q12 + ss * q22;
        double Qe12 = -cs * q11 + (cc - ss) * q12 + cs * q22;
        double Qe22 = ss * q11 - 2.0 * cs * q12 + cc * q22;
        double Te11 = 0, Te12 = 0, Te21 = 0, Te22 = 0;
        if (kJ) {
            Te11 = cr * T11 + sr * T21;
            Te12 = cr * T12 + sr * T22;
            Te21 = -sr * T11 + cr * T21;
            Te22 = -sr * T12 + cr * T22;
        }
        // surface curvature matrix in (s1, s2) = (e_perp, n x e_perp): C_ab = s_a^T W s_b / |grad|
        double s2x = ny * ez - nz * ey, s2y = nz * ex - nx * ez, s2z = nx * ey - ny * ex;
        double wex, wey, wez, wsx, wsy, wsz;
        symv(W, ex, ey, ez, wex, wey, wez);
        symv(W, s2x, s2y, s2z, wsx, wsy, wsz);
        double C11 = (ex * wex + ey * wey + ez * wez) * inv_gn;
        double C12 = (ex * wsx + ey * wsy + ez * wsz) * inv_gn;
        double C22 = (s2x * wsx + s2y * wsy + s2z * wsz) * inv_gn;
        // Eq. (SnellVec): common tangential wave vector
        const double ki = o.k0 * n_in, kt = o.k0 * n_out;
        const double kin = ki * ci;
        double tx = ki * k0v - kin * nx, ty = ki * k1v - kin * ny, tz = ki * k2v - kin * nz;
        double tau2 = tx * tx + ty * ty + tz * tz;
        double ktn2 = kt * kt - tau2;
        const double mr = n_out / n_in, mr2 = mr * mr;
        // Eq. (Fres)
        bool tok = ktn2 > 0.0;
        double ktn = 0.0;
        double rp_r, rp_i, rq_r, rq_i, tp_r = 0.0, tq_r = 0.0;
        double inv_ci, inv_ktn = 0.0;
        if (tok) {
            ktn = copysign(sqrt(ktn2), kin);
            // one reciprocal serves 1/(k_in + k_tn), 1/(m^2 k_in + k_tn), 1/ci and 1/k_tn
            const double den1 = kin + ktn, den2 = mr2 * kin + ktn;
            const double aa = den1 * den2, bb = ci * ktn;
            const double inv = 1.0 / (aa * bb);
            const double i1 = den2 * bb * inv, i2 = den1 * bb * inv;
            inv_ci = aa * ktn * inv;
            inv_ktn = aa * ci * inv;
            rp_r = (kin - ktn) * i1;
            rq_r = (mr2 * kin - ktn) * i2;
            tp_r = 2.0 * kin * i1;
            tq_r = 2.0 * mr * kin * i2;
            rp_i = 0.0;
            rq_i = 0.0;
        } else {
            // total internal reflection: k_tn = i sign(k_in) kappa
            double kap = copysign(sqrt(-ktn2), kin);
            double d1 = 1.0 / (kin * kin + kap * kap);
            rp_r = (kin * kin - kap * kap) * d1;
            rp_i = -2.0 * kin * kap * d1;
            double u = mr2 * kin;
            double d2 = 1.0 / (u * u + kap * kap);
            rq_r = (u * u - kap * kap) * d2;
            rq_i = -2.0 * u * kap * d2;
            inv_ci = 1.0 / ci;
        }
        const double inv_ki = (q == 1) ? ik_host : ik_obj, inv_kt = (q == 1) ? ik_obj : ik_host;
        // reflected wave: k_l = tau - k_in n, signed cosine -ci; Eq. (WavefrontEqVec) in the
        // diagonal bases with n.(k_l - k_i) = -2 k_in
        ExitWave wl;
        {
            wl.k[0] = (tx - kin * nx) * inv_ki;
            wl.k[1] = (ty - kin * ny) * inv_ki;
            wl.k[2] = (tz - kin * nz) * inv_ki;
            double dn = -2.0 * kin;
            wl.q11 = (ki * Qe11 + C11 * dn) * inv_ki;
            wl.q12 = (-ki * ci * Qe12 + C12 * dn) * inv_ki * inv_ci;
            wl.q22 = (ki * ci * ci * Qe22 + C22 * dn) * inv_ki * inv_ci * inv_ci;
            wl.e1r = rp_r * Ep_r - rp_i * Ep_i;
            wl.e1i = rp_r * Ep_i + rp_i * Ep_r;
            wl.e2r = rq_r * Eq_r - rq_i * Eq_i;
            wl.e2i = rq_r * Eq_i + rq_i * Eq_r;
            if (kJ) {
                wl.t11 = Te11; wl.t12 = Te12; wl.t21 = -Te21; wl.t22 = -Te22;
            }
        }
        ExitWave wt;
        double ct = 0.0;
        if (tok) {
            wt.k[0] = (tx + ktn * nx) * inv_kt;
            wt.k[1] = (ty + ktn * ny) * inv_kt;
            wt.k[2] = (tz + ktn * nz) * inv_kt;
            ct = ktn * inv_kt;  // signed cosine of the transmitted wave
            double dn = ktn - kin;
            double inv_ct = kt * inv_ktn;
            wt.q11 = (ki * Qe11 + C11 * dn) * inv_kt;
            wt.q12 = -(-ki * ci * Qe12 + C12 * dn) * inv_kt * inv_ct;
            wt.q22 = (ki * ci * ci * Qe22 + C22 * dn) * inv_kt * inv_ct * inv_ct;
            wt.e1r = tp_r * Ep_r;
            wt.e1i = tp_r * Ep_i;
            wt.e2r = tq_r * Eq_r;
            wt.e2i = tq_r * Eq_i;
            if (kJ) {
                double f = ct / ci;
                wt.t11 = Te11; wt.t12 = Te12; wt.t21 = f * Te21; wt.t22 = f * Te22;
            }
        }
        const double cos_ratio = tok ? fabs(ct / ci) : 0.0;
        if (q == 1) {
            // order 0: external reflection (Eq. epsilon_VCRM, p = 0)
            wl.ep[0] = ex; wl.ep[1] = ey; wl.ep[2] = ez;
            wl.pdet = 1.0;
            wl.cosprod = 1.0;
            wl.path = path;
            wl.r[0] = r0; wl.r[1] = r1; wl.r[2] = r2;
            wl.nf_legs = 0;
            wl.sT = -sT;
            sink.emit(0, wl);
            if (!tok) return;
            k0v = wt.k[0]; k1v = wt.k[1]; k2v = wt.k[2];
            q11 = wt.q11; q12 = wt.q12; q22 = wt.q22;
            E1r = wt.e1r; E1i = wt.e1i; E2r = wt.e2r; E2i = wt.e2i;
            if (kJ) { T11 = wt.t11; T12 = wt.t12; T21 = wt.t21; T22 = wt.t22; }
            cosprod *= cos_ratio;
        } else {
            // order q-1 leaves by refraction; the reflected wave stays inside
            if (tok) {
                wt.ep[0] = ex; wt.ep[1] = ey; wt.ep[2] = ez;
                wt.pdet = pdet;
                wt.cosprod = cosprod * cos_ratio;
                wt.path = path;
                wt.r[0] = r0; wt.r[1] = r1; wt.r[2] = r2;
                wt.nf_legs = nf;
                wt.sT = sT;
                sink.emit(q - 1, wt);
            }
            k0v = wl.k[0]; k1v = wl.k[1]; k2v = wl.k[2];
            q11 = wl.q11; q12 = wl.q12; q22 = wl.q22;
            E1r = wl.e1r; E1i = wl.e1i; E2r = wl.e2r; E2i = wl.e2i;
            if (kJ) { T11 = wl.t11; T12 = wl.t12; T21 = wl.t21; T22 = wl.t22; }
            sT = -sT;
        }
        a0 = ex; a1 = ey; a2 = ez;
        if (q == 1) n_in = n_out;  // the transmitted wave continues inside
        if (q == pmax + 1) break;
        // chord to the next surface point along the inward direction
        double px = r0 - o.c[0], py = r1 - o.c[1], pz = r2 - o.c[2];
        double wkx, wky, wkz, wpx, wpy, wpz;
        symv(W, k0v, k1v, k2v, wkx, wky, wkz);
        symv(W, px, py, pz, wpx, wpy, wpz);
        double Ak = k0v * wkx + k1v * wky + k2v * wkz;
        double Bk = k0v * wpx + k1v * wpy + k2v * wpz;
        double Ck = px * wpx + py * wpy + pz * wpz - 1.0;
        double dk = Bk * Bk - Ak * Ck;
        if (dk < 0.0) dk = 0.0;
        double d = (-Bk + sqrt(dk)) / Ak;
        if (!(d > 0.0)) return;
        // free propagation: Q(d) = Q (I + d Q)^{-1} = (Q + d det Q I) / det(I + d Q)
        double A11 = 1.0 + d * q11, A22 = 1.0 + d * q22, A12 = d * q12;
        double detA = A11 * A22 - A12 * A12;
        if (detA == 0.0) return;
        double idet = 1.0 / detA;
        double dq = q11 * q22 - q12 * q12;
        q11 = (q11 + d * dq) * idet;
        q12 = q12 * idet;
        q22 = (q22 + d * dq) * idet;
        pdet *= fabs(detA);
        nf += neg_eigs_sym(A11, A12, A22);
        if (detA < 0.0) sT = -sT;
        if (kJ) {
            double n11 = A11 * T11 + A12 * T21, n12 = A11 * T12 + A12 * T22;
            double n21 = A12 * T11 + A22 * T21, n22 = A12 * T12 + A22 * T22;
            T11 = n11; T12 = n12; T21 = n21; T22 = n22;
        }
        path += n_in * d;
        r0 += d * k0v;
        r1 += d * k1v;
        r2 += d * k2v;
    }
}

}  // namespace rtw
