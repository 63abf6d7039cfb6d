// rtw_device.cuh -- device helpers shared by the dense field and the learned proposal:
// accumulation of F e^{i Psi} onto (e_theta, e_phi), and Newton steps on the exact trace.
#pragma once

#include "rtw_internal.h"
#include "rtw_trace.cuh"

namespace rtw {

// As add_contribution, with the phase reduced to (-pi, pi] in double precision and its sine and
// cosine taken in single precision (error below 3e-7 rad, inside the 1e-6 rad bound of the path).
__device__ __forceinline__ void add_contribution_reduced(const double* F, double psi, const double* eth,
                                                        const double* eph, double* dst)
{
    constexpr double kInv2Pi = 0.15915494309189533577, k2PiHi = 6.28318530717958623200;
    const double r = fma(-k2PiHi, rint(psi * kInv2Pi), psi);
    float sf, cf;
    sincosf((float)r, &sf, &cf);
    const double sp = sf, cp = cf;
    double tr = 0.0, ti = 0.0, pr = 0.0, pi = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double re = F[2 * c] * cp - F[2 * c + 1] * sp;
        const double im = F[2 * c] * sp + F[2 * c + 1] * cp;
        tr += re * eth[c];
        ti += im * eth[c];
        pr += re * eph[c];
        pi += im * eph[c];
    }
    atomicAdd(dst + 0, tr);
    atomicAdd(dst + 1, ti);
    atomicAdd(dst + 2, pr);
    atomicAdd(dst + 3, pi);
}

// As add_contribution_reduced onto (e_r, e_theta, e_phi): at a finite point the ray need not be
// radial, so the field has a radial part (6 doubles at dst)
__device__ __forceinline__ void add_contribution_reduced3(const double* F, double psi, const double* er,
                                                         const double* eth, const double* eph, double* dst)
{
    constexpr double kInv2Pi = 0.15915494309189533577, k2PiHi = 6.28318530717958623200;
    const double r = fma(-k2PiHi, rint(psi * kInv2Pi), psi);
    float sf, cf;
    sincosf((float)r, &sf, &cf);
    const double sp = sf, cp = cf;
    double rr = 0.0, ri = 0.0, tr = 0.0, ti = 0.0, pr = 0.0, pi = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double re = F[2 * c] * cp - F[2 * c + 1] * sp;
        const double im = F[2 * c] * sp + F[2 * c + 1] * cp;
        rr += re * er[c];
        ri += im * er[c];
        tr += re * eth[c];
        ti += im * eth[c];
        pr += re * eph[c];
        pi += im * eph[c];
    }
    atomicAdd(dst + 0, rr);
    atomicAdd(dst + 1, ri);
    atomicAdd(dst + 2, tr);
    atomicAdd(dst + 3, ti);
    atomicAdd(dst + 4, pr);
    atomicAdd(dst + 5, pi);
}

struct CaptureSink {
    int want;
    bool got;
    ExitWave w;
    __device__ void emit(int p, const ExitWave& ew)
    {
        if (p == want) {
            w = ew;
            got = true;
        }
    }
};

// Residual |t - s_p(x, y)| of the trace in precision T (double: the exact trace; float: the
// mixed-precision trace); the exit wave of order p in cs.
template <typename T = double>
__device__ __forceinline__ bool newton_eval(const ObjDev& o, int p, const double t[3], double x, double y,
                                            CaptureSink& cs, FarRecord& r, double& res)
{
    cs.want = p;
    cs.got = false;
    trace_ray<T, true>(o, x, y, p, cs);
    if (!cs.got || !far_record(o, cs.w, r)) return false;
    const double d0 = t[0] - r.s[0], d1 = t[1] - r.s[1], d2 = t[2] - r.s[2];
    res = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    return true;
}

// Newton steps on the exact double-precision trace in the impact point (x, y) until the exit
// direction of order p equals the unit target t.  The Jacobian ds/d(x, y) in the exit basis
// (e_perp, e_perp x s) is the exit wavefront-curvature matrix times the transfer matrix the trace
// carries (J = Q' T).  A step is halved (at most max_halvings times) until the new point leaves in order p
// with a smaller residual.  Converged when |s - t| < tol at one of the first max_checks
// evaluations (so at most max_checks - 1 steps) and the root lies within rmax of the seed
// (rmax <= 0: anywhere), so that the ray found is the branch the seed stands for; the root
// impact point goes to root (when given).
// T: precision of the traces (float for a cheap first approach to the root).
template <typename T = double>
__device__ __forceinline__ bool newton_point(const ObjDev& o, int p, const double t[3], double x, double y,
                                             double rmax, FarRecord& out, int max_checks = 30, double tol = 1e-11,
                                             double* root = nullptr, int max_halvings = 12)
{
    const double x0 = x, y0 = y;
    CaptureSink cs;
    FarRecord r;
    double res;
    if (!newton_eval<T>(o, p, t, x, y, cs, r, res)) return false;
    for (int it = 0; it < max_checks; ++it) {
        if (res < tol) {
            if (rmax > 0.0 && hypot(x - x0, y - y0) > rmax) return false;
            out = r;
            if (root) {
                root[0] = x;
                root[1] = y;
            }
            return true;
        }
        if (it == max_checks - 1) break;
        const ExitWave& w = cs.w;
        const double d[3] = {t[0] - r.s[0], t[1] - r.s[1], t[2] - r.s[2]};
        const double J00 = w.q11 * w.t11 + w.q12 * w.t21, J01 = w.q11 * w.t12 + w.q12 * w.t22;
        const double J10 = w.q12 * w.t11 + w.q22 * w.t21, J11 = w.q12 * w.t12 + w.q22 * w.t22;
        const double v2[3] = {w.ep[1] * w.k[2] - w.ep[2] * w.k[1], w.ep[2] * w.k[0] - w.ep[0] * w.k[2],
                              w.ep[0] * w.k[1] - w.ep[1] * w.k[0]};
        const double r0 = w.ep[0] * d[0] + w.ep[1] * d[1] + w.ep[2] * d[2];
        const double r1 = v2[0] * d[0] + v2[1] * d[1] + v2[2] * d[2];
        const double det = J00 * J11 - J01 * J10;
        if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
        const double dx = (J11 * r0 - J01 * r1) / det, dy = (J00 * r1 - J10 * r0) / det;
        double lam = 1.0;
        bool accepted = false;
        for (int h = 0; h <= max_halvings; ++h, lam *= 0.5) {
            CaptureSink cc;
            FarRecord rc;
            double resc;
            if (newton_eval<T>(o, p, t, x + lam * dx, y + lam * dy, cc, rc, resc) && resc < res) {
                x += lam * dx;
                y += lam * dy;
                cs = cc;
                r = rc;
                res = resc;
                accepted = true;
                break;
            }
        }
        if (!accepted) return false;
    }
    return false;
}

}  // namespace rtw
