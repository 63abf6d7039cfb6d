// rtw_caustic.cu -- 2-D physical optics at the 3-D caustics of a square-grid far field.
//
// The paper corrects the ray sum near caustics by a diffraction integral of the complex amplitudes
// the rays carry ("Diffraction effect correction based on VCRM") and leaves the 3-D form "under
// study".  The reading taken here: for every order p >= p_min, the directions that cell triangles of
// order p which are not consistent cover (C_p, bit 8 + p of the field's mask words) set the weight
//     s_p(u) = ramp(angle from u to the nearest direction of C_p; po_full, po_end)
// (1 up to po_full, cos^2 down to 0 at po_end), and the field of that order becomes
//     (1 - s_p) F_rays + s_p F_PO.
// F_PO of a direction u in a tile of tile_theta x tile_phi directions is Kirchhoff's integral over
// the plane through the object centre c normal to the tile's centre direction a:
//     F_PO(u) = k0 / (2 pi i) (u . a) sum_j w_j U_j dA_j e^{-i k0 u . x_j},
// every ray of order p carried to the plane as in rtw_field_po2d (x_j, U_j), weighted by the taper w_j
// of the angle between its exit direction and a (1 up to rho + cone_full, 0 from rho + cone_end, rho
// the tile's radius about a), dA_j from central differences of the crossing points; (u . a) is the
// obliquity of the plane's far field (Rayleigh-Sommerfeld).
//
// Kernels, per order: the nearest caustic columns of every direction row (a warp per row), the
// weights s_p (a thread per direction, over the rows within po_end), a bounding cone of the exit
// directions of every 16 x 16 block of the ray grid, and the tile sums (a CTA per tile with a non-zero
// weight).  A tile's CTA walks the ray blocks whose cones meet the tile's cone; its threads carry a
// block and a one-vertex halo to the plane in FP64 (plane coordinates eta = ((x - c).e1, (x - c).e2)),
// the block's rays inside the cone become terms (w U dA as single-precision complex vectors, eta
// relative to the block's first term), and every thread adds the terms into one direction:
// k0 u . (x - c) = k0 (u.e1, u.e2) . eta, the part within the block a few radians at most (one FP32
// sincos), the block's reference part in FP64, the block sums added to FP64 accumulators.
#include <cuda_runtime.h>

#include "rtw_launch.h"
#include "rtw_trace.cuh"

namespace rtw {

namespace {

constexpr double kCPi = 3.14159265358979323846;
constexpr int kRB = 16;              // ray block side
constexpr int kHalo = kRB + 2;       // with the one-vertex halo
constexpr int kTileThreads = 256;    // threads of a tile's CTA (at most one direction each)
constexpr unsigned int kMaskCausticC = 1u, kMaskPoC = 4u;

__device__ __forceinline__ double c_ramp(double x, double x0, double x1)
{
    if (x <= x0) return 1.0;
    if (x >= x1) return 0.0;
    const double c = cos(0.5 * kCPi * (x - x0) / (x1 - x0));
    return c * c;
}

__device__ __forceinline__ double c_acos(double x) { return acos(fmin(1.0, fmax(-1.0, x))); }

// nearest caustic column at or left of (nl) and at or right of (nr) every column of a row, the row
// read as a circle (phi wraps); -1 in a row without caustic directions.  A warp per row.
__global__ void caustic_rows_kernel(const unsigned int* __restrict__ words, int nt, int nph, unsigned int bit,
                                    int* __restrict__ nl, int* __restrict__ nr)
{
    const int row = blockIdx.x * (blockDim.x / 32) + (int)(threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= nt) return;
    const unsigned int* w = words + (long long)row * nph;
    int* L = nl + (long long)row * nph;
    int* R = nr + (long long)row * nph;
    int first = -1, last = -1;
    for (int j0 = 0; j0 < nph; j0 += 32) {
        const int j = j0 + lane;
        const unsigned int b = __ballot_sync(0xffffffffu, j < nph && (w[j] & bit));
        if (b) {
            if (first < 0) first = j0 + __ffs(b) - 1;
            last = j0 + 31 - __clz(b);
        }
    }
    if (last < 0) {
        for (int j = lane; j < nph; j += 32) L[j] = R[j] = -1;
        return;
    }
    int carry = last;  // left of the first caustic column the nearest one wraps to the row's last
    for (int j0 = 0; j0 < nph; j0 += 32) {
        const int j = j0 + lane;
        const unsigned int b = __ballot_sync(0xffffffffu, j < nph && (w[j] & bit));
        const unsigned int upto = b & (0xffffffffu >> (31 - lane));
        if (j < nph) L[j] = upto ? j0 + 31 - __clz(upto) : carry;
        if (b) carry = j0 + 31 - __clz(b);
    }
    carry = first;
    for (int j0 = ((nph - 1) / 32) * 32; j0 >= 0; j0 -= 32) {
        const int j = j0 + lane;
        const unsigned int b = __ballot_sync(0xffffffffu, j < nph && (w[j] & bit));
        const unsigned int from = b & (0xffffffffu << lane);
        if (j < nph) R[j] = from ? j0 + __ffs(from) - 1 : carry;
        if (b) carry = j0 + __ffs(b) - 1;
    }
}

// s_p of every direction: the angle to the nearest caustic direction among the rows within po_end
// (a caustic direction in a farther row is farther than po_end); marks the tiles with a weight
__global__ void caustic_weight_kernel(const int* __restrict__ nl, const int* __restrict__ nr, int nt, int nph,
                                      double po_full, double po_end, int tt, int tp, int ntp, double* __restrict__ sw,
                                      unsigned char* __restrict__ tile_on)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)nt * nph) return;
    const int it = (int)(k / nph), jp = (int)(k % nph);
    const double dth = kCPi / nt, dph = 2.0 * kCPi / nph;
    double st, ct;
    sincos((it + 0.5) * dth, &st, &ct);
    const double th = (it + 0.5) * dth;
    int r0 = (int)ceil((th - po_end) / dth - 0.5), r1 = (int)floor((th + po_end) / dth - 0.5);
    r0 = r0 < 0 ? 0 : r0;
    r1 = r1 > nt - 1 ? nt - 1 : r1;
    double best = -2.0;
    for (int r = r0; r <= r1; ++r) {
        const int cl = nl[(long long)r * nph + jp];
        if (cl < 0) continue;
        const int cr = nr[(long long)r * nph + jp];
        double sr, cr_;
        sincos((r + 0.5) * dth, &sr, &cr_);
        best = fmax(best, ct * cr_ + st * sr * cos((cl - jp) * dph));
        best = fmax(best, ct * cr_ + st * sr * cos((cr - jp) * dph));
    }
    const double d = best < -1.5 ? 2.0 * kCPi : c_acos(best);
    const double s = d < po_end ? c_ramp(d, po_full, po_end) : 0.0;
    sw[k] = s;
    if (s > 0.0) tile_on[(it / tt) * ntp + jp / tp] = 1;
}

// bounding cone of the exit directions of one 16 x 16 ray block (mean direction, radius; w = 4
// for a block without a valid ray)
__global__ void __launch_bounds__(kRB* kRB) ray_block_cone_kernel(RaysDev st, int order, long long ray0,
                                                                  long long nx, long long ny, int nbx,
                                                                  float4* __restrict__ cone)
{
    __shared__ double red[kRB * kRB / 32][4];
    const int bx = blockIdx.x % nbx, by = blockIdx.x / nbx;
    const long long ix = (long long)bx * kRB + threadIdx.x % kRB, iy = (long long)by * kRB + threadIdx.x / kRB;
    double s[3] = {0.0, 0.0, 0.0};
    double cnt = 0.0;
    if (ix < nx && iy < ny) {
        const long long i = (long long)order * st.R + ray0 + iy * nx + ix;
        if (st.flags[i] & kFlagValid) {
            const double2 a = st.s01[i];
            s[0] = a.x;
            s[1] = a.y;
            s[2] = st.s2psi[i].x;
            cnt = 1.0;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double v[4] = {s[0], s[1], s[2], cnt};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], off);
        if (lane == 0) red[wid][c] = v[c];
    }
    __syncthreads();
    double m[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 4; ++c)
        for (int w = 0; w < kRB * kRB / 32; ++w) m[c] += red[w][c];
    const double mn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    double ang = 0.0;
    if (m[3] > 0.0 && mn > 0.0 && cnt > 0.0) ang = c_acos((s[0] * m[0] + s[1] * m[1] + s[2] * m[2]) / mn);
    if (!(m[3] > 0.0 && mn > 0.0)) ang = 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ang = fmax(ang, __shfl_down_sync(0xffffffffu, ang, off));
    __syncthreads();
    if (lane == 0) red[wid][0] = ang;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < kRB * kRB / 32; ++w) r = fmax(r, red[w][0]);
        if (!(m[3] > 0.0 && mn > 0.0))
            cone[blockIdx.x] = make_float4(0.0f, 0.0f, 1.0f, 4.0f);
        else
            cone[blockIdx.x] = make_float4((float)(m[0] / mn), (float)(m[1] / mn), (float)(m[2] / mn), (float)r);
    }
}

struct TileArgs {
    RaysDev st;
    int order, np;
    long long ray0, nx, ny;
    int nbx, nby;
    const float4* cone;
    double c[3];
    double k0;
    int nt, nph, tt, tp, ntp;
    double cone_full, cone_end;
    const double* sw;
    const unsigned char* tile_on;
    double* field;         // [directions][np][4], per order
    unsigned int* words;   // mask words
    unsigned int bit;      // caustic bit of the order
    double* weights;       // [directions][np] or null
};

// position of this thread's flag among the set flags of the CTA, in thread order; *total receives
// their number (all threads of the CTA take part)
__device__ __forceinline__ int cta_rank(bool flag, int* warp_cnt, int* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned int b = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) warp_cnt[wid] = __popc(b);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        before += w < wid ? warp_cnt[w] : 0;
        all += warp_cnt[w];
    }
    *total = all;
    return before + __popc(b & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(kTileThreads) caustic_tile_kernel(TileArgs A)
{
    __shared__ float4 tq0[kTileThreads], tq1[kTileThreads];  // terms: (c0, c1), (c2, d eta)
    __shared__ double2 eta[kHalo * kHalo];
    __shared__ double tauv[kHalo * kHalo];
    __shared__ unsigned char okv[kHalo * kHalo];
    __shared__ int blist[kTileThreads];
    __shared__ int warp_cnt[kTileThreads / 32];
    __shared__ double rred[kTileThreads / 32];
    __shared__ double2 eta_ref;
    const int tile = blockIdx.x;
    if (!A.tile_on[tile]) return;
    const int t = threadIdx.x;
    const int bt = tile / A.ntp, bp = tile % A.ntp;
    const int r0 = bt * A.tt, r1 = min(r0 + A.tt, A.nt);
    const int c0 = bp * A.tp, c1 = min(c0 + A.tp, A.nph);
    const int tw = c1 - c0, ndt = (r1 - r0) * tw;
    const double dth = kCPi / A.nt, dph = 2.0 * kCPi / A.nph;
    double sa_, ca_, sp_, cp_;
    sincos(0.5 * (r0 + r1) * dth, &sa_, &ca_);
    sincos(-kCPi + 0.5 * (c0 + c1) * dph, &sp_, &cp_);
    const double a[3] = {sa_ * cp_, sa_ * sp_, ca_};
    const double e1[3] = {ca_ * cp_, ca_ * sp_, -sa_}, e2[3] = {-sp_, cp_, 0.0};
    // this thread's direction
    const bool mine = t < ndt;
    const int it = r0 + (mine ? t / tw : 0), jp = c0 + (mine ? t % tw : 0);
    double st, ct, sp, cp;
    sincos((it + 0.5) * dth, &st, &ct);
    sincos(-kCPi + (jp + 0.5) * dph, &sp, &cp);
    const double u[3] = {st * cp, st * sp, ct};
    // rho: the largest angle from a to a direction of the tile
    double ang = mine ? c_acos(u[0] * a[0] + u[1] * a[1] + u[2] * a[2]) : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ang = fmax(ang, __shfl_down_sync(0xffffffffu, ang, off));
    if ((t & 31) == 0) rred[t >> 5] = ang;
    __syncthreads();
    double rho = 0.0;
    for (int w = 0; w < kTileThreads / 32; ++w) rho = fmax(rho, rred[w]);
    const double cf = rho + A.cone_full, ce = rho + A.cone_end;
    const double b1 = u[0] * e1[0] + u[1] * e1[1] + u[2] * e1[2], b2 = u[0] * e2[0] + u[1] * e2[1] + u[2] * e2[2];
    const float kb1 = (float)(A.k0 * b1), kb2 = (float)(A.k0 * b2);
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const long long n = (long long)A.st.np * A.st.R;
    const long long base = (long long)A.order * A.st.R + A.ray0;
    const int nblocks = A.nbx * A.nby;
    const float fce = (float)ce;
    for (int b0 = 0; b0 < nblocks; b0 += kTileThreads) {
        // the ray blocks of this batch whose cones meet the tile's cone
        bool meet = false;
        if (b0 + t < nblocks) {
            const float4 cb = A.cone[b0 + t];
            if (cb.w < 3.0f) {
                const float d = acosf(fminf(1.0f, fmaxf(-1.0f, (float)a[0] * cb.x + (float)a[1] * cb.y +
                                                                   (float)a[2] * cb.z)));
                meet = d <= fce + cb.w + 1e-4f;
            }
        }
        int nmeet = 0;
        const int pos = cta_rank(meet, warp_cnt, &nmeet);
        if (meet) blist[pos] = b0 + t;
        __syncthreads();
        for (int m = 0; m < nmeet; ++m) {
            const int rb = blist[m];
            const long long bx = rb % A.nbx, by = rb / A.nbx;
            const long long hx0 = bx * kRB - 1, hy0 = by * kRB - 1;
            // every vertex of the block and its halo carried to the plane
            for (int v = t; v < kHalo * kHalo; v += kTileThreads) {
                const long long ix = hx0 + v % kHalo, iy = hy0 + v / kHalo;
                unsigned char ok = 0;
                double2 e = make_double2(0.0, 0.0);
                double tau = 0.0;
                if (ix >= 0 && iy >= 0 && ix < A.nx && iy < A.ny) {
                    const long long i = base + iy * A.nx + ix;
                    if (A.st.flags[i] & kFlagValid) {
                        const double2 s01 = A.st.s01[i];
                        const double s[3] = {s01.x, s01.y, A.st.s2psi[i].x};
                        const double sa = a[0] * s[0] + a[1] * s[1] + a[2] * s[2];
                        if (fabs(sa) > 1e-6) {
                            const double* aux = A.st.aux + i;
                            const double r[3] = {aux[kAuxRx * n], aux[kAuxRy * n], aux[kAuxRz * n]};
                            tau = (a[0] * (A.c[0] - r[0]) + a[1] * (A.c[1] - r[1]) + a[2] * (A.c[2] - r[2])) / sa;
                            const double d[3] = {r[0] + tau * s[0] - A.c[0], r[1] + tau * s[1] - A.c[1],
                                                 r[2] + tau * s[2] - A.c[2]};
                            e = make_double2(d[0] * e1[0] + d[1] * e1[1] + d[2] * e1[2],
                                             d[0] * e2[0] + d[1] * e2[1] + d[2] * e2[2]);
                            ok = 1;
                        }
                    }
                }
                okv[v] = ok;
                eta[v] = e;
                tauv[v] = tau;
            }
            __syncthreads();
            // the block's rays in the cone become terms
            bool term = false;
            float4 q0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), q1 = q0;
            double2 my_eta = make_double2(0.0, 0.0);
            {
                const int lx = t % kRB, ly = t / kRB;
                const int v = (ly + 1) * kHalo + lx + 1;
                if (okv[v]) {
                    const long long i = base + (by * kRB + ly) * A.nx + bx * kRB + lx;
                    const double2 s01 = A.st.s01[i];
                    const double sa = a[0] * s01.x + a[1] * s01.y + a[2] * A.st.s2psi[i].x;
                    const double w = c_ramp(c_acos(sa), cf, ce);
                    const int vxm = okv[v - 1] ? v - 1 : v, vxp = okv[v + 1] ? v + 1 : v;
                    const int vym = okv[v - kHalo] ? v - kHalo : v, vyp = okv[v + kHalo] ? v + kHalo : v;
                    if (w > 0.0 && vxm != vxp && vym != vyp) {
                        const double fx = 1.0 / (double)(vxp - vxm), fy = 1.0 / (double)((vyp - vym) / kHalo);
                        const double exa = (eta[vxp].x - eta[vxm].x) * fx, exb = (eta[vxp].y - eta[vxm].y) * fx;
                        const double eya = (eta[vyp].x - eta[vym].x) * fy, eyb = (eta[vyp].y - eta[vym].y) * fy;
                        const double area = fabs(exa * eyb - exb * eya);
                        const double* aux = A.st.aux + i;
                        const double tau = tauv[v];
                        const double a11 = 1.0 + tau * aux[kAuxQ11 * n], a12 = tau * aux[kAuxQ12 * n],
                                     a22 = 1.0 + tau * aux[kAuxQ22 * n];
                        const double det = a11 * a22 - a12 * a12;
                        if (det != 0.0) {
                            const int nfl = neg_eigs_sym(a11, a12, a22);
                            const int nf = (int)aux[kAuxNfLegs * n] + (tau > 0.0 ? nfl : -nfl);
                            const double mag = sqrt(aux[kAuxDlegs * n] / fabs(det)) * w * area;
                            // e^{i k0 (L + tau)} from the phase reduced to [-pi, pi] in FP64
                            const double ph = A.k0 * (aux[kAuxPath * n] + tau);
                            const double red = ph - 2.0 * kCPi * rint(ph * (0.5 / kCPi));
                            float sn, cs;
                            __sincosf((float)red, &sn, &cs);
                            double pr = cs, pi = sn;
                            switch (nf & 3) {  // (-i)^nf
                            case 1: pr = sn; pi = -cs; break;
                            case 2: pr = -cs; pi = -sn; break;
                            case 3: pr = -sn; pi = cs; break;
                            default: break;
                            }
                            pr *= mag;
                            pi *= mag;
                            const double er0 = aux[kAuxExr * n], ei0 = aux[kAuxExi * n];
                            const double er1 = aux[kAuxEyr * n], ei1 = aux[kAuxEyi * n];
                            const double er2 = aux[kAuxEzr * n], ei2 = aux[kAuxEzi * n];
                            q0 = make_float4((float)(er0 * pr - ei0 * pi), (float)(er0 * pi + ei0 * pr),
                                             (float)(er1 * pr - ei1 * pi), (float)(er1 * pi + ei1 * pr));
                            q1 = make_float4((float)(er2 * pr - ei2 * pi), (float)(er2 * pi + ei2 * pr), 0.0f, 0.0f);
                            my_eta = eta[v];
                            term = true;
                        }
                    }
                }
            }
            int nterm = 0;
            const int tp_ = cta_rank(term, warp_cnt, &nterm);
            if (term && tp_ == 0) eta_ref = my_eta;
            __syncthreads();
            if (term) {
                q1.z = (float)(my_eta.x - eta_ref.x);
                q1.w = (float)(my_eta.y - eta_ref.y);
                tq0[tp_] = q0;
                tq1[tp_] = q1;
            }
            __syncthreads();
            if (mine && nterm > 0) {
                float f[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                for (int m2 = 0; m2 < nterm; ++m2) {
                    const float4 p0 = tq0[m2], p1 = tq1[m2];
                    float ph = -(kb1 * p1.z + kb2 * p1.w);
                    ph = fmaf(-6.28318548f, rintf(ph * 0.159154943f), ph);
                    float sn, cs;
                    __sincosf(ph, &sn, &cs);
                    f[0] += p0.x * cs - p0.y * sn;
                    f[1] += p0.x * sn + p0.y * cs;
                    f[2] += p0.z * cs - p0.w * sn;
                    f[3] += p0.z * sn + p0.w * cs;
                    f[4] += p1.x * cs - p1.y * sn;
                    f[5] += p1.x * sn + p1.y * cs;
                }
                // the block's reference: e^{-i k0 (b1 eta_ref.x + b2 eta_ref.y)}
                const double ph = -A.k0 * (b1 * eta_ref.x + b2 * eta_ref.y);
                const double red = ph - 2.0 * kCPi * rint(ph * (0.5 / kCPi));
                float sn, cs;
                __sincosf((float)red, &sn, &cs);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    acc[2 * c] += (double)f[2 * c] * cs - (double)f[2 * c + 1] * sn;
                    acc[2 * c + 1] += (double)f[2 * c] * sn + (double)f[2 * c + 1] * cs;
                }
            }
            __syncthreads();
        }
    }
    if (!mine) return;
    const long long k = (long long)it * A.nph + jp;
    const double s = A.sw[k];
    if (!(s > 0.0)) return;
    // F = k0 / (2 pi i) (u . a) e^{-i k0 u . c} acc, projected on e_theta, e_phi
    double sn, cs;
    sincos(-A.k0 * (u[0] * A.c[0] + u[1] * A.c[1] + u[2] * A.c[2]), &sn, &cs);
    const double eth[3] = {ct * cp, ct * sp, -st}, eph[3] = {-sp, cp, 0.0};
    double tr = 0.0, ti = 0.0, fr = 0.0, fi = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double vr = acc[2 * c] * cs - acc[2 * c + 1] * sn, vi = acc[2 * c] * sn + acc[2 * c + 1] * cs;
        tr += vr * eth[c];
        ti += vi * eth[c];
        fr += vr * eph[c];
        fi += vi * eph[c];
    }
    const double f = A.k0 / (2.0 * kCPi) * (u[0] * a[0] + u[1] * a[1] + u[2] * a[2]);  // -i f (re + i im)
    double* o = A.field + ((size_t)k * A.np + A.order) * 4;
    o[0] = (1.0 - s) * o[0] + s * (f * ti);
    o[1] = (1.0 - s) * o[1] + s * (-f * tr);
    o[2] = (1.0 - s) * o[2] + s * (f * fi);
    o[3] = (1.0 - s) * o[3] + s * (-f * fr);
    unsigned int wv = A.words[k] | kMaskPoC;
    if (s == 1.0) wv &= ~A.bit;
    A.words[k] = wv;
    if (A.weights) A.weights[(size_t)k * A.np + A.order] = s;
}

// bit 0 of the mask words again from the order bits that are left
__global__ void caustic_fix_mask_kernel(unsigned int* __restrict__ words, long long ndir)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= ndir) return;
    const unsigned int w = words[k];
    words[k] = (w & ~kMaskCausticC) | ((w >> 8) ? kMaskCausticC : 0u);
}

__global__ void sum_orders_kernel(const double* __restrict__ per, double* __restrict__ out, long long ndir, int np)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ndir * 4) return;
    const long long k = t >> 2;
    const int c = (int)(t & 3);
    double v = 0.0;
    for (int p = 0; p < np; ++p) v += per[((size_t)k * np + p) * 4 + c];
    out[t] = v;
}

}  // namespace

size_t caustic_scratch_bytes(long long ndir, long long ntiles, long long nblocks)
{
    // nl, nr (int), s (double) per direction; a flag per tile; a cone per ray block
    return (size_t)ndir * (4 + 4 + 8) + (size_t)((ntiles + 255) / 256 * 256) + (size_t)nblocks * 16 + 1024;
}

cudaError_t launch_caustic_order(const RaysDev& st, const ObjDev& o, int order, int nt, int nph, int tt, int tp,
                                 double po_full, double po_end, double cone_full, double cone_end, unsigned int* words,
                                 double* field, double* weights, void* scratch, cudaStream_t s)
{
    const long long ndir = (long long)nt * nph;
    const int ntt = (nt + tt - 1) / tt, ntp = (nph + tp - 1) / tp;
    const long long ntiles = (long long)ntt * ntp;
    const int nbx = (int)((o.nx + kRB - 1) / kRB), nby = (int)((o.ny + kRB - 1) / kRB);
    const long long nblocks = (long long)nbx * nby;
    char* b = (char*)scratch;
    double* sw = (double*)b;
    int* nl = (int*)(sw + ndir);
    int* nr = nl + ndir;
    unsigned char* tile_on = (unsigned char*)(nr + ndir);
    float4* cone = (float4*)(tile_on + (ntiles + 255) / 256 * 256);
    const unsigned int bit = 0x100u << order;
    cudaError_t e = cudaMemsetAsync(tile_on, 0, (size_t)ntiles, s);
    if (e != cudaSuccess) return e;
    caustic_rows_kernel<<<(nt + 7) / 8, 256, 0, s>>>(words, nt, nph, bit, nl, nr);
    caustic_weight_kernel<<<(unsigned)((ndir + 255) / 256), 256, 0, s>>>(nl, nr, nt, nph, po_full, po_end, tt, tp, ntp,
                                                                         sw, tile_on);
    ray_block_cone_kernel<<<(unsigned)nblocks, kRB * kRB, 0, s>>>(st, order, o.ray_offset, o.nx, o.ny, nbx, cone);
    TileArgs A;
    A.st = st;
    A.order = order;
    A.np = st.np;
    A.ray0 = o.ray_offset;
    A.nx = o.nx;
    A.ny = o.ny;
    A.nbx = nbx;
    A.nby = nby;
    A.cone = cone;
    A.c[0] = o.c[0];
    A.c[1] = o.c[1];
    A.c[2] = o.c[2];
    A.k0 = o.k0;
    A.nt = nt;
    A.nph = nph;
    A.tt = tt;
    A.tp = tp;
    A.ntp = ntp;
    A.cone_full = cone_full;
    A.cone_end = cone_end;
    A.sw = sw;
    A.tile_on = tile_on;
    A.field = field;
    A.words = words;
    A.bit = bit;
    A.weights = weights;
    caustic_tile_kernel<<<(unsigned)ntiles, kTileThreads, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_caustic_finish(unsigned int* words, long long ndir, const double* per_order, double* out, int np,
                                  cudaStream_t s)
{
    caustic_fix_mask_kernel<<<(unsigned)((ndir + 255) / 256), 256, 0, s>>>(words, ndir);
    if (out) sum_orders_kernel<<<(unsigned)((4 * ndir + 255) / 256), 256, 0, s>>>(per_order, out, ndir, np);
    return cudaGetLastError();
}

}  // namespace rtw
