// rtw_po2d.cu -- 2-D physical optics over an aperture of rays (the "Diffraction effect correction
// based on VCRM": near a caustic the ray sum is replaced by a diffraction integral of the complex
// amplitudes the rays carry; here Kirchhoff's integral over a plane, both directions numerical).
//
// The rays of a window of grid vertices carry their exit waves, kept by the trace with
// RTW_TRACE_APERTURE, to the plane through the object centre with normal a:
//     tau = a.(c - r) / a.s,  x = r + tau s,
//     U = E' sqrt(D_legs / |det(I + tau Q')|) (-i)^{N_f} e^{i k0 (L + tau)}
// (Eqs. IntVCRM, DivFactVCRM, PhasePath; the focal lines of the last stretch are counted forward
// for tau > 0 and undone backward).  The plane's area per grid cell at a ray comes from central
// differences of the neighbours' crossing points, and rays are weighted by the angle g of their exit
// direction to a: 1 up to cone_full, cos^2 down to 0 at cone_end.  Then
//     F(s) = k0 / (2 pi i) sum_j w_j U_j dA_j e^{-i k0 s.x_j}
// projected on (e_theta, e_phi).  The sum is a dense (direction x ray) contraction of complex
// exponentials: it runs on the FP64 pipe with one sincos per term, directions in tiles of
// kPoDirTile so that each ray is loaded once per tile, rays in slices across blocks.
#include <cuda_runtime.h>

#include "rtw_launch.h"
#include "rtw_trace.cuh"

namespace rtw {

namespace {

constexpr int kPoBlock = 256;
constexpr int kPoDirTile = 4;
constexpr double kPoPi = 3.14159265358979323846;

__device__ __forceinline__ double po_ramp(double x, double x0, double x1)
{
    if (x <= x0) return 1.0;
    if (x >= x1) return 0.0;
    const double c = cos(0.5 * kPoPi * (x - x0) / (x1 - x0));
    return c * c;
}

// one ray of the window: its crossing point, field U (3 complex) and weight; ok = the order leaves
__global__ void po2d_aperture_kernel(RaysDev st, int order, long long nx, long long ix0, long long iy0, int wx,
                                     int wy, double cx, double cy, double cz, double ax, double ay, double az,
                                     double k0, double cone_full, double cone_end, double* __restrict__ xa,
                                     double* __restrict__ U, double* __restrict__ wgt, unsigned char* __restrict__ ok)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)wx * wy) return;
    const long long jx = q % wx, jy = q / wx;
    const long long j = (iy0 + jy) * nx + (ix0 + jx);
    const long long i = (long long)order * st.R + j;
    ok[q] = 0;
    wgt[q] = 0.0;
    if (!(st.flags[i] & kFlagValid)) return;
    const long long n = (long long)st.np * st.R;
    const double* aux = st.aux + i;
    const double2 s01 = st.s01[i], s2 = st.s2psi[i];
    const double sx = s01.x, sy = s01.y, sz = s2.x;
    const double rx = aux[kAuxRx * n], ry = aux[kAuxRy * n], rz = aux[kAuxRz * n];
    const double sa = ax * sx + ay * sy + az * sz;
    if (!(fabs(sa) > 1e-6)) return;
    const double tau = (ax * (cx - rx) + ay * (cy - ry) + az * (cz - rz)) / sa;
    xa[3 * q] = rx + tau * sx;
    xa[3 * q + 1] = ry + tau * sy;
    xa[3 * q + 2] = rz + tau * sz;
    const double a11 = 1.0 + tau * aux[kAuxQ11 * n], a12 = tau * aux[kAuxQ12 * n], a22 = 1.0 + tau * aux[kAuxQ22 * n];
    const double det = a11 * a22 - a12 * a12;
    if (det == 0.0) return;
    const int nfl = neg_eigs_sym(a11, a12, a22);
    const int nf = (int)aux[kAuxNfLegs * n] + (tau > 0.0 ? nfl : -nfl);
    const double mag = sqrt(aux[kAuxDlegs * n] / fabs(det));
    double sn, cs;
    sincos(k0 * (aux[kAuxPath * n] + tau), &sn, &cs);
    // (-i)^nf e^{i phase}
    double pr = cs, pi = sn;
    switch (nf & 3) {
    case 1: pr = sn; pi = -cs; break;
    case 2: pr = -cs; pi = -sn; break;
    case 3: pr = -sn; pi = cs; break;
    default: break;
    }
    pr *= mag;
    pi *= mag;
    const double er[3] = {aux[kAuxExr * n], aux[kAuxEyr * n], aux[kAuxEzr * n]};
    const double ei[3] = {aux[kAuxExi * n], aux[kAuxEyi * n], aux[kAuxEzi * n]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        U[6 * q + 2 * c] = er[c] * pr - ei[c] * pi;
        U[6 * q + 2 * c + 1] = er[c] * pi + ei[c] * pr;
    }
    const double ca = fmin(1.0, fmax(-1.0, sa));
    wgt[q] = po_ramp(acos(ca), cone_full, cone_end);
    ok[q] = 1;
}

// area of the plane per grid cell at each ray (central differences, one-sided at the window edge and
// next to rays that do not leave), times the weight; rays of non-zero weight are appended to the
// compact list (x, W) that the sum walks
__global__ void po2d_area_kernel(int wx, int wy, double ax, double ay, double az, const double* __restrict__ xa,
                                 const double* __restrict__ U, const double* __restrict__ wgt,
                                 const unsigned char* __restrict__ ok, double* __restrict__ cx,
                                 double* __restrict__ cw, unsigned int* __restrict__ count)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)wx * wy) return;
    if (!ok[q] || wgt[q] == 0.0) return;
    const int jx = (int)(q % wx), jy = (int)(q / wx);
    const long long qxm = jx > 0 && ok[q - 1] ? q - 1 : q, qxp = jx + 1 < wx && ok[q + 1] ? q + 1 : q;
    const long long qym = jy > 0 && ok[q - wx] ? q - wx : q, qyp = jy + 1 < wy && ok[q + wx] ? q + wx : q;
    if (qxm == qxp || qym == qyp) return;
    const double fx = 1.0 / (double)(qxp - qxm), fy = 1.0 / (double)((qyp - qym) / wx);
    double ex[3], ey[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ex[c] = (xa[3 * qxp + c] - xa[3 * qxm + c]) * fx;
        ey[c] = (xa[3 * qyp + c] - xa[3 * qym + c]) * fy;
    }
    const double crx = ex[1] * ey[2] - ex[2] * ey[1], cry = ex[2] * ey[0] - ex[0] * ey[2],
                 crz = ex[0] * ey[1] - ex[1] * ey[0];
    const double w = wgt[q] * fabs(crx * ax + cry * ay + crz * az);
    const unsigned int k = atomicAdd(count, 1u);
#pragma unroll
    for (int c = 0; c < 3; ++c) cx[3 * (long long)k + c] = xa[3 * q + c];
#pragma unroll
    for (int c = 0; c < 6; ++c) cw[6 * (long long)k + c] = w * U[6 * q + c];
}

// partial sums of a tile of kPoDirTile directions over one slice of the compact list; the block's
// sums are added to acc (6 doubles per direction: the vector sum, re and im)
__global__ void __launch_bounds__(kPoBlock) po2d_sum_kernel(const double* __restrict__ dirs, long long ndir,
                                                            double k0, const double* __restrict__ cx,
                                                            const double* __restrict__ cw,
                                                            const unsigned int* __restrict__ count, double* acc)
{
    __shared__ double red[kPoBlock / 32][kPoDirTile * 6];
    const long long d0 = (long long)blockIdx.x * kPoDirTile;
    double sv[kPoDirTile][3];
#pragma unroll
    for (int t = 0; t < kPoDirTile; ++t) {
        const long long d = d0 + t < ndir ? d0 + t : ndir - 1;
        double st_, ct, sp, cp;
        sincos(dirs[2 * d], &st_, &ct);
        sincos(dirs[2 * d + 1], &sp, &cp);
        sv[t][0] = -k0 * st_ * cp;
        sv[t][1] = -k0 * st_ * sp;
        sv[t][2] = -k0 * ct;
    }
    double sum[kPoDirTile][6];
#pragma unroll
    for (int t = 0; t < kPoDirTile; ++t)
#pragma unroll
        for (int c = 0; c < 6; ++c) sum[t][c] = 0.0;
    const long long n = *count;
    const long long per = (n + gridDim.y - 1) / gridDim.y;
    const long long lo = (long long)blockIdx.y * per, hi = lo + per < n ? lo + per : n;
    for (long long k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const double x0 = cx[3 * k], x1 = cx[3 * k + 1], x2 = cx[3 * k + 2];
        double w[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) w[c] = cw[6 * k + c];
#pragma unroll
        for (int t = 0; t < kPoDirTile; ++t) {
            double sn, cs;
            sincos(sv[t][0] * x0 + sv[t][1] * x1 + sv[t][2] * x2, &sn, &cs);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sum[t][2 * c] += w[2 * c] * cs - w[2 * c + 1] * sn;
                sum[t][2 * c + 1] += w[2 * c] * sn + w[2 * c + 1] * cs;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < kPoDirTile; ++t)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double v = sum[t][c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp][t * 6 + c] = v;
        }
    __syncthreads();
    if (threadIdx.x < kPoDirTile * 6) {
        const int t = threadIdx.x / 6;
        double v = 0.0;
        for (int wv = 0; wv < kPoBlock / 32; ++wv) v += red[wv][threadIdx.x];
        if (d0 + t < ndir) atomicAdd(acc + 6 * (d0 + t) + (threadIdx.x % 6), v);
    }
}

// F = k0 / (2 pi i) times the vector sum, projected on e_theta, e_phi
__global__ void po2d_finish_kernel(const double* __restrict__ dirs, long long ndir, double k0,
                                   const double* __restrict__ acc, double2* __restrict__ out)
{
    const long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (d >= ndir) return;
    double st_, ct, sp, cp;
    sincos(dirs[2 * d], &st_, &ct);
    sincos(dirs[2 * d + 1], &sp, &cp);
    const double et[3] = {ct * cp, ct * sp, -st_}, ep[3] = {-sp, cp, 0.0};
    double tr = 0.0, ti = 0.0, fr = 0.0, fi = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        tr += acc[6 * d + 2 * c] * et[c];
        ti += acc[6 * d + 2 * c + 1] * et[c];
        fr += acc[6 * d + 2 * c] * ep[c];
        fi += acc[6 * d + 2 * c + 1] * ep[c];
    }
    const double f = k0 / (2.0 * kPoPi);  // -i f (re + i im) = f (im - i re)
    out[2 * d] = make_double2(f * ti, -f * tr);
    out[2 * d + 1] = make_double2(f * fi, -f * fr);
}

}  // namespace

size_t po2d_scratch_bytes(long long nwin, long long ndir)
{
    // xa 3, U 6, wgt 1 doubles and ok 1 byte per window ray; compact x 3, W 6 doubles per ray;
    // 6 accumulators per direction; the count
    const size_t a = (size_t)nwin * (3 + 6 + 1 + 3 + 6) * sizeof(double);
    const size_t b = ((size_t)nwin + 255) / 256 * 256;
    return a + b + (size_t)ndir * 6 * sizeof(double) + 256;
}

cudaError_t launch_po2d(const RaysDev& st, int order, long long nx, const long long win[4], const double c[3],
                        const double axis[3], double k0, double cone_full, double cone_end, const double* dirs,
                        long long ndir, double2* out, void* scratch, cudaStream_t s)
{
    const int wx = (int)(win[1] - win[0] + 1), wy = (int)(win[3] - win[2] + 1);
    const long long nwin = (long long)wx * wy;
    char* b = (char*)scratch;
    double* xa = (double*)b;
    double* U = xa + 3 * nwin;
    double* wgt = U + 6 * nwin;
    double* cxp = wgt + nwin;
    double* cw = cxp + 3 * nwin;
    double* acc = cw + 6 * nwin;
    unsigned char* ok = (unsigned char*)(acc + 6 * ndir);
    // the count occupies the last 256 bytes of the block (the host reads it there)
    unsigned int* count = (unsigned int*)((char*)scratch + po2d_scratch_bytes(nwin, ndir) - 256);
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 6 * (size_t)ndir, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const unsigned gw = (unsigned)((nwin + kPoBlock - 1) / kPoBlock);
    po2d_aperture_kernel<<<gw, kPoBlock, 0, s>>>(st, order, nx, win[0], win[2], wx, wy, c[0], c[1], c[2], axis[0],
                                                 axis[1], axis[2], k0, cone_full, cone_end, xa, U, wgt, ok);
    po2d_area_kernel<<<gw, kPoBlock, 0, s>>>(wx, wy, axis[0], axis[1], axis[2], xa, U, wgt, ok, cxp, cw, count);
    // direction tiles x ray slices: about four blocks per SM in all
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (ndir + kPoDirTile - 1) / kPoDirTile;
    long long slices = (4LL * sms + tiles - 1) / tiles;
    slices = slices < 1 ? 1 : (slices > 1024 ? 1024 : slices);
    slices = slices > (nwin + kPoBlock - 1) / kPoBlock ? (nwin + kPoBlock - 1) / kPoBlock : slices;
    if (slices < 1) slices = 1;
    po2d_sum_kernel<<<dim3((unsigned)tiles, (unsigned)slices), kPoBlock, 0, s>>>(dirs, ndir, k0, cxp, cw, count, acc);
    po2d_finish_kernel<<<(unsigned)((ndir + 255) / 256), 256, 0, s>>>(dirs, ndir, k0, acc, out);
    return cudaGetLastError();
}

}  // namespace rtw
