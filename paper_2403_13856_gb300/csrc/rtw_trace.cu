// rtw_trace.cu -- trace kernels: one thread per incident ray, structure-of-arrays ray state.
#include <algorithm>

#include "rtw_launch.h"
#include "rtw_trace.cuh"

namespace rtw {

namespace {

// Stores the far-field record (kNear: the record at the sphere |M| = st.near_r) of every emitted
// order into the SoA ray state (16-byte vectors).
template <bool kNear>
struct StateSink {
    const ObjDev* o;
    RaysDev st;
    long long j;
    bool aux;
    unsigned int emitted;
    float f2max;  // largest |F|^2 of the ray's valid records that are not near-caustic

    __device__ void emit(int p, const ExitWave& w)
    {
        FarRecord fr;
        if constexpr (kNear) {
            if (!near_record(*o, w, st.near_r, fr)) return;
        } else {
            if (!far_record(*o, w, fr)) return;
        }
        const long long i = (long long)p * st.R + j;
        st.s01[i] = make_double2(fr.s[0], fr.s[1]);
        st.s2psi[i] = make_double2(fr.s[2], fr.psi);
        st.Fx[i] = make_double2(fr.F[0], fr.F[1]);
        st.Fy[i] = make_double2(fr.F[2], fr.F[3]);
        st.Fz[i] = make_double2(fr.F[4], fr.F[5]);
        st.flags[i] = fr.flags;
        if (st.frec) {
            // the field record, narrowed in the integer pipe (one double subtraction per low part)
            float Ff[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) Ff[c] = f64_to_f32_int(fr.F[c]);
            float sh[3], sl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sh[c] = f64_to_f32_int(fr.s[c]);
                sl[c] = f64_to_f32_int(fr.s[c] - f32_to_f64_int(sh[c]));
            }
            const float ph = f64_to_f32_int(fr.psi);
            const float pl = f64_to_f32_int(fr.psi - f32_to_f64_int(ph));
            const float th = atan2f(sqrtf(sh[0] * sh[0] + sh[1] * sh[1]), sh[2]), az = atan2f(sh[1], sh[0]);
            st.frec[2 * i] = make_float4(th, az, sh[0], sh[1]);
            st.frec[2 * i + 1] = make_float4(sh[2], sl[0], sl[1], sl[2]);
            st.fval[2 * i] = make_float4(ph, pl, Ff[0], Ff[1]);
            st.fval[2 * i + 1] = make_float4(Ff[2], Ff[3], Ff[4], Ff[5]);
            if (st.fmax && !(fr.flags & kFlagCaustic)) {
                float f2 = 0.0f;
#pragma unroll
                for (int c = 0; c < 6; ++c) f2 = fmaf(Ff[c], Ff[c], f2);
                f2max = fmaxf(f2max, f2);
            }
        }
        emitted |= 1u << p;
        if (aux) {
            const long long n = (long long)st.np * st.R;
            double* a = st.aux + i;
            a[kAuxRx * n] = w.r[0];
            a[kAuxRy * n] = w.r[1];
            a[kAuxRz * n] = w.r[2];
            // exit field of the Fresnel chain as a vector: e1 ep + e2 (ep x s)
            double v2x = w.ep[1] * w.k[2] - w.ep[2] * w.k[1];
            double v2y = w.ep[2] * w.k[0] - w.ep[0] * w.k[2];
            double v2z = w.ep[0] * w.k[1] - w.ep[1] * w.k[0];
            a[kAuxExr * n] = w.e1r * w.ep[0] + w.e2r * v2x;
            a[kAuxExi * n] = w.e1i * w.ep[0] + w.e2i * v2x;
            a[kAuxEyr * n] = w.e1r * w.ep[1] + w.e2r * v2y;
            a[kAuxEyi * n] = w.e1i * w.ep[1] + w.e2i * v2y;
            a[kAuxEzr * n] = w.e1r * w.ep[2] + w.e2r * v2z;
            a[kAuxEzi * n] = w.e1i * w.ep[2] + w.e2i * v2z;
            a[kAuxQ11 * n] = w.q11;
            a[kAuxQ12 * n] = w.q12;
            a[kAuxQ22 * n] = w.q22;
            a[kAuxEpx * n] = w.ep[0];
            a[kAuxEpy * n] = w.ep[1];
            a[kAuxEpz * n] = w.ep[2];
            a[kAuxDlegs * n] = 1.0 / w.pdet;
            a[kAuxPath * n] = w.path;
            a[kAuxNfLegs * n] = (double)w.nf_legs;
        }
    }
};

// Records in the [ray][order] layout of rtw_trace_points.
struct PointSink {
    const ObjDev* o;
    long long j;
    int np;
    double* s_out;
    double* F_out;
    double* psi_out;
    uint32_t* flags_out;

    __device__ void emit(int p, const ExitWave& w)
    {
        FarRecord fr;
        if (!far_record(*o, w, fr)) return;
        const long long i = j * np + p;
        if (s_out)
            for (int c = 0; c < 3; ++c) s_out[3 * i + c] = fr.s[c];
        if (F_out)
            for (int c = 0; c < 6; ++c) F_out[6 * i + c] = fr.F[c];
        if (psi_out) psi_out[i] = fr.psi;
        if (flags_out) flags_out[i] = fr.flags;
    }
};

__device__ __forceinline__ int find_object(const ObjDev* objs, int nobj, long long j)
{
    int lo = 0, hi = nobj - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (objs[mid].ray_offset <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// traces global ray j of object o and clears the flags of the orders it does not reach
// kSuper: the object set holds superellipsoids; each object takes the path of its own shape.
// the largest |F|^2 of the warp's rays, per object (oi), into st.fmax
__device__ __forceinline__ void record_fmax(const RaysDev& st, int oi, float f2max)
{
    if (!st.fmax) return;
    const unsigned int act = __activemask();
    const unsigned int peers = __match_any_sync(act, oi);
    // non-negative floats order as their bit patterns
    const unsigned int v = __reduce_max_sync(peers, __float_as_uint(f2max < 3.0e38f ? f2max : 0.0f));
    if ((threadIdx.x & 31) == __ffs(peers) - 1 && v) atomicMax(st.fmax + oi, v);
}

template <typename T, bool kNear = false, bool kSuper = false>
__device__ __forceinline__ void trace_one(const ObjDev* o, const RaysDev& st, long long j, int pmax, int aux, int oi)
{
    StateSink<kNear> sink{o, st, j, aux != 0, 0u, 0.0f};
    double x, y;
    if (ray_origin(*o, j - o->ray_offset, x, y)) {
        if constexpr (kSuper) {
            if (o->shape_e != 1.0) trace_ray<double, false, StateSink<kNear>, true>(*o, x, y, pmax, sink);
            else trace_ray<double, false>(*o, x, y, pmax, sink);
        } else {
            trace_ray<T, false>(*o, x, y, pmax, sink);
        }
    }
    for (int p = 0; p < st.np; ++p)
        if (!(sink.emitted & (1u << p))) st.flags[(long long)p * st.R + j] = 0u;
    record_fmax(st, oi, sink.f2max);
}

template <typename T, bool kNear = false, bool kSuper = false>
__device__ __forceinline__ void trace_kernel_body(const ObjDev* __restrict__ objs, int nobj, RaysDev st, int pmax,
                                                  int aux)
{
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= st.R) return;
    const int oi = nobj > 1 ? find_object(objs, nobj, j) : 0;
    trace_one<T, kNear, kSuper>(objs + oi, st, j, pmax, aux, oi);
}

// object owning work item `it` (largest i with item_first <= it)
__device__ __forceinline__ int find_item_object(const ObjDev* objs, int nobj, long long it)
{
    int lo = 0, hi = nobj - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (objs[mid].item_first <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Persistent batched trace: each CTA takes work items (object, 256 consecutive rays of it) from a
// counter until none is left.  Items are equal in cost up to misses, so taking them in order is
// the balanced schedule.  BS threads and MINB CTAs per SM are template parameters (the register
// cap follows from them); the loop ends after at most nitems / gridDim.x + 1 items per CTA.
template <typename T, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) trace_items_kernel(const ObjDev* __restrict__ objs, int nobj, RaysDev st,
                                                               int pmax, unsigned long long* next, long long nitems)
{
    __shared__ long long s_item;
    __shared__ int s_obj;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(next, 1ull);
            s_item = it;
            s_obj = it < nitems ? find_item_object(objs, nobj, it) : 0;
        }
        __syncthreads();
        const long long it = s_item;
        if (it >= nitems) return;
        const ObjDev* o = objs + s_obj;
        const long long first = (it - o->item_first) * kRaysPerItem;
        const long long nr = o->nx * o->ny;
        for (int r = threadIdx.x; r < kRaysPerItem; r += BS) {
            const long long local = first + r;
            if (local >= nr) break;
            trace_one<T>(o, st, o->ray_offset + local, pmax, 0, s_obj);
        }
    }
}

// every step in double precision (no aperture data: the writes of trace_kernel_fp64_aux compile away)
__global__ void __launch_bounds__(128) trace_kernel_fp64(const ObjDev* __restrict__ objs, int nobj, RaysDev st,
                                                         int pmax, int aux)
{
    (void)aux;
    trace_kernel_body<double>(objs, nobj, st, pmax, 0);
}

// the same, keeping the exit-wave data of the physical-optics integrals (RTW_TRACE_APERTURE)
__global__ void __launch_bounds__(128) trace_kernel_fp64_aux(const ObjDev* __restrict__ objs, int nobj,
                                                             RaysDev st, int pmax, int aux)
{
    (void)aux;
    trace_kernel_body<double>(objs, nobj, st, pmax, 1);
}

// the same, recording every ray where it crosses the sphere |M| = st.near_r
__global__ void __launch_bounds__(128) trace_kernel_fp64_near(const ObjDev* __restrict__ objs, int nobj,
                                                              RaysDev st, int pmax, int aux)
{
    trace_kernel_body<double, true>(objs, nobj, st, pmax, aux);
}

// object sets with superellipsoids (every step in double precision)
__global__ void __launch_bounds__(128) trace_kernel_fp64_super(const ObjDev* __restrict__ objs, int nobj,
                                                               RaysDev st, int pmax, int aux)
{
    trace_kernel_body<double, false, true>(objs, nobj, st, pmax, aux);
}

// the same, recording every ray where it crosses the sphere |M| = st.near_r
__global__ void __launch_bounds__(128) trace_kernel_fp64_super_near(const ObjDev* __restrict__ objs, int nobj,
                                                                    RaysDev st, int pmax, int aux)
{
    trace_kernel_body<double, true, true>(objs, nobj, st, pmax, aux);
}

// geometry, Fresnel and curvature in single precision; intersection points (polished by a
// double-precision Newton step), optical path and phase in double precision
__global__ void __launch_bounds__(128) trace_kernel_mixed(const ObjDev* __restrict__ objs, int nobj, RaysDev st,
                                                          int pmax, int aux)
{
    trace_kernel_body<float>(objs, nobj, st, pmax, aux);
}

// every step in double-float (pairs of single-precision numbers); positions and the optical path
// in double precision
__global__ void __launch_bounds__(128) trace_kernel_df(const ObjDev* __restrict__ objs, int nobj, RaysDev st,
                                                       int pmax, int aux)
{
    trace_kernel_body<df>(objs, nobj, st, pmax, aux);
}

__global__ void __launch_bounds__(128) trace_points_kernel(const ObjDev* __restrict__ obj, const double* __restrict__ xy,
                                                           long long n, int pmax, double* s_out, double* F_out,
                                                           double* psi_out, uint32_t* flags_out)
{
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int np = pmax + 1;
    if (flags_out)
        for (int p = 0; p < np; ++p) flags_out[j * np + p] = 0u;
    PointSink sink{obj, j, np, s_out, F_out, psi_out, flags_out};
    trace_ray_fp64<false>(*obj, xy[2 * j], xy[2 * j + 1], pmax, sink);
}

__global__ void export_kernel(RaysDev st, int order, long long first, long long count, double* s_out, double* F_out,
                              double* psi_out, uint32_t* flags_out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const long long i = (long long)order * st.R + first + t;
    const uint32_t f = st.flags[i];
    if (flags_out) flags_out[t] = f;
    const bool v = (f & kFlagValid) != 0;
    if (s_out) {
        double2 a = v ? st.s01[i] : make_double2(0.0, 0.0), b = v ? st.s2psi[i] : make_double2(0.0, 0.0);
        s_out[3 * t] = a.x;
        s_out[3 * t + 1] = a.y;
        s_out[3 * t + 2] = b.x;
    }
    if (psi_out) psi_out[t] = v ? st.s2psi[i].y : 0.0;
    if (F_out) {
        double2 fx = v ? st.Fx[i] : make_double2(0.0, 0.0), fy = v ? st.Fy[i] : make_double2(0.0, 0.0),
                fz = v ? st.Fz[i] : make_double2(0.0, 0.0);
        F_out[6 * t] = fx.x;
        F_out[6 * t + 1] = fx.y;
        F_out[6 * t + 2] = fy.x;
        F_out[6 * t + 3] = fy.y;
        F_out[6 * t + 4] = fz.x;
        F_out[6 * t + 5] = fz.y;
    }
}

}  // namespace

cudaError_t launch_trace(const ObjDev* d_objs, int nobj, RaysDev st, int pmax, bool aux, unsigned int* status,
                         cudaStream_t s, bool super_shapes)
{
    (void)status;
    if (st.R == 0) return cudaSuccess;
    const int bs = 128;
    const long long nb = (st.R + bs - 1) / bs;
    if (super_shapes && st.near_r > 0.0)
        trace_kernel_fp64_super_near<<<(unsigned)nb, bs, 0, s>>>(d_objs, nobj, st, pmax, aux ? 1 : 0);
    else if (super_shapes)
        trace_kernel_fp64_super<<<(unsigned)nb, bs, 0, s>>>(d_objs, nobj, st, pmax, aux ? 1 : 0);
    else if (st.near_r > 0.0)
        trace_kernel_fp64_near<<<(unsigned)nb, bs, 0, s>>>(d_objs, nobj, st, pmax, aux ? 1 : 0);
    else if (st.precision == 1)
        trace_kernel_mixed<<<(unsigned)nb, bs, 0, s>>>(d_objs, nobj, st, pmax, aux ? 1 : 0);
    else if (st.precision == 2)
        trace_kernel_df<<<(unsigned)nb, bs, 0, s>>>(d_objs, nobj, st, pmax, aux ? 1 : 0);
    else if (aux)
        trace_kernel_fp64_aux<<<(unsigned)nb, bs, 0, s>>>(d_objs, nobj, st, pmax, 1);
    else
        trace_kernel_fp64<<<(unsigned)nb, bs, 0, s>>>(d_objs, nobj, st, pmax, 0);
    return cudaGetLastError();
}

namespace {

template <typename T, int BS, int MINB>
cudaError_t launch_items(const ObjDev* d_objs, int nobj, const RaysDev& st, int pmax, unsigned long long* next,
                         long long nitems, int ctas_per_sm, cudaStream_t s)
{
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_items_kernel<T, BS, MINB>, BS, 0);
    if (e != cudaSuccess) return e;
    const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, std::max(occ, 1)) : std::max(occ, 1);
    const long long grid = std::min<long long>((long long)sms * per_sm, nitems);
    trace_items_kernel<T, BS, MINB><<<(unsigned)grid, BS, 0, s>>>(d_objs, nobj, st, pmax, next, nitems);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_items_variant(int variant, const ObjDev* d_objs, int nobj, const RaysDev& st, int pmax,
                                 unsigned long long* next, long long nitems, int ctas_per_sm, cudaStream_t s)
{
    switch (variant) {
    case 1: return launch_items<T, 64, 1>(d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
    case 2: return launch_items<T, 128, 1>(d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
    case 3: return launch_items<T, 256, 1>(d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
    case 4: return launch_items<T, 128, 3>(d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
    case 5: return launch_items<T, 256, 2>(d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_trace_items(const ObjDev* d_objs, int nobj, RaysDev st, int pmax, unsigned long long* next,
                               long long nitems, int variant, int ctas_per_sm, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (st.precision == 1)
        return launch_items_variant<float>(variant, d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
    if (st.precision == 2) {
        // double-float: the 128-thread instances only (register use as FP64)
        return variant == 4 ? launch_items<df, 128, 3>(d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s)
                            : launch_items<df, 128, 1>(d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
    }
    return launch_items_variant<double>(variant, d_objs, nobj, st, pmax, next, nitems, ctas_per_sm, s);
}

cudaError_t launch_trace_points(const ObjDev* d_obj, const double* xy, long long n, int pmax, double* s_out,
                                double* F_out, double* psi_out, uint32_t* flags_out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int bs = 128;
    trace_points_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(d_obj, xy, n, pmax, s_out, F_out, psi_out,
                                                                       flags_out);
    return cudaGetLastError();
}

cudaError_t launch_export(RaysDev st, int order, long long first, long long count, double* s_out, double* F_out,
                          double* psi_out, uint32_t* flags_out, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const int bs = 256;
    export_kernel<<<(unsigned)((count + bs - 1) / bs), bs, 0, s>>>(st, order, first, count, s_out, F_out, psi_out,
                                                                     flags_out);
    return cudaGetLastError();
}

}  // namespace rtw
