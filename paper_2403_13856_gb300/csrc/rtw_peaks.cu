// rtw_peaks.cu -- throughput kernels of the floating-point pipes, the denominators of the trace
// kernels' rooflines (the paper has no counterpart).
//
// Every thread runs kChains independent fused multiply-add chains x <- x b + c (|b| < 1, so the
// values stay finite), unrolled, with no memory traffic: a launch of SMs x blocks_per_sm blocks of
// 256 threads keeps every scheduler issuing FMAs back to back.  The chains' sum is written to the
// sink only when it equals a value no chain can reach, so the compiler keeps every FMA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rtw.h"
#include "rtw_host.h"

namespace rtw {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) pipe_peak_kernel(long long iters, T* sink)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)k;
    const T b = (T)0.9990234375, c = (T)0.0009765625;  // exact in both precisions
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == (T)-1) sink[0] = s;
}

// packed single precision: one fma.rn.f32x2 instruction per pair of chains
__global__ void __launch_bounds__(kPeakThreads) pipe_peak_f32x2_kernel(long long iters, float* sink)
{
    float2 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = make_float2((threadIdx.x + 1) * 1e-3f + k, (threadIdx.x + 2) * 1e-3f - k);
    const float2 b = make_float2(0.9990234375f, 0.9990234375f), c = make_float2(0.0009765625f, 0.0009765625f);
    const unsigned long long bb = *reinterpret_cast<const unsigned long long*>(&b);
    const unsigned long long cc = *reinterpret_cast<const unsigned long long*>(&c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                unsigned long long v = *reinterpret_cast<unsigned long long*>(&x[k]);
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v) : "l"(bb), "l"(cc));
                x[k] = *reinterpret_cast<float2*>(&v);
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
    if (s == -1.0f) sink[0] = s;
}

}  // namespace
}  // namespace rtw

extern "C" {

int rtw_pipe_peak(int kind, int64_t iters, int blocks_per_sm, void* sink, double* flops, void* stream)
{
    using rtw::host::fail;
    if (!sink || !flops) return fail(RTW_ERR_ARG, "rtw_pipe_peak: null pointer");
    if (iters < 1 || iters > (1ll << 30) || blocks_per_sm < 1 || blocks_per_sm > 32)
        return fail(RTW_ERR_ARG, "rtw_pipe_peak: iters in [1, 2^30], blocks_per_sm in [1, 32]");
    int dev = 0, sms = 0;
    RTW_CUDA(cudaGetDevice(&dev));
    RTW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    cudaStream_t s = (cudaStream_t)stream;
    const double fma_per_thread = (double)iters * rtw::kUnroll * rtw::kChains;
    double per_fma = 2.0;
    switch (kind) {
    case RTW_PEAK_FP64:
        rtw::pipe_peak_kernel<double><<<grid, rtw::kPeakThreads, 0, s>>>(iters, (double*)sink);
        break;
    case RTW_PEAK_FP32:
        rtw::pipe_peak_kernel<float><<<grid, rtw::kPeakThreads, 0, s>>>(iters, (float*)sink);
        break;
    case RTW_PEAK_FP32X2:
        rtw::pipe_peak_f32x2_kernel<<<grid, rtw::kPeakThreads, 0, s>>>(iters, (float*)sink);
        per_fma = 4.0;  // two lanes of a packed pair
        break;
    default:
        return fail(RTW_ERR_ARG, "rtw_pipe_peak: kind %d", kind);
    }
    RTW_CUDA(cudaGetLastError());
    *flops = per_fma * fma_per_thread * grid * rtw::kPeakThreads;
    return RTW_OK;
}

}  // extern "C"
