// rtw_mlp.cu -- training of the learned inverse-map proposal around the tensor-core passes of
// rtw_mlp_tc.cu: the loss and its gradient at the outputs, the chunk-ordered sum of the weight
// gradients, Adam, and the training samples drawn from the exact trace.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "rtw_launch.h"
#include "rtw_mlp.cuh"
#include "rtw_trace.cuh"

namespace rtw {

namespace {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// valid rows of the batch (count kept as a double, exact below 2^53)
__global__ void mlp_count_kernel(const uint8_t* __restrict__ valid, long long rows, double* scal)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int v = (i < rows && valid[i]) ? 1 : 0;
    const int n = __syncthreads_count(v);
    if (threadIdx.x == 0 && n) atomicAdd(scal + 1, (double)n);
}

// loss of each row and dL/dy: the row's label names the head of its branch (label - 1, from
// the ray's focal-line count); that head carries the squared distance, the logits a softmax
// cross-entropy towards it; mean over the labelled rows (per-block partial sums of the loss into
// lpart, added in a fixed order by mlp_loss_sum_kernel: the same value on every run)
__global__ void __launch_bounds__(256) mlp_loss_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                                       const uint8_t* __restrict__ valid, long long rows, float beta,
                                                       MlpActs acts, double* __restrict__ lpart)
{
    __shared__ double red[8];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double li = 0.0;  // this row's share of the loss
    if (i < rows) {
        float dy[kMlpOut];
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) dy[k] = 0.0f;
        if (valid[i]) {
            const double nv = acts.scal[1];
            const float inv = nv > 0.0 ? (float)(1.0 / nv) : 0.0f;
            const float* y = Y + i * kMlpOut;
            const float t0 = T[2 * i], t1 = T[2 * i + 1];
            const int j = (valid[i] - 1) & (kMlpHeads - 1);
            const float e0 = y[2 * j] - t0, e1 = y[2 * j + 1] - t1;
            const float best = e0 * e0 + e1 * e1;
            float zmax = y[8];
#pragma unroll
            for (int k = 1; k < kMlpHeads; ++k) zmax = fmaxf(zmax, y[8 + k]);
            float p[kMlpHeads], se = 0.0f;
#pragma unroll
            for (int k = 0; k < kMlpHeads; ++k) {
                p[k] = expf(y[8 + k] - zmax);
                se += p[k];
            }
            const float ise = 1.0f / se;
#pragma unroll
            for (int k = 0; k < kMlpHeads; ++k) p[k] *= ise;
            li = (double)((best - beta * logf(p[j])) * inv);
            dy[2 * j] = 2.0f * (y[2 * j] - t0) * inv;
            dy[2 * j + 1] = 2.0f * (y[2 * j + 1] - t1) * inv;
#pragma unroll
            for (int k = 0; k < kMlpHeads; ++k) dy[8 + k] = beta * (p[k] - (k == j ? 1.0f : 0.0f)) * inv;
        }
#pragma unroll
        for (int k = 0; k < kMlpOut; k += 2) {
            *reinterpret_cast<float2*>(acts.dy + i * kMlpOut + k) = make_float2(dy[k], dy[k + 1]);
            *reinterpret_cast<uint32_t*>(acts.dyb + i * kMlpOut + k) = pack_bf16(dy[k], dy[k + 1]);
        }
    }
    // the block's loss in a fixed order (warps, then the block), one partial per block
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) li += __shfl_down_sync(0xffffffffu, li, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = li;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < 8; ++w) b += red[w];
        lpart[blockIdx.x] = b;
    }
}

// the loss: the blocks' partials added in a fixed order (thread t takes partials t, t + 256, ...,
// then a fixed tree over the threads): the same value on every run
__global__ void __launch_bounds__(256) mlp_loss_sum_kernel(const double* __restrict__ lpart, int nblocks, double* scal)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) s += lpart[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[0] = red[0];
}

// grad[i] = sum over chunks of part[chunk][i], in chunk order
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nchunks, float* __restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float s = 0.0f;
    for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * kMlpParams + i];
    grad[i] = s;
}

// Adam on the FP32 master parameters (update = 0: only refresh the bf16 copies), then the bf16
// weight copies in forward (out x in) and transposed (in x out) layout
__global__ void mlp_adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ grad, int update, float lr, float b1, float b2, float eps,
                                float c1, float c2, __nv_bfloat16* w1, __nv_bfloat16* w2, __nv_bfloat16* w3,
                                __nv_bfloat16* w4, __nv_bfloat16* w2t, __nv_bfloat16* w3t, __nv_bfloat16* w4t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float th = theta[i];
    if (update) {
        const float gr = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gr;
        const float vi = b2 * v[i] + (1.0f - b2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        th -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        theta[i] = th;
    }
    const __nv_bfloat16 hb = __float2bfloat16_rn(th);
    if (i < kMlpB1) {
        w1[i - kMlpW1] = hb;
    } else if (i >= kMlpW2 && i < kMlpB2) {
        const int k = i - kMlpW2, o = k / kMlpH, in = k % kMlpH;
        w2[k] = hb;
        w2t[in * kMlpH + o] = hb;
    } else if (i >= kMlpW3 && i < kMlpB3) {
        const int k = i - kMlpW3, o = k / kMlpH, in = k % kMlpH;
        w3[k] = hb;
        w3t[in * kMlpH + o] = hb;
    } else if (i >= kMlpW4 && i < kMlpB4) {
        const int k = i - kMlpW4, o = k / kMlpH, in = k % kMlpH;
        w4[k] = hb;
        w4t[in * kMlpOut + o] = hb;
    }
}

// exit directions and focal-line counts of orders 0..pmax of one ray
struct DirSink {
    const ObjDev* o;
    double s[kMaxOrders][3];
    uint8_t nf[kMaxOrders];
    unsigned int got;
    __device__ void emit(int p, const ExitWave& w)
    {
        FarRecord r;
        if (far_record(*o, w, r)) {
            s[p][0] = r.s[0];
            s[p][1] = r.s[1];
            s[p][2] = r.s[2];
            nf[p] = (uint8_t)flag_nf(r.flags);
            got |= 1u << p;
        }
    }
};

// Training samples: ray i enters object obj_index[i] at unit-disk point uv[i]; for every order p
// it leaves along s_p, giving features (s_p, object) and target uv in network p's batch.
__global__ void mlp_samples_kernel(const ObjDev* __restrict__ objs, const ObjFeat* __restrict__ feat, int nobj,
                                   const double* __restrict__ uv, const int* __restrict__ oidx, long long n, int pmax,
                                   __nv_bfloat16* __restrict__ X, float* __restrict__ T, uint8_t* __restrict__ valid)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int oraw = oidx[i];
    const bool known = oraw >= 0 && oraw < nobj;  // an unknown object index gives invalid rows
    const int oi = known ? oraw : 0;
    const ObjDev* o = objs + oi;
    const ObjFeat& f = feat[oi];
    const double u0 = uv[2 * i], u1 = uv[2 * i + 1];
    const double d1 = u1 / f.l11, d0 = (u0 - f.l10 * d1) / f.l00;
    DirSink sink;
    sink.o = o;
    sink.got = 0u;
    if (known) trace_ray_fp64<false>(*o, o->c[0] + d0, o->c[1] + d1, pmax, sink);
    for (int p = 0; p <= pmax; ++p) {
        const long long r = (long long)p * n + i;
        const bool ok = (sink.got >> p) & 1u;
        valid[r] = ok ? (uint8_t)(1 + (sink.nf[p] & 3)) : 0;  // label: head N_f mod 4
        T[2 * r] = (float)u0;
        T[2 * r + 1] = (float)u1;
        __nv_bfloat16* x = X + r * kMlpIn;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
        if (ok) {
            s0 = (float)sink.s[p][0];
            s1 = (float)sink.s[p][1];
            s2 = (float)sink.s[p][2];
        }
        x[0] = __float2bfloat16_rn(s0);
        x[1] = __float2bfloat16_rn(s1);
        x[2] = __float2bfloat16_rn(s2);
        for (int k = 0; k < 13; ++k) x[3 + k] = __float2bfloat16_rn(f.f[k]);
    }
}

}  // namespace

cudaError_t mlp_prepare_kernels() { return mlp_prepare_tc_kernel(); }

cudaError_t launch_mlp_grad(const MlpWeights& w, const __nv_bfloat16* X, const float* T, const uint8_t* valid,
                            long long rows, float beta, const MlpActs& acts, float* part, float* grad,
                            unsigned int* status, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(acts.scal, 0, 2 * sizeof(double), s);
    if (e == cudaSuccess) e = launch_mlp_train_tc(w, X, rows, acts, status, s);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((rows + 255) / 256);
    mlp_count_kernel<<<nb, 256, 0, s>>>(valid, rows, acts.scal);
    // the loss partials borrow the weight-gradient partial buffer, which is written only later
    double* lpart = reinterpret_cast<double*>(part);
    mlp_loss_kernel<<<nb, 256, 0, s>>>(acts.y, T, valid, rows, beta, acts, lpart);
    mlp_loss_sum_kernel<<<1, 256, 0, s>>>(lpart, (int)nb, acts.scal);
    e = launch_mlp_backward_tc(w, rows, acts, status, s);
    if (e != cudaSuccess) return e;
    const int nchunks = launch_mlp_wgrad_tc(X, rows, acts, part, status, s, &e);
    if (e != cudaSuccess) return e;
    mlp_reduce_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(part, nchunks, grad);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* theta, float* m, float* v, const float* grad, int update, float lr, float b1,
                            float b2, float eps, float c1, float c2, __nv_bfloat16* w1, __nv_bfloat16* w2,
                            __nv_bfloat16* w3, __nv_bfloat16* w4, __nv_bfloat16* w2t, __nv_bfloat16* w3t,
                            __nv_bfloat16* w4t, cudaStream_t s)
{
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, m, v, grad, update, lr, b1, b2, eps, c1, c2, w1,
                                                              w2, w3, w4, w2t, w3t, w4t);
    return cudaGetLastError();
}

cudaError_t launch_mlp_samples(const ObjDev* objs, const ObjFeat* feat, int nobj, const double* uv, const int* oidx,
                               long long n, int pmax, __nv_bfloat16* X, float* T, uint8_t* valid, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    mlp_samples_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(objs, feat, nobj, uv, oidx, n, pmax, X, T, valid);
    return cudaGetLastError();
}

}  // namespace rtw
