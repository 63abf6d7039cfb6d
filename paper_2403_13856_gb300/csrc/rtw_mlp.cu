// rtw_mlp.cu -- BF16 tensor-core kernels of the learned inverse-map proposal: fused forward
// (activations stay in registers from layer to layer), backward data pass, weight gradients,
// Adam, and the training samples drawn from the exact trace.
//
// Tensor-core tiles are mma.sync m16n8k16 (bf16 x bf16 -> f32).  A warp owns 16 rows; the f32
// accumulator fragment of one layer's 16 x 16 column block is, element for element, the bf16
// A fragment of the next layer's k-block, so a row tile runs through all four layers without
// leaving registers.  Weights sit in shared memory with rows padded by 8 bf16 so that the eight
// rows a fragment load touches fall in distinct banks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "rtw_launch.h"
#include "rtw_mlp.cuh"
#include "rtw_trace.cuh"

namespace rtw {

namespace {

constexpr int kLd16 = kMlpIn + 8;   // padded row of a 16-wide weight matrix
constexpr int kLd128 = kMlpH + 8;   // padded row of a 128-wide weight matrix

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// GELU, tanh form, and its derivative (single precision)
__device__ __forceinline__ float gelu_f(float z)
{
    const float c = 0.7978845608028654f;  // sqrt(2 / pi)
    return 0.5f * z * (1.0f + tanhf(c * (z + 0.044715f * z * z * z)));
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float c = 0.7978845608028654f;
    const float t = tanhf(c * (z + 0.044715f * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * z * z);
}

// acc (16 rows x 8 NT columns) = A (16 x 16 KK) . W^T with W (8 NT rows x 16 KK, row stride LD) in
// shared memory: B(k, n) = W[n][k], the column-major B fragment is a row segment of W
template <int NT, int KK, int LD>
__device__ __forceinline__ void layer_mma(float (&acc)[NT][4], const uint32_t (&a)[KK][4], const __nv_bfloat16* W,
                                          int g, int t)
{
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < KK; ++kk) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const __nv_bfloat16* w = W + (8 * j + g) * LD + 16 * kk + 2 * t;
            mma16816(acc[j], a[kk], *reinterpret_cast<const uint32_t*>(w), *reinterpret_cast<const uint32_t*>(w + 8));
        }
    }
}

// A fragment of a row-major bf16 matrix with 16 columns (rows beyond `rows` read as zero)
__device__ __forceinline__ void load_a16(const __nv_bfloat16* M, long long r0, long long rows, int g, int t,
                                         uint32_t (&a)[4])
{
    const long long ra = r0 + g, rb = r0 + g + 8;
    a[0] = ra < rows ? *reinterpret_cast<const uint32_t*>(M + ra * 16 + 2 * t) : 0u;
    a[1] = rb < rows ? *reinterpret_cast<const uint32_t*>(M + rb * 16 + 2 * t) : 0u;
    a[2] = ra < rows ? *reinterpret_cast<const uint32_t*>(M + ra * 16 + 8 + 2 * t) : 0u;
    a[3] = rb < rows ? *reinterpret_cast<const uint32_t*>(M + rb * 16 + 8 + 2 * t) : 0u;
}

// copies a (rows x cols) bf16 matrix into shared memory with row stride ld
__device__ __forceinline__ void stage(__nv_bfloat16* dst, const __nv_bfloat16* src, int rows, int cols, int ld)
{
    const int pairs = rows * cols / 2;
    for (int i = threadIdx.x; i < pairs; i += blockDim.x) {
        const int r = (2 * i) / cols, c = (2 * i) % cols;
        *reinterpret_cast<uint32_t*>(dst + r * ld + c) = reinterpret_cast<const uint32_t*>(src)[i];
    }
}

constexpr size_t kFwdSmem = sizeof(__nv_bfloat16) * (kMlpH * kLd16 + 2 * kMlpH * kLd128 + kMlpOut * kLd128) +
                            sizeof(float) * (3 * kMlpH + kMlpOut);

// bias + GELU on an accumulator block, packed as the next layer's A fragments; in training the
// pre-activations and the bf16 activations are stored
template <int NT, bool kTrain>
__device__ __forceinline__ void activate(const float (&acc)[NT][4], const float* bias, uint32_t (&an)[NT / 2][4],
                                         int g, int t, long long r0, long long rows, float* z, __nv_bfloat16* h)
{
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int col = 8 * j + 2 * t;
        const float z0 = acc[j][0] + bias[col], z1 = acc[j][1] + bias[col + 1];
        const float z2 = acc[j][2] + bias[col], z3 = acc[j][3] + bias[col + 1];
        const uint32_t p01 = pack_bf16(gelu_f(z0), gelu_f(z1)), p23 = pack_bf16(gelu_f(z2), gelu_f(z3));
        if (j & 1) {
            an[j >> 1][2] = p01;
            an[j >> 1][3] = p23;
        } else {
            an[j >> 1][0] = p01;
            an[j >> 1][1] = p23;
        }
        if (kTrain) {
            const long long ra = r0 + g, rb = r0 + g + 8;
            if (ra < rows) {
                *reinterpret_cast<float2*>(z + ra * kMlpH + col) = make_float2(z0, z1);
                *reinterpret_cast<uint32_t*>(h + ra * kMlpH + col) = p01;
            }
            if (rb < rows) {
                *reinterpret_cast<float2*>(z + rb * kMlpH + col) = make_float2(z2, z3);
                *reinterpret_cast<uint32_t*>(h + rb * kMlpH + col) = p23;
            }
        }
    }
}

// Forward pass: 4 warps per CTA, 16 rows per warp, grid-stride over 64-row tiles.
template <bool kTrain>
__global__ void __launch_bounds__(128) mlp_fwd_kernel(MlpWeights w, const __nv_bfloat16* __restrict__ X, long long rows,
                                                      float* __restrict__ Y, MlpActs acts)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* w2 = w1 + kMlpH * kLd16;
    __nv_bfloat16* w3 = w2 + kMlpH * kLd128;
    __nv_bfloat16* w4 = w3 + kMlpH * kLd128;
    float* bias = reinterpret_cast<float*>(w4 + kMlpOut * kLd128);
    stage(w1, w.w1, kMlpH, kMlpIn, kLd16);
    stage(w2, w.w2, kMlpH, kMlpH, kLd128);
    stage(w3, w.w3, kMlpH, kMlpH, kLd128);
    stage(w4, w.w4, kMlpOut, kMlpH, kLd128);
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
        bias[i] = w.theta[kMlpB1 + i];
        bias[kMlpH + i] = w.theta[kMlpB2 + i];
        bias[2 * kMlpH + i] = w.theta[kMlpB3 + i];
    }
    for (int i = threadIdx.x; i < kMlpOut; i += blockDim.x) bias[3 * kMlpH + i] = w.theta[kMlpB4 + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (long long tile = blockIdx.x; tile * 64 < rows; tile += gridDim.x) {
        const long long r0 = tile * 64 + 16 * warp;
        if (r0 >= rows) continue;
        uint32_t a0[1][4];
        load_a16(X, r0, rows, g, t, a0[0]);
        float acc[16][4];
        uint32_t a[8][4];
        layer_mma<16, 1, kLd16>(acc, a0, w1, g, t);
        activate<16, kTrain>(acc, bias, a, g, t, r0, rows, acts.z1, acts.h1);
        layer_mma<16, 8, kLd128>(acc, a, w2, g, t);
        activate<16, kTrain>(acc, bias + kMlpH, a, g, t, r0, rows, acts.z2, acts.h2);
        layer_mma<16, 8, kLd128>(acc, a, w3, g, t);
        activate<16, kTrain>(acc, bias + 2 * kMlpH, a, g, t, r0, rows, acts.z3, acts.h3);
        float out[2][4];
        layer_mma<2, 8, kLd128>(out, a, w4, g, t);
        const float* b4 = bias + 3 * kMlpH;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int col = 8 * j + 2 * t;
            const long long ra = r0 + g, rb = r0 + g + 8;
            if (ra < rows)
                *reinterpret_cast<float2*>(Y + ra * kMlpOut + col) = make_float2(out[j][0] + b4[col], out[j][1] + b4[col + 1]);
            if (rb < rows)
                *reinterpret_cast<float2*>(Y + rb * kMlpOut + col) = make_float2(out[j][2] + b4[col], out[j][3] + b4[col + 1]);
        }
    }
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
// cross-entropy towards it; mean over the labelled rows
__global__ void mlp_loss_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                const uint8_t* __restrict__ valid, long long rows, float beta, MlpActs acts)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows) return;
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
        atomicAdd(acts.scal, (double)((best - beta * logf(p[j])) * inv));
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

constexpr size_t kBwdSmem = sizeof(__nv_bfloat16) * (kMlpH * kLd16 + 2 * kMlpH * kLd128);

// dz of a layer from the accumulator of dh: dz = dh g'(z); stored in bf16 and packed as the next
// backward product's A fragments
template <int NT>
__device__ __forceinline__ void back_act(const float (&acc)[NT][4], const float* z, uint32_t (&an)[NT / 2][4], int g,
                                         int t, long long r0, long long rows, __nv_bfloat16* dz)
{
    const long long ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int col = 8 * j + 2 * t;
        float2 za = make_float2(0.0f, 0.0f), zb = make_float2(0.0f, 0.0f);
        if (ra < rows) za = *reinterpret_cast<const float2*>(z + ra * kMlpH + col);
        if (rb < rows) zb = *reinterpret_cast<const float2*>(z + rb * kMlpH + col);
        const uint32_t p01 = pack_bf16(acc[j][0] * gelu_grad_f(za.x), acc[j][1] * gelu_grad_f(za.y));
        const uint32_t p23 = pack_bf16(acc[j][2] * gelu_grad_f(zb.x), acc[j][3] * gelu_grad_f(zb.y));
        if (j & 1) {
            an[j >> 1][2] = p01;
            an[j >> 1][3] = p23;
        } else {
            an[j >> 1][0] = p01;
            an[j >> 1][1] = p23;
        }
        if (ra < rows) *reinterpret_cast<uint32_t*>(dz + ra * kMlpH + col) = p01;
        if (rb < rows) *reinterpret_cast<uint32_t*>(dz + rb * kMlpH + col) = p23;
    }
}

// Backward data pass: dh3 = dy W4, dz3 = dh3 g'(z3), dh2 = dz3 W3, ... (transposed weights in
// shared memory play the role W plays in the forward pass).
__global__ void __launch_bounds__(128) mlp_bwd_kernel(MlpWeights w, long long rows, MlpActs acts)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* w4t = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* w3t = w4t + kMlpH * kLd16;
    __nv_bfloat16* w2t = w3t + kMlpH * kLd128;
    stage(w4t, w.w4t, kMlpH, kMlpOut, kLd16);
    stage(w3t, w.w3t, kMlpH, kMlpH, kLd128);
    stage(w2t, w.w2t, kMlpH, kMlpH, kLd128);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (long long tile = blockIdx.x; tile * 64 < rows; tile += gridDim.x) {
        const long long r0 = tile * 64 + 16 * warp;
        if (r0 >= rows) continue;
        uint32_t a0[1][4];
        load_a16(acts.dyb, r0, rows, g, t, a0[0]);
        float acc[16][4];
        uint32_t a[8][4];
        layer_mma<16, 1, kLd16>(acc, a0, w4t, g, t);
        back_act<16>(acc, acts.z3, a, g, t, r0, rows, acts.dz3);
        layer_mma<16, 8, kLd128>(acc, a, w3t, g, t);
        back_act<16>(acc, acts.z2, a, g, t, r0, rows, acts.dz2);
        layer_mma<16, 8, kLd128>(acc, a, w2t, g, t);
        back_act<16>(acc, acts.z1, a, g, t, r0, rows, acts.dz1);
    }
}

// Weight gradients of one layer over a chunk of rows: dW[o][i] = sum_m D[m][o] A[m][i] (the
// product D^T A on the tensor cores, one warp per 16 outputs), db[o] = sum_m D[m][o].  Partial
// sums per chunk go to part[chunk] and are added in chunk order afterwards (deterministic).
constexpr int kWgradRows = 512;

template <int O, int I>
__device__ void wgrad_layer(const __nv_bfloat16* __restrict__ D, const __nv_bfloat16* __restrict__ A, long long rows,
                            long long m0, float* __restrict__ partW, float* __restrict__ partB, unsigned char* smem)
{
    __nv_bfloat16* ds = reinterpret_cast<__nv_bfloat16*>(smem);  // 16 x (O + 8)
    __nv_bfloat16* as = ds + 16 * (O + 8);                        // 16 x (I + 8)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    constexpr int NT = I / 8;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    float bsum = 0.0f;
    const long long m1 = min(m0 + (long long)kWgradRows, rows);
    for (long long mb = m0; mb < m1; mb += 16) {
        __syncthreads();
        for (int e = threadIdx.x; e < 16 * O; e += blockDim.x) {
            const int r = e / O, c = e % O;
            ds[r * (O + 8) + c] = (mb + r < m1) ? D[(mb + r) * O + c] : __float2bfloat16(0.0f);
        }
        for (int e = threadIdx.x; e < 16 * I; e += blockDim.x) {
            const int r = e / I, c = e % I;
            as[r * (I + 8) + c] = (mb + r < m1) ? A[(mb + r) * I + c] : __float2bfloat16(0.0f);
        }
        __syncthreads();
        if (threadIdx.x < O)
            for (int r = 0; r < 16; ++r) bsum += __bfloat162float(ds[r * (O + 8) + threadIdx.x]);
        if (16 * warp < O) {
            const int o0 = 16 * warp;
            uint32_t a[4];
            a[0] = pack_raw(ds[(2 * t) * (O + 8) + o0 + g], ds[(2 * t + 1) * (O + 8) + o0 + g]);
            a[1] = pack_raw(ds[(2 * t) * (O + 8) + o0 + g + 8], ds[(2 * t + 1) * (O + 8) + o0 + g + 8]);
            a[2] = pack_raw(ds[(2 * t + 8) * (O + 8) + o0 + g], ds[(2 * t + 9) * (O + 8) + o0 + g]);
            a[3] = pack_raw(ds[(2 * t + 8) * (O + 8) + o0 + g + 8], ds[(2 * t + 9) * (O + 8) + o0 + g + 8]);
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int n = 8 * j + g;
                const uint32_t b0 = pack_raw(as[(2 * t) * (I + 8) + n], as[(2 * t + 1) * (I + 8) + n]);
                const uint32_t b1 = pack_raw(as[(2 * t + 8) * (I + 8) + n], as[(2 * t + 9) * (I + 8) + n]);
                mma16816(acc[j], a, b0, b1);
            }
        }
    }
    if (16 * warp < O) {
        const int o0 = 16 * warp;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int col = 8 * j + 2 * t;
            partW[(o0 + g) * I + col] = acc[j][0];
            partW[(o0 + g) * I + col + 1] = acc[j][1];
            partW[(o0 + g + 8) * I + col] = acc[j][2];
            partW[(o0 + g + 8) * I + col + 1] = acc[j][3];
        }
    }
    if (threadIdx.x < O) partB[threadIdx.x] = bsum;
}

constexpr size_t kWgradSmem = sizeof(__nv_bfloat16) * 16 * 2 * (kMlpH + 8);

__global__ void __launch_bounds__(256) mlp_wgrad_kernel(const __nv_bfloat16* __restrict__ X, long long rows,
                                                        MlpActs acts, float* __restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const long long m0 = (long long)blockIdx.x * kWgradRows;
    float* p = part + (size_t)blockIdx.x * kMlpParams;
    switch (blockIdx.y) {
    case 0: wgrad_layer<kMlpH, kMlpIn>(acts.dz1, X, rows, m0, p + kMlpW1, p + kMlpB1, smem); break;
    case 1: wgrad_layer<kMlpH, kMlpH>(acts.dz2, acts.h1, rows, m0, p + kMlpW2, p + kMlpB2, smem); break;
    case 2: wgrad_layer<kMlpH, kMlpH>(acts.dz3, acts.h2, rows, m0, p + kMlpW3, p + kMlpB3, smem); break;
    default: wgrad_layer<kMlpOut, kMlpH>(acts.dyb, acts.h3, rows, m0, p + kMlpW4, p + kMlpB4, smem); break;
    }
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

cudaError_t mlp_prepare_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    if (e == cudaSuccess) e = mlp_prepare_tc_kernel();
    return e;
}

static int grid_for(long long rows)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (rows + 63) / 64;
    return (int)std::min<long long>(tiles, (long long)sms * 2);
}

cudaError_t launch_mlp_grad(const MlpWeights& w, const __nv_bfloat16* X, const float* T, const uint8_t* valid,
                            long long rows, float beta, const MlpActs& acts, float* part, float* grad, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(acts.scal, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    mlp_fwd_kernel<true><<<grid_for(rows), 128, kFwdSmem, s>>>(w, X, rows, acts.y, acts);
    const unsigned nb = (unsigned)((rows + 255) / 256);
    mlp_count_kernel<<<nb, 256, 0, s>>>(valid, rows, acts.scal);
    mlp_loss_kernel<<<nb, 256, 0, s>>>(acts.y, T, valid, rows, beta, acts);
    mlp_bwd_kernel<<<grid_for(rows), 128, kBwdSmem, s>>>(w, rows, acts);
    const int nchunks = (int)((rows + kWgradRows - 1) / kWgradRows);
    mlp_wgrad_kernel<<<dim3((unsigned)nchunks, 4), 256, kWgradSmem, s>>>(X, rows, acts, part);
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
