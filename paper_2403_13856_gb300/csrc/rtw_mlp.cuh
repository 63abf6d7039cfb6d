// rtw_mlp.cuh -- device pieces of the learned inverse-map proposal (internal to librtw).
//
// Per scattering order one network: 16 features -> 3 hidden layers of 128 (GELU, tanh form) ->
// 16 outputs (4 candidate entry points uv in unit-disk coordinates, 4 logits, 4 unused).
// Weights in bfloat16 for the tensor cores, FP32 accumulation, FP32 master weights and Adam
// moments.  Parameter layout (floats): W1 (128 x 16), b1, W2 (128 x 128), b2, W3, b3,
// W4 (16 x 128), b4; every W row-major (out x in).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rtw {

constexpr int kMlpIn = 16, kMlpH = 128, kMlpOut = 16, kMlpHeads = 4;
constexpr int kMlpW1 = 0;
constexpr int kMlpB1 = kMlpW1 + kMlpH * kMlpIn;
constexpr int kMlpW2 = kMlpB1 + kMlpH;
constexpr int kMlpB2 = kMlpW2 + kMlpH * kMlpH;
constexpr int kMlpW3 = kMlpB2 + kMlpH;
constexpr int kMlpB3 = kMlpW3 + kMlpH * kMlpH;
constexpr int kMlpW4 = kMlpB3 + kMlpH;
constexpr int kMlpB4 = kMlpW4 + kMlpOut * kMlpH;
constexpr int kMlpParams = kMlpB4 + kMlpOut;

// bfloat16 copies of one network's weights as the kernels read them
struct MlpWeights {
    const __nv_bfloat16* w1;   // 128 x 16  (out x in)
    const __nv_bfloat16* w2;   // 128 x 128
    const __nv_bfloat16* w3;   // 128 x 128
    const __nv_bfloat16* w4;   // 16 x 128
    const __nv_bfloat16* w2t;  // 128 x 128 (in x out), for the backward pass
    const __nv_bfloat16* w3t;
    const __nv_bfloat16* w4t;  // 128 x 16
    const float* theta;        // FP32 master parameters (biases are read from here)
};

// training activations of a batch of rows
struct MlpActs {
    float* z1;             // rows x 128 pre-activations
    float* z2;
    float* z3;
    __nv_bfloat16* h1;     // rows x 128 bf16(g(z))
    __nv_bfloat16* h2;
    __nv_bfloat16* h3;
    float* y;              // rows x 16
    float* dy;             // rows x 16
    __nv_bfloat16* dyb;    // rows x 16
    __nv_bfloat16* dz1;    // rows x 128
    __nv_bfloat16* dz2;
    __nv_bfloat16* dz3;
    double* scal;          // [0] loss sum, [1] valid rows
};

// per-object inputs of the learned path: features 3..15 (rotation body -> lab row-major,
// semi-axes over the largest, m - 1) and the Cholesky factor of the projected ellipse
struct ObjFeat {
    float f[13];
    float pad[3];
    double l00, l10, l11;
    double pad2;
};

}  // namespace rtw
