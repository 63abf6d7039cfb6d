// rtw_mlp_api.cu -- host side of the learned inverse-map proposal: network handles, training
// samples, forward, gradients and Adam (the C ABI of include/rtw.h, "learned proposal").
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "rtw.h"
#include "rtw_host.h"
#include "rtw_launch.h"

using rtw::host::align_up;
using rtw::host::fail;

namespace {

// one network: FP32 master parameters, Adam moments, gradient, bf16 weight copies
struct Net {
    float* theta = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    __nv_bfloat16* w1 = nullptr;
    __nv_bfloat16* w2 = nullptr;
    __nv_bfloat16* w3 = nullptr;
    __nv_bfloat16* w4 = nullptr;
    __nv_bfloat16* w2t = nullptr;
    __nv_bfloat16* w3t = nullptr;
    __nv_bfloat16* w4t = nullptr;
    long long step = 0;
};

}  // namespace

struct rtw_mlp {
    int device = 0;
    int n_orders = 0;
    void* block = nullptr;  // every network's parameters
    std::vector<Net> nets;
    // training workspace for up to ws_rows rows
    void* ws = nullptr;
    long long ws_rows = 0;
    rtw::MlpActs acts{};
    float* part = nullptr;
};

namespace {

rtw::MlpWeights weights_of(const Net& n)
{
    rtw::MlpWeights w;
    w.w1 = n.w1;
    w.w2 = n.w2;
    w.w3 = n.w3;
    w.w4 = n.w4;
    w.w2t = n.w2t;
    w.w3t = n.w3t;
    w.w4t = n.w4t;
    w.theta = n.theta;
    return w;
}

int refresh(const Net& n, cudaStream_t s)
{
    RTW_CUDA(rtw::launch_mlp_adam(n.theta, n.m, n.v, n.grad, 0, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, n.w1, n.w2, n.w3, n.w4,
                                  n.w2t, n.w3t, n.w4t, s));
    return RTW_OK;
}

int check_order(const rtw_mlp* m, int order)
{
    if (!m) return fail(RTW_ERR_ARG, "learned proposal: null network handle");
    if (order < 0 || order >= m->n_orders) return fail(RTW_ERR_ARG, "learned proposal: order %d out of range", order);
    return RTW_OK;
}

// training workspace for `rows` rows
int ensure_ws(rtw_mlp* m, long long rows)
{
    if (rows <= m->ws_rows) return RTW_OK;
    const size_t r = (size_t)rows;
    const size_t nchunks = (r + 511) / 512;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t oz1 = take(r * 128 * 4), oz2 = take(r * 128 * 4), oz3 = take(r * 128 * 4);
    const size_t oh1 = take(r * 128 * 2), oh2 = take(r * 128 * 2), oh3 = take(r * 128 * 2);
    const size_t oy = take(r * 16 * 4), ody = take(r * 16 * 4), odyb = take(r * 16 * 2);
    const size_t odz1 = take(r * 128 * 2), odz2 = take(r * 128 * 2), odz3 = take(r * 128 * 2);
    const size_t oscal = take(2 * sizeof(double));
    const size_t opart = take(nchunks * rtw::kMlpParams * sizeof(float));
    if (m->ws) cudaFree(m->ws);
    m->ws = nullptr;
    m->ws_rows = 0;
    if (cudaMalloc(&m->ws, off) != cudaSuccess) return fail(RTW_ERR_NOMEM, "learned proposal: workspace of %zu bytes", off);
    char* b = (char*)m->ws;
    m->acts.z1 = (float*)(b + oz1);
    m->acts.z2 = (float*)(b + oz2);
    m->acts.z3 = (float*)(b + oz3);
    m->acts.h1 = (__nv_bfloat16*)(b + oh1);
    m->acts.h2 = (__nv_bfloat16*)(b + oh2);
    m->acts.h3 = (__nv_bfloat16*)(b + oh3);
    m->acts.y = (float*)(b + oy);
    m->acts.dy = (float*)(b + ody);
    m->acts.dyb = (__nv_bfloat16*)(b + odyb);
    m->acts.dz1 = (__nv_bfloat16*)(b + odz1);
    m->acts.dz2 = (__nv_bfloat16*)(b + odz2);
    m->acts.dz3 = (__nv_bfloat16*)(b + odz3);
    m->acts.scal = (double*)(b + oscal);
    m->part = (float*)(b + opart);
    m->ws_rows = rows;
    return RTW_OK;
}

}  // namespace

namespace rtw {
namespace host {

// per-object feature table of the learned path (host arithmetic from the object description)
void object_features(const ObjHost& o, ObjFeat& f)
{
    std::memset(&f, 0, sizeof(f));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) f.f[3 * i + j] = (float)o.R[i][j];
    const double L = std::fmax(o.a[0], std::fmax(o.a[1], o.a[2]));
    for (int i = 0; i < 3; ++i) f.f[9 + i] = (float)(o.a[i] / L);
    f.f[12] = (float)(o.m - 1.0);
    f.l00 = std::sqrt(o.S[0][0]);
    f.l10 = o.S[1][0] / f.l00;
    f.l11 = std::sqrt(o.S[1][1] - f.l10 * f.l10);
}

MlpWeights mlp_weights(const rtw_mlp* m, int order) { return weights_of(m->nets[(size_t)order]); }

}  // namespace host
}  // namespace rtw

extern "C" {

int rtw_mlp_create(int n_orders, const float* init, rtw_mlp** out)
{
    if (!out || n_orders < 1 || n_orders > rtw::kMaxOrders) return fail(RTW_ERR_ARG, "rtw_mlp_create: arguments");
    *out = nullptr;
    rtw_mlp* m = new (std::nothrow) rtw_mlp();
    if (!m) return fail(RTW_ERR_NOMEM, "rtw_mlp_create: host allocation");
    RTW_CUDA(cudaGetDevice(&m->device));
    RTW_CUDA(rtw::mlp_prepare_kernels());
    const size_t P = rtw::kMlpParams;
    const size_t fl = align_up(P * sizeof(float), 256);
    const size_t bf = align_up(P * sizeof(__nv_bfloat16), 256);
    const size_t per = 4 * fl + 2 * bf;  // theta m v grad, forward and transposed bf16 copies
    if (cudaMalloc(&m->block, per * (size_t)n_orders) != cudaSuccess) {
        delete m;
        return fail(RTW_ERR_NOMEM, "rtw_mlp_create: parameters");
    }
    cudaMemset(m->block, 0, per * (size_t)n_orders);
    m->n_orders = n_orders;
    m->nets.resize((size_t)n_orders);
    for (int p = 0; p < n_orders; ++p) {
        char* b = (char*)m->block + per * (size_t)p;
        Net& n = m->nets[(size_t)p];
        n.theta = (float*)b;
        n.m = (float*)(b + fl);
        n.v = (float*)(b + 2 * fl);
        n.grad = (float*)(b + 3 * fl);
        __nv_bfloat16* w = (__nv_bfloat16*)(b + 4 * fl);
        n.w1 = w + rtw::kMlpW1;
        n.w2 = w + rtw::kMlpW2;
        n.w3 = w + rtw::kMlpW3;
        n.w4 = w + rtw::kMlpW4;
        __nv_bfloat16* wt = (__nv_bfloat16*)(b + 4 * fl + bf);
        n.w2t = wt + rtw::kMlpW2;
        n.w3t = wt + rtw::kMlpW3;
        n.w4t = wt + rtw::kMlpW4;
        if (init) RTW_CUDA(cudaMemcpy(n.theta, init + P * (size_t)p, P * sizeof(float), cudaMemcpyHostToDevice));
        int rc = refresh(n, nullptr);
        if (rc != RTW_OK) return rc;
    }
    RTW_CUDA(cudaDeviceSynchronize());
    *out = m;
    return RTW_OK;
}

void rtw_mlp_destroy(rtw_mlp* m)
{
    if (!m) return;
    if (m->block) cudaFree(m->block);
    if (m->ws) cudaFree(m->ws);
    delete m;
}

int rtw_mlp_get(const rtw_mlp* m, int order, float* theta, float* adam_m, float* adam_v, int64_t* step)
{
    int rc = check_order(m, order);
    if (rc != RTW_OK) return rc;
    const Net& n = m->nets[(size_t)order];
    const size_t b = rtw::kMlpParams * sizeof(float);
    if (theta) RTW_CUDA(cudaMemcpy(theta, n.theta, b, cudaMemcpyDeviceToHost));
    if (adam_m) RTW_CUDA(cudaMemcpy(adam_m, n.m, b, cudaMemcpyDeviceToHost));
    if (adam_v) RTW_CUDA(cudaMemcpy(adam_v, n.v, b, cudaMemcpyDeviceToHost));
    if (step) *step = n.step;
    return RTW_OK;
}

int rtw_mlp_set(rtw_mlp* m, int order, const float* theta, const float* adam_m, const float* adam_v, int64_t step)
{
    int rc = check_order(m, order);
    if (rc != RTW_OK) return rc;
    Net& n = m->nets[(size_t)order];
    const size_t b = rtw::kMlpParams * sizeof(float);
    if (theta) RTW_CUDA(cudaMemcpy(n.theta, theta, b, cudaMemcpyHostToDevice));
    if (adam_m) RTW_CUDA(cudaMemcpy(n.m, adam_m, b, cudaMemcpyHostToDevice));
    if (adam_v) RTW_CUDA(cudaMemcpy(n.v, adam_v, b, cudaMemcpyHostToDevice));
    if (step < 0) return fail(RTW_ERR_ARG, "rtw_mlp_set: step < 0");
    n.step = step;
    rc = refresh(n, nullptr);
    if (rc != RTW_OK) return rc;
    RTW_CUDA(cudaDeviceSynchronize());
    return RTW_OK;
}

int rtw_mlp_samples(const rtw_object* obj, const double* uv, const int32_t* obj_index, int64_t n, int p_max,
                    void* X, float* T, uint8_t* valid, void* stream)
{
    if (!obj || (n > 0 && (!uv || !obj_index || !X || !T || !valid)))
        return fail(RTW_ERR_ARG, "rtw_mlp_samples: null pointer");
    if (n < 0 || p_max < 0 || p_max >= rtw::kMaxOrders) return fail(RTW_ERR_ARG, "rtw_mlp_samples: sizes");
    if (n == 0) return RTW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<rtw::ObjDev> od((size_t)obj->count);
    std::vector<rtw::ObjFeat> of((size_t)obj->count);
    for (int i = 0; i < obj->count; ++i) {
        if (obj->h[(size_t)i].src) return fail(RTW_ERR_UNSUPPORTED, "rtw_mlp_samples: plane waves only");
        if (obj->h[(size_t)i].shape_e != 1.0) return fail(RTW_ERR_UNSUPPORTED, "rtw_mlp_samples: ellipsoids only");
        rtw::host::fill_objdev(obj->h[(size_t)i], od[(size_t)i]);
        od[(size_t)i].grid = rtw::kGridSquare;
        rtw::host::object_features(obj->h[(size_t)i], of[(size_t)i]);
    }
    // per-call tables, freed after the kernel has been ordered
    void* tab = nullptr;
    const size_t b0 = align_up(sizeof(rtw::ObjDev) * od.size(), 256), b1 = sizeof(rtw::ObjFeat) * of.size();
    RTW_CUDA(cudaMallocAsync(&tab, b0 + b1, s));
    RTW_CUDA(cudaMemcpyAsync(tab, od.data(), sizeof(rtw::ObjDev) * od.size(), cudaMemcpyHostToDevice, s));
    RTW_CUDA(cudaMemcpyAsync((char*)tab + b0, of.data(), b1, cudaMemcpyHostToDevice, s));
    cudaError_t e = rtw::launch_mlp_samples((const rtw::ObjDev*)tab, (const rtw::ObjFeat*)((char*)tab + b0),
                                            obj->count, uv, obj_index, n, p_max, (__nv_bfloat16*)X, T, valid, s);
    cudaFreeAsync(tab, s);
    if (e != cudaSuccess) return rtw::host::cuda_fail(e, "mlp samples launch");
    return RTW_OK;
}

int rtw_mlp_forward(const rtw_mlp* m, int order, const void* X, int64_t rows, float* Y, void* stream)
{
    int rc = check_order(m, order);
    if (rc != RTW_OK) return rc;
    if (rows < 0 || (rows > 0 && (!X || !Y))) return fail(RTW_ERR_ARG, "rtw_mlp_forward: arguments");
    if (((uintptr_t)X | (uintptr_t)Y) & 15u) return fail(RTW_ERR_ARG, "rtw_mlp_forward: X and Y must be 16-byte aligned");
    unsigned int* status = rtw::host::status_word(m->device);
    if (!status) return fail(RTW_ERR_CUDA, "rtw_mlp_forward: status word");
    RTW_CUDA(rtw::launch_mlp_forward(weights_of(m->nets[(size_t)order]), (const __nv_bfloat16*)X, rows, Y, status,
                                     (cudaStream_t)stream));
    return RTW_OK;
}

int rtw_mlp_activation_eval(const float* x, float* y, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !y))) return fail(RTW_ERR_ARG, "rtw_mlp_activation_eval: arguments");
    RTW_CUDA(rtw::launch_activation_eval(x, y, n, (cudaStream_t)stream));
    return RTW_OK;
}

int rtw_mlp_grad(rtw_mlp* m, int order, const void* X, const float* T, const uint8_t* valid, int64_t rows, float beta,
                 double* loss_out, void* stream)
{
    int rc = check_order(m, order);
    if (rc != RTW_OK) return rc;
    if (rows < 1 || !X || !T || !valid) return fail(RTW_ERR_ARG, "rtw_mlp_grad: arguments");
    if ((uintptr_t)X & 15u) return fail(RTW_ERR_ARG, "rtw_mlp_grad: X must be 16-byte aligned");
    if (rows >= (1ll << 31)) return fail(RTW_ERR_ARG, "rtw_mlp_grad: rows < 2^31");
    rc = ensure_ws(m, rows);
    if (rc != RTW_OK) return rc;
    unsigned int* status = rtw::host::status_word(m->device);
    if (!status) return fail(RTW_ERR_CUDA, "rtw_mlp_grad: status word");
    cudaStream_t s = (cudaStream_t)stream;
    Net& n = m->nets[(size_t)order];
    RTW_CUDA(rtw::launch_mlp_grad(weights_of(n), (const __nv_bfloat16*)X, T, valid, rows, beta, m->acts, m->part, n.grad,
                                  status, s));
    if (loss_out) RTW_CUDA(cudaMemcpyAsync(loss_out, m->acts.scal, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return RTW_OK;
}

int rtw_mlp_grad_get(const rtw_mlp* m, int order, float* grad, void* stream)
{
    int rc = check_order(m, order);
    if (rc != RTW_OK) return rc;
    if (!grad) return fail(RTW_ERR_ARG, "rtw_mlp_grad_get: null pointer");
    RTW_CUDA(cudaMemcpyAsync(grad, m->nets[(size_t)order].grad, rtw::kMlpParams * sizeof(float), cudaMemcpyDefault,
                             (cudaStream_t)stream));
    return RTW_OK;
}

int rtw_mlp_adam(rtw_mlp* m, int order, float lr, const float* grad, void* stream)
{
    int rc = check_order(m, order);
    if (rc != RTW_OK) return rc;
    if (!(lr > 0.0f)) return fail(RTW_ERR_ARG, "rtw_mlp_adam: lr must be positive");
    Net& n = m->nets[(size_t)order];
    n.step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)n.step)), c2 = (float)(1.0 - std::pow(b2, (double)n.step));
    RTW_CUDA(rtw::launch_mlp_adam(n.theta, n.m, n.v, grad ? grad : n.grad, 1, lr, (float)b1, (float)b2, 1e-8f, c1, c2,
                                  n.w1, n.w2, n.w3, n.w4, n.w2t, n.w3t, n.w4t, (cudaStream_t)stream));
    return RTW_OK;
}

}  // extern "C"
