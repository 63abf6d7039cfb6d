// rtw_learned.cu -- the far field from learned entry-point proposals: for every (object,
// direction) row and order p, network p proposes 4 entry points; each confident head seeds Newton
// steps on the exact FP64 trace; converged roots are deduplicated and summed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "rtw.h"
#include "rtw_device.cuh"
#include "rtw_host.h"
#include "rtw_launch.h"

using rtw::host::align_up;
using rtw::host::fail;

namespace rtw {
namespace {

constexpr unsigned int kMaskCausticL = 1u;  // the dense path's RTW_MASK_CAUSTIC bit
// root-count byte: bit 7 marks a row where a confident head's Newton steps did not converge
constexpr uint8_t kRootUncertain = 0x80u;
// single-precision first approach (RTW_MIXED): at most kMixedChecks evaluations to |s - t| < kMixedTol
constexpr int kMixedChecks = 7;
constexpr double kMixedTol = 3e-6;

// features of row (object o, direction dk): s (3) then the object's 13, in bfloat16
__global__ void learned_features_kernel(const ObjFeat* __restrict__ feat, const double* __restrict__ tab, int nt,
                                        int nph, long long nrows, __nv_bfloat16* __restrict__ X)
{
    const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    const long long ndir = (long long)nt * nph;
    const int o = (int)(row / ndir);
    const long long dk = row - (long long)o * ndir;
    const int it = (int)(dk / nph), jp = (int)(dk % nph);
    const double ct = tab[it], st = tab[nt + it], cp = tab[2 * nt + jp], sp = tab[2 * nt + nph + jp];
    __nv_bfloat16* x = X + row * kMlpIn;
    x[0] = __float2bfloat16_rn((float)(st * cp));
    x[1] = __float2bfloat16_rn((float)(st * sp));
    x[2] = __float2bfloat16_rn((float)ct);
    const ObjFeat& f = feat[o];
#pragma unroll
    for (int k = 0; k < 13; ++k) x[3 + k] = __float2bfloat16_rn(f.f[k]);
}

// one thread per row: heads of network p -> Newton -> deduplicated roots -> F e^{i Psi}; kMixed: a
// first approach on the single-precision trace (its own instantiation, so that the double-precision
// form keeps its registers)
template <bool kMixed>
__global__ void __launch_bounds__(128) learned_newton_kernel(const ObjDev* __restrict__ objs,
                                                             const ObjFeat* __restrict__ feat,
                                                             const double* __restrict__ tab, int nt, int nph,
                                                             long long nrows, const float* __restrict__ Y, int p,
                                                             float p_min, int max_steps, double tol, int max_halvings,
                                                             int nout, double* __restrict__ out,
                                                             unsigned int* __restrict__ mask,
                                                             uint8_t* __restrict__ roots, int np)
{
    const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    const long long ndir = (long long)nt * nph;
    const int oi = (int)(row / ndir);
    const long long dk = row - (long long)oi * ndir;
    const int it = (int)(dk / nph), jp = (int)(dk % nph);
    const double ct = tab[it], st = tab[nt + it], cp = tab[2 * nt + jp], sp = tab[2 * nt + nph + jp];
    const double t[3] = {st * cp, st * sp, ct};
    const double eth[3] = {ct * cp, ct * sp, -st};
    const double eph[3] = {-sp, cp, 0.0};
    const ObjDev& o = objs[oi];
    const ObjFeat& f = feat[oi];
    const float* y = Y + row * kMlpOut;
    float zmax = y[8];
#pragma unroll
    for (int k = 1; k < kMlpHeads; ++k) zmax = fmaxf(zmax, y[8 + k]);
    float w[kMlpHeads], se = 0.0f;
#pragma unroll
    for (int k = 0; k < kMlpHeads; ++k) {
        w[k] = expf(y[8 + k] - zmax);
        se += w[k];
    }
    const double dedup = 1e-6 * o.lmax;
    // default tolerance: the phase error k0 L |s - t| of a converged ray stays below 1e-4 rad
    const double tl = tol > 0.0 ? tol : fmin(1e-6, 1e-4 / (o.k0 * o.lmax));
    double found[kMlpHeads][2];
    int nfound = 0;
    bool uncertain = false;
    double* dst = out + (row * nout + (nout > 1 ? p : 0)) * 4;
    for (int k = 0; k < kMlpHeads; ++k) {
        if (w[k] / se < p_min) continue;
        double u0 = y[2 * k], u1 = y[2 * k + 1];
        // an entry point lies inside the section: seeds beyond radius 0.999 move onto it
        const double ru = sqrt(u0 * u0 + u1 * u1);
        if (ru > 0.999) {
            u0 *= 0.999 / ru;
            u1 *= 0.999 / ru;
        }
        const double d1 = u1 / f.l11, d0 = (u0 - f.l10 * d1) / f.l00;
        double sx = o.c[0] + d0, sy = o.c[1] + d1;
        FarRecord fr;
        double root[2];
        if constexpr (kMixed) {
            // a first approach on the single-precision trace, then the double-precision steps
            if (newton_point<float>(o, p, t, sx, sy, 0.0, fr, kMixedChecks, kMixedTol, root, max_halvings)) {
                sx = root[0];
                sy = root[1];
            }
        }
        if (!newton_point(o, p, t, sx, sy, 0.0, fr, max_steps + 1, tl, root, max_halvings)) {
            uncertain = true;
            continue;
        }
        bool dup = false;
        for (int q = 0; q < nfound; ++q)
            if (hypot(root[0] - found[q][0], root[1] - found[q][1]) <= dedup) dup = true;
        if (dup) continue;
        found[nfound][0] = root[0];
        found[nfound][1] = root[1];
        ++nfound;
        if (fr.flags & kFlagCaustic) {
            atomicOr(mask + row, kMaskCausticL);
            continue;
        }
        add_contribution_reduced(fr.F, fr.psi, eth, eph, dst);
    }
    if (roots) roots[row * np + p] = (uint8_t)nfound | (uncertain ? kRootUncertain : (uint8_t)0);
}

// rows (object, direction) with an uncertain order, counted per object
__global__ void uncertain_count_kernel(const uint8_t* __restrict__ roots, long long nrows, long long ndir, int np,
                                       unsigned int* __restrict__ count)
{
    const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    bool u = false;
    for (int p = 0; p < np; ++p) u = u || (roots[row * np + p] & kRootUncertain);
    if (u) atomicAdd(count + row / ndir, 1u);
}

// (theta, phi) and direction index of every uncertain row of object o
__global__ void uncertain_list_kernel(const uint8_t* __restrict__ roots, int o, int nt, int nph, int np,
                                      double* __restrict__ list, unsigned int* __restrict__ idx,
                                      unsigned int* __restrict__ cursor, unsigned int cap)
{
    const long long ndir = (long long)nt * nph;
    const long long dk = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dk >= ndir) return;
    const long long row = (long long)o * ndir + dk;
    bool u = false;
    for (int p = 0; p < np; ++p) u = u || (roots[row * np + p] & kRootUncertain);
    if (!u) return;
    const unsigned int pos = atomicAdd(cursor, 1u);
    if (pos >= cap) return;
    const int it = (int)(dk / nph), jp = (int)(dk - (long long)it * nph);
    list[2 * pos] = (it + 0.5) * (3.14159265358979323846 / nt);
    list[2 * pos + 1] = -3.14159265358979323846 + (jp + 0.5) * (2.0 * 3.14159265358979323846 / nph);
    idx[pos] = (unsigned int)dk;
}

// the dense values of the uncertain (row, order) entries of object o replace the learned ones
__global__ void uncertain_scatter_kernel(const double* __restrict__ dense, const uint8_t* __restrict__ dmask,
                                         const unsigned int* __restrict__ idx, unsigned int n,
                                         const uint8_t* __restrict__ roots, int o, long long ndir, int np,
                                         double* __restrict__ out, uint8_t* __restrict__ mask_out)
{
    const unsigned int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long dk = idx[k];
    const long long row = (long long)o * ndir + dk;
    for (int p = 0; p < np; ++p) {
        if (!(roots[row * np + p] & kRootUncertain)) continue;
        for (int c = 0; c < 4; ++c) out[(row * np + p) * 4 + c] = dense[((long long)k * np + p) * 4 + c];
    }
    if (mask_out) mask_out[row] |= dmask[k];
}

}  // namespace

cudaError_t launch_learned(const ObjDev* objs, const ObjFeat* feat, const double* tab, int nt, int nph, long long nrows,
                           const MlpWeights* nets, int np, __nv_bfloat16* X, float* Y, float p_min, int max_steps,
                           double tol, int max_halvings, int mixed, int nout, double* out, unsigned int* mask,
                           uint8_t* roots, unsigned int* status, cudaStream_t s)
{
    if (nrows <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((nrows + 127) / 128);
    learned_features_kernel<<<nb, 128, 0, s>>>(feat, tab, nt, nph, nrows, X);
    cudaError_t e = cudaGetLastError();
    for (int p = 0; p < np && e == cudaSuccess; ++p) {
        e = launch_mlp_forward(nets[p], X, nrows, Y, status, s);
        if (e != cudaSuccess) break;
        if (mixed)
            learned_newton_kernel<true><<<nb, 128, 0, s>>>(objs, feat, tab, nt, nph, nrows, Y, p, p_min, max_steps,
                                                            tol, max_halvings, nout, out, mask, roots, np);
        else
            learned_newton_kernel<false><<<nb, 128, 0, s>>>(objs, feat, tab, nt, nph, nrows, Y, p, p_min, max_steps,
                                                             tol, max_halvings, nout, out, mask, roots, np);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace rtw

namespace {

// CS4's fallback: every (object, direction) row where a confident head did not converge is redone by
// the dense path -- the object's square ray grid of fallback_rays[i] rays traced in double precision
// and its field summed on the list of those directions -- and the dense per-order values replace the
// learned ones of the uncertain orders (masks are or-ed).
int dense_fallback(const rtw_object* obj, const rtw_learned_params* lp, const rtw_dirs* dirs, int np, double* out,
                   uint8_t* mask_out, const uint8_t* roots, cudaStream_t s)
{
    const int nt = dirs->n_theta, nph = dirs->n_phi;
    const long long ndir = (long long)nt * nph, nrows = ndir * obj->count;
    unsigned int* count = nullptr;
    RTW_CUDA(cudaMallocAsync(&count, sizeof(unsigned int) * (size_t)(obj->count + 1), s));
    std::vector<unsigned int> hc((size_t)obj->count);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int) * (size_t)(obj->count + 1), s);
    if (e == cudaSuccess) {
        rtw::uncertain_count_kernel<<<(unsigned)((nrows + 255) / 256), 256, 0, s>>>(roots, nrows, ndir, np, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hc.data(), count, sizeof(unsigned int) * hc.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFreeAsync(count, s);
        return rtw::host::cuda_fail(e, "rtw_field_learned: fallback count");
    }
    const unsigned int kmax = hc.empty() ? 0u : *std::max_element(hc.begin(), hc.end());
    int rc = RTW_OK;
    if (kmax > 0) {
        // list, indices, dense values and masks of one object at a time
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t o = off;
            off = align_up(off + bytes, 256);
            return o;
        };
        const size_t o_list = take(sizeof(double) * 2 * kmax), o_idx = take(sizeof(unsigned int) * kmax);
        const size_t o_dense = take(sizeof(double) * 4 * (size_t)np * kmax), o_dmask = take(kmax);
        char* w = nullptr;
        RTW_CUDA(cudaMallocAsync((void**)&w, off, s));
        double* list = (double*)(w + o_list);
        unsigned int* idx = (unsigned int*)(w + o_idx);
        double* dense = (double*)(w + o_dense);
        uint8_t* dmask = (uint8_t*)(w + o_dmask);
        rtw_rays* rays = nullptr;
        for (int i = 0; i < obj->count && rc == RTW_OK; ++i) {
            if (!hc[(size_t)i]) continue;
            e = cudaMemsetAsync(count + obj->count, 0, sizeof(unsigned int), s);
            if (e == cudaSuccess) {
                rtw::uncertain_list_kernel<<<(unsigned)((ndir + 255) / 256), 256, 0, s>>>(
                    roots, i, nt, nph, np, list, idx, count + obj->count, kmax);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) {
                rc = rtw::host::cuda_fail(e, "rtw_field_learned: fallback list");
                break;
            }
            rtw_object one;
            one.count = 1;
            one.device = obj->device;
            one.h.push_back(obj->h[(size_t)i]);
            rtw_trace_params tp{};
            tp.grid = RTW_GRID_SQUARE;
            tp.p_max = np - 1;
            tp.n_rays = lp->fallback_rays[i];
            tp.precision = RTW_FP64;
            rc = rtw_trace(&one, &tp, s, &rays);
            if (rc != RTW_OK) break;
            rtw_dirs ld{};
            ld.kind = RTW_DIRS_LIST;
            ld.list = list;
            ld.n_list = hc[(size_t)i];
            for (int k = 0; k < 4; ++k) ld.cell_window[k] = -1;
            rc = rtw_field(rays, &ld, RTW_DENSE, RTW_FIELD_PER_ORDER, dense, dmask, s);
            if (rc != RTW_OK) break;
            rtw::uncertain_scatter_kernel<<<(hc[(size_t)i] + 255) / 256, 256, 0, s>>>(
                dense, dmask, idx, hc[(size_t)i], roots, i, ndir, np, out, mask_out);
            e = cudaGetLastError();
            if (e != cudaSuccess) rc = rtw::host::cuda_fail(e, "rtw_field_learned: fallback scatter");
        }
        if (rays) {
            cudaStreamSynchronize(s);
            rtw_destroy_rays(rays);
        }
        cudaFreeAsync(w, s);
    }
    cudaFreeAsync(count, s);
    return rc;
}

}  // namespace

extern "C" {

int rtw_field_learned(const rtw_object* obj, const rtw_mlp* m, const rtw_learned_params* lp, const rtw_dirs* dirs,
                      int flags, void* field_out, uint8_t* mask_out, uint8_t* roots_out, void* stream)
{
    if (!obj || !m || !lp || !dirs || !field_out) return fail(RTW_ERR_ARG, "rtw_field_learned: null pointer");
    const int np = lp->p_max + 1;
    if (lp->p_max < 0) return fail(RTW_ERR_ARG, "rtw_field_learned: p_max < 0");
    for (int p = 0; p < np; ++p) {
        int64_t step = 0;
        if (rtw_mlp_get(m, p, nullptr, nullptr, nullptr, &step) != RTW_OK)
            return fail(RTW_ERR_ARG, "rtw_field_learned: no network for order %d", p);
    }
    if (dirs->kind != RTW_DIRS_GRID || dirs->n_theta < 1 || dirs->n_phi < 2)
        return fail(RTW_ERR_ARG, "rtw_field_learned: a (theta, phi) grid with n_theta >= 1, n_phi >= 2");
    if (flags & ~RTW_FIELD_PER_ORDER) return fail(RTW_ERR_ARG, "rtw_field_learned: flags 0x%x", flags);
    if (lp->max_steps < 0 || lp->max_steps > 30 || lp->p_min < 0.0f || lp->p_min > 1.0f || lp->tol < 0.0 ||
        lp->chunk_rows < 0 || lp->max_halvings < 0 || lp->max_halvings > 30)
        return fail(RTW_ERR_ARG, "rtw_field_learned: parameters out of range");
    if (lp->precision != RTW_FP64 && lp->precision != RTW_MIXED)
        return fail(RTW_ERR_ARG, "rtw_field_learned: precision %d (RTW_FP64 or RTW_MIXED)", lp->precision);
    if (lp->fallback_rays && !(flags & RTW_FIELD_PER_ORDER))
        return fail(RTW_ERR_ARG, "rtw_field_learned: the dense fallback needs RTW_FIELD_PER_ORDER");
    if (lp->fallback_rays)
        for (int i = 0; i < obj->count; ++i)
            if (lp->fallback_rays[i] < 1) return fail(RTW_ERR_ARG, "rtw_field_learned: fallback_rays[%d] < 1", i);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    RTW_CUDA(cudaGetDevice(&dev));
    unsigned int* status = rtw::host::status_word(dev);
    if (!status) return fail(RTW_ERR_CUDA, "rtw_field_learned: status word");
    const int max_steps = lp->max_steps > 0 ? lp->max_steps : 3;
    const int max_halvings = lp->max_halvings > 0 ? lp->max_halvings : 3;
    const double tol = lp->tol;  // 0: per object, min(1e-6, 1e-4 / (k0 max(a, b, c)))
    const float p_min = lp->p_min > 0.0f ? lp->p_min : 0.05f;
    const long long ndir = (long long)dirs->n_theta * dirs->n_phi;
    const int nout = (flags & RTW_FIELD_PER_ORDER) ? np : 1;
    const long long chunk_rows = lp->chunk_rows > 0 ? lp->chunk_rows : (1ll << 24);
    const int per_chunk = (int)std::max<long long>(1, std::min<long long>(obj->count, chunk_rows / ndir));
    const long long rows_max = (long long)per_chunk * ndir;

    std::vector<rtw::ObjDev> od((size_t)obj->count);
    std::vector<rtw::ObjFeat> of((size_t)obj->count);
    for (int i = 0; i < obj->count; ++i) {
        if (obj->h[(size_t)i].src) return fail(RTW_ERR_UNSUPPORTED, "rtw_field_learned: plane waves only");
        if (obj->h[(size_t)i].shape_e != 1.0) return fail(RTW_ERR_UNSUPPORTED, "rtw_field_learned: ellipsoids only");
        rtw::host::fill_objdev(obj->h[(size_t)i], od[(size_t)i]);
        od[(size_t)i].grid = rtw::kGridSquare;
        rtw::host::object_features(obj->h[(size_t)i], of[(size_t)i]);
    }
    std::vector<rtw::MlpWeights> nets((size_t)np);
    for (int p = 0; p < np; ++p) nets[(size_t)p] = rtw::host::mlp_weights(m, p);

    // stream-ordered workspace: tables, features, outputs of one network, mask words
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_obj = take(sizeof(rtw::ObjDev) * od.size());
    const size_t o_feat = take(sizeof(rtw::ObjFeat) * of.size());
    const size_t o_tab = take(sizeof(double) * 4 * ((size_t)dirs->n_theta + (size_t)dirs->n_phi));
    const size_t o_x = take(sizeof(__nv_bfloat16) * rtw::kMlpIn * (size_t)rows_max);
    const size_t o_y = take(sizeof(float) * rtw::kMlpOut * (size_t)rows_max);
    const size_t o_mask = take(sizeof(unsigned int) * (size_t)rows_max);
    // the dense fallback reads the root counts: an internal copy when the caller keeps none
    const size_t o_roots = take(lp->fallback_rays && !roots_out ? (size_t)obj->count * ndir * np : 0);
    void* ws = nullptr;
    RTW_CUDA(cudaMallocAsync(&ws, off, s));
    char* b = (char*)ws;
    rtw::ObjDev* d_obj = (rtw::ObjDev*)(b + o_obj);
    rtw::ObjFeat* d_feat = (rtw::ObjFeat*)(b + o_feat);
    double* tab = (double*)(b + o_tab);
    __nv_bfloat16* X = (__nv_bfloat16*)(b + o_x);
    float* Y = (float*)(b + o_y);
    unsigned int* words = (unsigned int*)(b + o_mask);
    uint8_t* roots = roots_out ? roots_out : (lp->fallback_rays ? (uint8_t*)(b + o_roots) : nullptr);
    int rc = RTW_OK;
    cudaError_t e = cudaMemcpyAsync(d_obj, od.data(), sizeof(rtw::ObjDev) * od.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_feat, of.data(), sizeof(rtw::ObjFeat) * of.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(field_out, 0, sizeof(double) * 4 * (size_t)nout * ndir * obj->count, s);
    if (e == cudaSuccess) e = rtw::launch_dir_tables(dirs->n_theta, dirs->n_phi, tab, s);
    for (int c0 = 0; c0 < obj->count && e == cudaSuccess; c0 += per_chunk) {
        const int cn = std::min(per_chunk, obj->count - c0);
        const long long rows = (long long)cn * ndir;
        e = cudaMemsetAsync(words, 0, sizeof(unsigned int) * (size_t)rows, s);
        if (e != cudaSuccess) break;
        e = rtw::launch_learned(d_obj + c0, d_feat + c0, tab, dirs->n_theta, dirs->n_phi, rows, nets.data(), np, X, Y,
                                p_min, max_steps, tol, max_halvings, lp->precision == RTW_MIXED ? 1 : 0, nout,
                                (double*)field_out + 4 * (size_t)nout * ndir * c0, words,
                                roots ? roots + (size_t)np * ndir * c0 : nullptr, status, s);
        if (e == cudaSuccess && mask_out)
            e = rtw::launch_finalize_mask(words, mask_out + (size_t)ndir * c0, d_obj + c0, cn, ndir, 1, dirs->n_theta,
                                          dirs->n_phi, 0.0, 0.0, s);
    }
    if (e != cudaSuccess) rc = rtw::host::cuda_fail(e, "rtw_field_learned");
    if (rc == RTW_OK && lp->fallback_rays)
        rc = dense_fallback(obj, lp, dirs, np, (double*)field_out, mask_out, roots, s);
    cudaFreeAsync(ws, s);
    return rc;
}

}  // extern "C"
