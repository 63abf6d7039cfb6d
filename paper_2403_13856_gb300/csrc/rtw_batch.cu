// rtw_batch.cu -- host side of rtw_far_field_batch: many ellipsoids, each with its own wave and
// square ray grid, traced and summed onto one (theta, phi) grid in a single launch sequence.
//
// Plan.  Objects are split, in order, into chunks whose ray state ((ray, order) pairs times 116
// bytes) fits the chunk bound.  Per chunk: one persistent trace kernel over work items (object,
// 256 rays), then the square-grid field in launch groups of objects.  The object table carries
// chunk-relative ray offsets and work-item offsets, so a chunk's launches take a slice of it.
// With use_graph the sequence of every chunk is recorded once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "rtw.h"
#include "rtw_host.h"
#include "rtw_launch.h"

using rtw::ObjDev;
using rtw::RaysDev;
using rtw::host::align_up;
using rtw::host::fail;

namespace {

struct Chunk {
    int first = 0, count = 0;  // objects
    long long R = 0;           // rays per order
    long long nitems = 0;      // work items of the trace
    rtw::host::GridPlan plan;
};

// bytes of the ray state of R rays and np orders, and its layout (as rtw_trace)
size_t state_layout(long long R, int np, int nobj, char* base, RaysDev* st)
{
    const size_t n = (size_t)np * (size_t)R;
    const size_t sizes[8] = {n * 16, n * 16, n * 16, n * 16, n * 16, n * 4, n * 64, 4 * (size_t)nobj};
    size_t off[8], total = 0;
    for (int k = 0; k < 8; ++k) {
        off[k] = total;
        total = align_up(total + sizes[k], 256);
    }
    if (base && st) {
        st->R = R;
        st->np = np;
        st->s01 = (double2*)(base + off[0]);
        st->s2psi = (double2*)(base + off[1]);
        st->Fx = (double2*)(base + off[2]);
        st->Fy = (double2*)(base + off[3]);
        st->Fz = (double2*)(base + off[4]);
        st->flags = (uint32_t*)(base + off[5]);
        st->aux = nullptr;
        st->frec = (float4*)(base + off[6]);
        st->fval = (float4*)(base + off[6] + n * 32);
        st->fmax = (unsigned int*)(base + off[7]);
    }
    return total;
}

}  // namespace

struct rtw_batch {
    int device = 0;
    std::vector<ObjDev> objs;
    std::vector<Chunk> chunks;
    rtw::host::GridPlan ws_plan;  // sizes the field workspace for every chunk
    long long total_rays = 0;
    int replayed = 0;
    ObjDev* d_objs = nullptr;
    size_t d_objs_cap = 0;
    void* state = nullptr;
    size_t state_bytes = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // recorded launch sequence and what it was recorded for
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
    // timing events: 3 per chunk (trace start, trace end = field start, field end)
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;

    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};

namespace {

template <typename T>
void put(std::vector<unsigned char>& k, const T& v)
{
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    k.insert(k.end(), p, p + sizeof(T));
}

// enqueues the whole sequence on q (eager or under capture)
int enqueue(rtw_batch* b, const rtw_batch_params* bp, const rtw_dirs* dirs, bool per_order, double* out,
            uint8_t* mask_out, bool timing, cudaStream_t q)
{
    const int np = bp->p_max + 1;
    const long long ndir = rtw::host::dir_count(dirs);
    const int nout = per_order ? np : 1;
    unsigned int* status = rtw::host::status_word(b->device);
    if (!status) return fail(RTW_ERR_CUDA, "rtw_far_field_batch: status word");
    char* ws = (char*)b->ws;
    unsigned long long* counter = (unsigned long long*)ws;
    // one carve for every chunk: the largest group and lists of all chunk plans
    rtw::host::GridWs w;
    rtw::host::grid_ws(b->ws_plan, np, dirs, ws + 256, &w);
    RTW_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 4 * (size_t)nout * (size_t)ndir * b->objs.size(), q));
    rtw::DirSet d;
    int rcd = rtw::host::dirs_prepare(dirs, w, &d, q);
    if (rcd != RTW_OK) return rcd;
    const int variant = bp->trace_variant > 0 ? bp->trace_variant : 2;
    int e = 0;
    for (const Chunk& c : b->chunks) {
        RaysDev st{};
        state_layout(c.R, np, c.count, (char*)b->state, &st);
        st.precision = bp->precision;
        RTW_CUDA(cudaMemsetAsync(st.fmax, 0, 4 * (size_t)c.count, q));
        if (timing) RTW_CUDA(cudaEventRecord(b->ev[(size_t)e++], q));
        RTW_CUDA(rtw::launch_trace_items(b->d_objs + c.first, c.count, st, bp->p_max, counter, c.nitems, variant,
                                         bp->trace_ctas_per_sm, q));
        if (timing) RTW_CUDA(cudaEventRecord(b->ev[(size_t)e++], q));
        int rc = rtw::host::grid_field_run(b->objs.data() + c.first, b->d_objs + c.first, c.count, st, c.plan, dirs,
                                           d, per_order, out + 4 * (size_t)nout * (size_t)ndir * (size_t)c.first,
                                           mask_out ? mask_out + (size_t)ndir * (size_t)c.first : nullptr, w,
                                           bp->classify_block, bp->mode == RTW_NEWTON ? 1 : 0, status,
                                           rtw::host::newton_counter(b->device), q);
        if (rc != RTW_OK) return rc;
        if (timing) RTW_CUDA(cudaEventRecord(b->ev[(size_t)e++], q));
    }
    b->ev_used = e;
    return RTW_OK;
}

}  // namespace

extern "C" {

int rtw_far_field_batch(const rtw_object* obj, const rtw_batch_params* bp, const rtw_dirs* dirs, int flags,
                        void* field_out, uint8_t* mask_out, rtw_batch** inout, void* stream)
{
    if (!obj || !bp || !dirs || !field_out || !inout || !bp->n_rays)
        return fail(RTW_ERR_ARG, "rtw_far_field_batch: null pointer");
    if (bp->p_max < 0 || bp->p_max >= rtw::kMaxOrders)
        return fail(RTW_ERR_ARG, "rtw_far_field_batch: p_max out of [0, 15]");
    if (bp->precision != RTW_FP64 && bp->precision != RTW_MIXED && bp->precision != RTW_DFLOAT)
        return fail(RTW_ERR_ARG, "rtw_far_field_batch: precision %d", bp->precision);
    if (flags & ~RTW_FIELD_PER_ORDER) return fail(RTW_ERR_ARG, "rtw_far_field_batch: flags 0x%x", flags);
    {
        int rcd = rtw::host::check_grid_dirs(dirs, false, "rtw_far_field_batch");
        if (rcd != RTW_OK) return rcd;
    }
    if (bp->trace_variant < 0 || bp->trace_variant > rtw::kTraceVariants)
        return fail(RTW_ERR_ARG, "rtw_far_field_batch: trace_variant %d", bp->trace_variant);
    if (bp->classify_block != 0 && bp->classify_block != 64 && bp->classify_block != 128 && bp->classify_block != 256)
        return fail(RTW_ERR_ARG, "rtw_far_field_batch: classify_block %d", bp->classify_block);
    if (bp->mode != RTW_DENSE && bp->mode != RTW_NEWTON)
        return fail(RTW_ERR_ARG, "rtw_far_field_batch: mode %d", bp->mode);
    if (bp->chunk_ray_orders < 0 || bp->trace_ctas_per_sm < 0)
        return fail(RTW_ERR_ARG, "rtw_far_field_batch: negative chunk bound or CTAs per SM");
    cudaStream_t s = (cudaStream_t)stream;
    const int np = bp->p_max + 1;
    const bool per_order = (flags & RTW_FIELD_PER_ORDER) != 0;

    // object table, chunks and work items (host arithmetic only)
    std::vector<ObjDev> objs((size_t)obj->count);
    std::vector<Chunk> chunks;
    const long long bound = bp->chunk_ray_orders > 0 ? bp->chunk_ray_orders : (1ll << 29);
    long long total = 0;
    rtw_trace_params tp{};
    tp.grid = RTW_GRID_SQUARE;
    tp.p_max = bp->p_max;
    tp.precision = bp->precision;
    for (int i = 0; i < obj->count; ++i) {
        if (bp->n_rays[i] < 1) return fail(RTW_ERR_ARG, "rtw_far_field_batch: n_rays[%d] < 1", i);
        tp.n_rays = bp->n_rays[i];
        double h = 0.0, fw = 0.0;
        long long nx = 0, ny = 0;
        if (obj->h[(size_t)i].src) return fail(RTW_ERR_UNSUPPORTED, "rtw_far_field_batch: plane waves only");
        if (obj->h[(size_t)i].shape_e != 1.0)
            return fail(RTW_ERR_UNSUPPORTED, "rtw_far_field_batch: ellipsoids only (superellipsoids: rtw_trace)");
        int rc = rtw::host::grid_of(obj->h[(size_t)i], &tp, &h, &nx, &ny, &fw);
        if (rc != RTW_OK) return rc;
        ObjDev& d = objs[(size_t)i];
        rtw::host::fill_objdev(obj->h[(size_t)i], d);
        d.grid = rtw::kGridSquare;
        d.h = h;
        d.nx = nx;
        d.ny = ny;
        const long long nr = nx * ny;
        if (chunks.empty() || (chunks.back().R + nr) * np > bound) {
            chunks.push_back(Chunk{});
            chunks.back().first = i;
        }
        Chunk& c = chunks.back();
        d.ray_offset = c.R;
        d.item_first = c.nitems;
        c.R += nr;
        c.nitems += (nr + rtw::kRaysPerItem - 1) / rtw::kRaysPerItem;
        c.count += 1;
        total += nr;
    }
    size_t state_bytes = 0;
    rtw::host::GridPlan ws_plan;
    ws_plan.group = 1;
    for (Chunk& c : chunks) {
        c.plan = rtw::host::plan_grid(objs.data() + c.first, c.count, np, dirs);
        state_bytes = std::max(state_bytes, state_layout(c.R, np, c.count, nullptr, nullptr));
        ws_plan.group = std::max(ws_plan.group, c.plan.group);
        ws_plan.max_group_cells = std::max(ws_plan.max_group_cells, c.plan.max_group_cells);
    }
    const size_t ws_bytes = 256 + rtw::host::grid_ws(ws_plan, np, dirs, nullptr, nullptr);

    rtw_batch* b = *inout;
    if (!b) {
        b = new (std::nothrow) rtw_batch();
        if (!b) return fail(RTW_ERR_NOMEM, "rtw_far_field_batch: host allocation");
        *inout = b;
        RTW_CUDA(cudaGetDevice(&b->device));
    }
    int dev = 0;
    RTW_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(RTW_ERR_ARG, "rtw_far_field_batch: handle belongs to device %d", b->device);

    // what a recorded graph depends on
    std::vector<unsigned char> key;
    key.reserve(objs.size() * sizeof(ObjDev) + 128);
    for (const ObjDev& o : objs) put(key, o);
    put(key, bp->p_max);
    put(key, bp->precision);
    put(key, bound);
    put(key, bp->trace_variant);
    put(key, bp->trace_ctas_per_sm);
    put(key, bp->classify_block);
    put(key, bp->mode);
    put(key, dirs->kind);
    put(key, dirs->n_theta);
    put(key, dirs->n_phi);
    put(key, dirs->list);
    put(key, dirs->n_list);
    put(key, flags);
    put(key, field_out);
    put(key, mask_out);
    b->replayed = 0;
    if (bp->use_graph && b->exec && key == b->key) {
        RTW_CUDA(cudaGraphLaunch(b->exec, s));
        b->replayed = 1;
        return RTW_OK;
    }
    b->drop_graph();

    // device memory: object table, ray state of the largest chunk, workspace
    if (b->d_objs_cap < objs.size()) {
        if (b->d_objs) cudaFree(b->d_objs);
        b->d_objs = nullptr;
        b->d_objs_cap = 0;
        if (cudaMalloc(&b->d_objs, sizeof(ObjDev) * objs.size()) != cudaSuccess)
            return fail(RTW_ERR_NOMEM, "rtw_far_field_batch: object table");
        b->d_objs_cap = objs.size();
    }
    if (b->state_bytes < state_bytes) {
        if (b->state) cudaFree(b->state);
        b->state = nullptr;
        b->state_bytes = 0;
        if (cudaMalloc(&b->state, state_bytes) != cudaSuccess)
            return fail(RTW_ERR_NOMEM, "rtw_far_field_batch: ray state of %zu bytes", state_bytes);
        b->state_bytes = state_bytes;
    }
    if (b->ws_bytes < ws_bytes) {
        if (b->ws) cudaFree(b->ws);
        b->ws = nullptr;
        b->ws_bytes = 0;
        if (cudaMalloc(&b->ws, ws_bytes) != cudaSuccess)
            return fail(RTW_ERR_NOMEM, "rtw_far_field_batch: workspace of %zu bytes", ws_bytes);
        b->ws_bytes = ws_bytes;
    }
    b->objs = std::move(objs);
    b->chunks = std::move(chunks);
    b->ws_plan = ws_plan;
    b->total_rays = total;
    // the table is copied from pageable memory: the copy has left b->objs when the call returns
    RTW_CUDA(cudaMemcpyAsync(b->d_objs, b->objs.data(), sizeof(ObjDev) * b->objs.size(), cudaMemcpyHostToDevice, s));

    if (!bp->use_graph) {
        if (bp->timing) {
            const size_t need = 3 * b->chunks.size();
            while (b->ev.size() < need) {
                cudaEvent_t e;
                RTW_CUDA(cudaEventCreate(&e));
                b->ev.push_back(e);
            }
        }
        b->ev_used = 0;
        return enqueue(b, bp, dirs, per_order, (double*)field_out, mask_out, bp->timing != 0, s);
    }
    if (!b->cap_stream) RTW_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    RTW_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(b, bp, dirs, per_order, (double*)field_out, mask_out, false, b->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc != RTW_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return rtw::host::cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        b->exec = nullptr;
        return rtw::host::cuda_fail(ce, "cudaGraphInstantiate");
    }
    b->key = std::move(key);
    b->ev_used = 0;
    RTW_CUDA(cudaGraphLaunch(b->exec, s));
    return RTW_OK;
}

int rtw_batch_info(const rtw_batch* b, int64_t* total_rays, int* n_chunks, int* replayed)
{
    if (!b) return fail(RTW_ERR_ARG, "rtw_batch_info: null handle");
    if (total_rays) *total_rays = b->total_rays;
    if (n_chunks) *n_chunks = (int)b->chunks.size();
    if (replayed) *replayed = b->replayed;
    return RTW_OK;
}

int rtw_batch_times(const rtw_batch* b, double* trace_ms, double* field_ms)
{
    if (!b) return fail(RTW_ERR_ARG, "rtw_batch_times: null handle");
    if (b->ev_used == 0) return fail(RTW_ERR_ARG, "rtw_batch_times: the last call recorded no timing events");
    RTW_CUDA(cudaEventSynchronize(b->ev[(size_t)b->ev_used - 1]));
    double t = 0.0, f = 0.0;
    for (int k = 0; k + 2 < b->ev_used; k += 3) {
        float a = 0.0f, c = 0.0f;
        RTW_CUDA(cudaEventElapsedTime(&a, b->ev[(size_t)k], b->ev[(size_t)k + 1]));
        RTW_CUDA(cudaEventElapsedTime(&c, b->ev[(size_t)k + 1], b->ev[(size_t)k + 2]));
        t += a;
        f += c;
    }
    if (trace_ms) *trace_ms = t;
    if (field_ms) *field_ms = f;
    return RTW_OK;
}

void rtw_destroy_batch(rtw_batch* b)
{
    if (!b) return;
    b->drop_graph();
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->d_objs) cudaFree(b->d_objs);
    if (b->state) cudaFree(b->state);
    if (b->ws) cudaFree(b->ws);
    delete b;
}

}  // extern "C"
