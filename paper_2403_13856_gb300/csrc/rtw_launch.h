// rtw_launch.h -- host-side launchers of the librtw kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "rtw_internal.h"
#include "rtw_mlp.cuh"

namespace rtw {

// Per-window data of the physical-optics integral around one in-plane fold of a fan.
struct PoWindow {
    int p;            // order
    int ok;           // 1 when the aperture field is usable
    long long jc;     // fold ray (local index)
    long long jlo, jhi;
    double alpha_c;   // in-plane exit angle of the fold ray
    double sc[3];     // fold ray direction (aperture normal)
};
constexpr int kMaxPoWindows = 64;

// cells of one object in a square-grid field launch
struct GridCells {
    long long ix0, iy0, ncx, ncy;  // cell window of the object's ray grid
    long long first;               // first launch thread of this object (prefix of ncx ncy np)
};

struct GridBatch {
    const GridCells* cells;  // device, nobj entries
    int nobj;
    long long total;         // threads of the launch
    long long ndir;          // directions per object
    int nout;                // (F_theta, F_phi) pairs per direction: orders or 1
};

// Directions of a square-grid field: the cell-centred (theta, phi) grid, or a list binned on a
// (theta, phi) grid of bins (then nt x nph are the bins and each bin lists its directions).
struct DirSet {
    int nt, nph;             // direction grid, or bin grid of a list
    const double* tab;       // cos theta, sin theta, cos phi, sin phi of the (bin) grid, then float copies
    int list;                // 1: the directions come from a list
    long long ndir;          // grid: nt nph; list: its length
    const int* bin_first;    // list: first entry of every bin (nt nph + 1)
    const int* bin_dir;      // list: direction indices, bin after bin
    const double* ldir;      // list: cos theta, sin theta, cos phi, sin phi per direction
    const float4* ldir_f;    // list: unit vector (x, y, z, 0) in single precision
    const double* lsrc;      // list: the caller's (theta, phi) pairs
    float pad;               // list: angular radius of a bin (widens the candidate cap)
};

struct CellRef {
    const ObjDev* o;
    int orel;  // object within the launch
    int p;
    long long cx, cy, base, nx;
};

struct FieldArgs {
    const ObjDev* d_obj;   // the launch's first object in the table (grid fields: objects follow)
    RaysDev st;
    int pmax;
    int per_order;
    double* out;           // [directions][nout][4]
    unsigned int* mask;    // [directions] scratch words
    unsigned int* status;  // error bits (may be null where no kernel of the launch can raise one)
    unsigned long long* nfail;  // Newton refinements that did not converge (may be null without Newton)
};

// message returned by rtw_last_error() on the calling thread
void set_last_error(const char* msg);

// trace; super_shapes: the object set holds superellipsoids (double precision)
cudaError_t launch_trace(const ObjDev* d_objs, int nobj, RaysDev st, int pmax, bool aux, unsigned int* status,
                         cudaStream_t s, bool super_shapes = false);
// persistent batched trace over work items; variant 1..kTraceVariants picks the block size and
// register cap: 1 (64, 1), 2 (128, 1), 3 (256, 1), 4 (128, 3 CTAs/SM), 5 (256, 2 CTAs/SM)
constexpr int kTraceVariants = 5;
cudaError_t launch_trace_items(const ObjDev* d_objs, int nobj, RaysDev st, int pmax, unsigned long long* next,
                               long long nitems, int variant, int ctas_per_sm, cudaStream_t s);
cudaError_t launch_trace_points(const ObjDev* d_obj, const double* xy, long long n, int pmax, double* s_out,
                                double* F_out, double* psi_out, uint32_t* flags_out, cudaStream_t s);
cudaError_t launch_export(RaysDev st, int order, long long first, long long count, double* s_out, double* F_out,
                          double* psi_out, uint32_t* flags_out, cudaStream_t s);

// field
cudaError_t launch_dir_tables(int nt, int nph, double* tab, cudaStream_t s);
// The square-grid field of one launch: classification of the cell triangles into (triangle,
// direction) hits, then their sum.  Without Newton refinement and with fmax (RaysDev::fmax of the
// launch's first object), every hit adds its contribution as 64-bit fixed-point integers: the output
// words then hold integers until launch_field_convert (once per launch group, after every slice).
// Otherwise every hit adds its doubles with atomics.
cudaError_t launch_field_grid(const FieldArgs& a, const GridBatch& b, const DirSet& d, unsigned long long* big,
                              unsigned int* nbig, unsigned int big_cap, unsigned long long* hit_tri,
                              unsigned int* hit_dir, unsigned int* nhit, unsigned int hit_cap, int classify_block,
                              int newton, cudaStream_t s, int stage = 0, const unsigned int* fmax = nullptr);
// fixed-point output words of nobj objects (per_obj words each) to doubles, in place
cudaError_t launch_field_convert(double* out, long long per_obj, int nobj, const unsigned int* fmax, cudaStream_t s);
// 2-D physical optics over a window of grid vertices [win0, win1] x [win2, win3] of one square-grid
// object (nx vertices per row; rays traced with the aperture data): plane through c with normal axis,
// rays weighted by the angle of their exit direction to it (1 up to cone_full, 0 from cone_end);
// dirs: ndir (theta, phi) pairs on the device; out: ndir x (F_theta, F_phi).  scratch holds
// po2d_scratch_bytes(window vertices, ndir) bytes.
size_t po2d_scratch_bytes(long long nwin, long long ndir);
cudaError_t launch_po2d(const RaysDev& st, int order, long long nx, const long long win[4], const double c[3],
                        const double axis[3], double k0, double cone_full, double cone_end, const double* dirs,
                        long long ndir, double2* out, void* scratch, cudaStream_t s);
// stage of launch_field_grid: 0 classifies the triangles and sums their hits; 1 only classifies
// (*nhit then holds the number of pairs the batch wants, which may exceed hit_cap); 2 sums the hits
// of a stage-1 run that fitted
enum { kFieldAll = 0, kFieldClassify = 1, kFieldSum = 2 };
// bins a direction list: unit vectors, bin of every direction, bin offsets and bin lists;
// count and cursor hold nt nph + 1 ints each
cudaError_t launch_bin_dirs(const double* list, long long n, int nt, int nph, double* ldir, float4* ldir_f,
                            int* binid, int* count, int* first, int* cursor, int* bin_dir, cudaStream_t s);
cudaError_t launch_field_fan(const FieldArgs& a, long long nrays, double fan_phi, int ndir, double alpha0,
                             double dalpha, PoWindow* d_win, int* d_nwin, double2* d_scratch, long long ap_cap, int po,
                             int newton, cudaStream_t s);
// learned proposal (rtw_mlp.cu; the inference forward pass is rtw_mlp_tc.cu)
cudaError_t mlp_prepare_kernels();
cudaError_t mlp_prepare_tc_kernel();
// the tensor-core inference kernel's hidden activation (GELU in single precision, before its bfloat16
// rounding) on n values
cudaError_t launch_activation_eval(const float* x, float* y, long long n, cudaStream_t s);
// X (rows x 16 bf16) and Y (rows x 16 f32) 16-byte aligned; a bounded wait that gives up sets the
// timeout bit of *status
cudaError_t launch_mlp_forward(const MlpWeights& w, const __nv_bfloat16* X, long long rows, float* Y,
                               unsigned int* status, cudaStream_t s);
// the tensor-core training passes (rtw_mlp_tc.cu): forward with the hidden layers' Z and H kept in
// acts (Y into acts.y); backward data pass from acts.dyb to acts.dz3, dz2, dz1; weight gradients of
// chunks of rows into part[chunk] (returns the number of chunks, *err the launch status)
cudaError_t launch_mlp_train_tc(const MlpWeights& w, const __nv_bfloat16* X, long long rows, const MlpActs& acts,
                                unsigned int* status, cudaStream_t s);
cudaError_t launch_mlp_backward_tc(const MlpWeights& w, long long rows, const MlpActs& acts, unsigned int* status,
                                   cudaStream_t s);
int launch_mlp_wgrad_tc(const __nv_bfloat16* X, long long rows, const MlpActs& acts, float* part, unsigned int* status,
                        cudaStream_t s, cudaError_t* err);
// forward with stored activations, loss, backward and weight gradients of one batch into grad, all
// products on the tensor cores; part holds ceil(rows / 512) x kMlpParams floats; X 16-byte aligned
cudaError_t launch_mlp_grad(const MlpWeights& w, const __nv_bfloat16* X, const float* T, const uint8_t* valid,
                            long long rows, float beta, const MlpActs& acts, float* part, float* grad,
                            unsigned int* status, cudaStream_t s);
cudaError_t launch_mlp_adam(float* theta, float* m, float* v, const float* grad, int update, float lr, float b1,
                            float b2, float eps, float c1, float c2, __nv_bfloat16* w1, __nv_bfloat16* w2,
                            __nv_bfloat16* w3, __nv_bfloat16* w4, __nv_bfloat16* w2t, __nv_bfloat16* w3t,
                            __nv_bfloat16* w4t, cudaStream_t s);
cudaError_t launch_mlp_samples(const ObjDev* objs, const ObjFeat* feat, int nobj, const double* uv, const int* oidx,
                               long long n, int pmax, __nv_bfloat16* X, float* T, uint8_t* valid, cudaStream_t s);

// learned field (rtw_learned.cu): features of nrows (object, direction) rows, then per order the
// network's forward pass and the Newton kernel
cudaError_t launch_learned(const ObjDev* objs, const ObjFeat* feat, const double* tab, int nt, int nph, long long nrows,
                           const MlpWeights* nets, int np, __nv_bfloat16* X, float* Y, float p_min, int max_steps,
                           double tol, int max_halvings, int mixed, int nout, double* out, unsigned int* mask,
                           uint8_t* roots, unsigned int* status, cudaStream_t s);

cudaError_t launch_grid_cells(const ObjDev* objs, int n, int np, bool windowed, const int64_t* win, GridCells* cells,
                              cudaStream_t s);
// kind 0: plane angles alpha0 + k dalpha; 1: (theta, phi) grid nt x nph; 2: list of (theta, phi) pairs
cudaError_t launch_finalize_mask(const unsigned int* words, unsigned char* mask_out, const ObjDev* objs, int nobj,
                                 long long ndir, int kind, int nt, int nph, double alpha0, double dalpha,
                                 cudaStream_t s, const double* list = nullptr);

// 2-D physical optics at the caustics of a square-grid field (rtw_caustic.cu): scratch bytes for
// ndir directions, ntiles tiles and nblocks 16 x 16 ray blocks; one order's correction of the
// per-order field ([directions][np][4]) and mask words (the caustic bit of the order cleared where its
// weight is 1, RTW_MASK_PO set where it is above 0); then bit 0 of the words from the order bits left,
// and (out not null) the sum over the orders into out ([directions][4])
size_t caustic_scratch_bytes(long long ndir, long long ntiles, long long nblocks);
cudaError_t launch_caustic_order(const RaysDev& st, const ObjDev& o, int order, int nt, int nph, int tt, int tp,
                                 double po_full, double po_end, double cone_full, double cone_end, unsigned int* words,
                                 double* field, double* weights, void* scratch, cudaStream_t s);
cudaError_t launch_caustic_finish(unsigned int* words, long long ndir, const double* per_order, double* out, int np,
                                  cudaStream_t s);

}  // namespace rtw
