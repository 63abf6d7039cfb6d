// rtw_host.h -- host-side helpers shared by the C-ABI translation units of librtw (internal).
//
// Object descriptions in double precision, error reporting, the per-device status word, the ray
// grid of an object, and the square-grid field run in launch groups of objects that both
// rtw_field and the batched entry point use.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <utility>
#include <vector>

#include "rtw.h"
#include "rtw_launch.h"

namespace rtw {
namespace host {

// One ellipsoid (or superellipsoid) and its incident wave, in double precision: semi-axes,
// rotation (body to lab), centre, index, wavelength, Jones vector, quadric matrix
// W = R diag(1/a^2) R^T, the projected ellipse S (x^T S x <= 1 on z = const; of the bounding
// ellipsoid for a superellipsoid) and its inverse, smallest and largest semi-axis.
struct ObjHost {
    double a[3];
    double R[3][3];
    double c[3];
    double m;
    double lambda;
    double jre[2], jim[2];
    double W[3][3];
    double S[2][2], Sinv[2][2];  // rays that hit: (w - gc)^T S (w - gc) < 1 on the grid's plane
    double lmin, lmax;
    double gc[2];                 // centre of the ray grid (plane wave: c_x, c_y)
    int src;                      // 1: point source
    double src_pos[3], e1[3], e2[3];
    double shape_e;               // superellipsoid exponent (1: the ellipsoid)
};

// sets the calling thread's last-error message and returns code
int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int cuda_fail(cudaError_t e, const char* what);
// device word of error bits raised by kernels (allocated once per device)
unsigned int* status_word(int dev);
// device counter of Newton refinements that did not converge (next to the status word)
unsigned long long* newton_counter(int dev);
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void fill_objdev(const ObjHost& o, ObjDev& d);
// validates one object description and its incident wave and fills o (host arithmetic only, no
// device call); i numbers the object in error messages
int make_object_host(const rtw_object_desc& d, const rtw_incident& w, int i, ObjHost& o);
// the device table entry of o for the ray grid of tp, its rays starting at ray_offset
int object_device_entry(const ObjHost& o, const rtw_trace_params* tp, long long ray_offset, ObjDev& d);
// ray grid of one object: spacing, size, fan half-width (host arithmetic only)
int grid_of(const ObjHost& o, const rtw_trace_params* tp, double* h, long long* nx, long long* ny, double* fan_w);

// number of directions of a (theta, phi) grid or list; the (bin) grid the kernels walk
long long dir_count(const rtw_dirs* dirs);
void dir_grid(const rtw_dirs* dirs, int* nt, int* nph);
// validates a (theta, phi) grid or list for a square-grid field (window allowed or not)
int check_grid_dirs(const rtw_dirs* dirs, bool window_allowed, const char* who);

// Launch groups of a square-grid field: objects [k group, (k+1) group) share one launch sequence;
// the group size is bounded by the hit list (4 (triangle, direction) pairs per direction and order
// of each object, at most 2^28 pairs).
struct GridPlan {
    int group = 1;
    long long max_group_cells = 0;  // cells x orders of the largest group
    bool windowed = false;
    bool super_shapes = false;      // the objects include superellipsoids
    bool sliced = false;            // run in row slices sized to the hit list (grid_field_run)
};
GridPlan plan_grid(const ObjDev* objs, int nobj, int np, const rtw_dirs* dirs);

// Grid-field workspace carved from one device block.
struct GridWs {
    unsigned int* mask_words = nullptr;  // group x directions
    double* tab = nullptr;               // tables of the direction (or bin) grid
    GridCells* cells = nullptr;          // group entries
    // direction lists: per-direction unit vectors and bins, bin offsets and lists
    double* ldir = nullptr;
    float4* ldir_f = nullptr;
    int* binid = nullptr;
    int* count = nullptr;
    int* first = nullptr;
    int* cursor = nullptr;
    int* bin_dir = nullptr;
    unsigned long long* big = nullptr;
    unsigned int* nbig = nullptr;
    unsigned int* nhit = nullptr;
    unsigned long long* hit_tri = nullptr;
    unsigned int* hit_dir = nullptr;
    unsigned int big_cap = 0, hit_cap = 0;
};
// Bytes of the workspace of plan g; carves it from base when base is not null.
size_t grid_ws(const GridPlan& g, int np, const rtw_dirs* dirs, char* base, GridWs* w);

// Fills the direction tables (and bins a list) in w; d describes the directions to the kernels.
int dirs_prepare(const rtw_dirs* dirs, const GridWs& w, DirSet* d, cudaStream_t s);

// Field of objects [0, nobj) of ray state st on the (theta, phi) grid or list of dirs (d from
// dirs_prepare on the same stream).  h_objs and d_objs
// are the same table on the host and the device.  Adds into out, which the caller cleared:
// [objects][directions][nout][4] doubles.  mask_out (may be null): [objects][directions] bytes.
// newton = 1 replaces every interpolated hit by the exact ray found by Newton steps.
// With superellipsoids (the number of ray branches per direction grows quickly with the order) or
// direction grids too fine for the hit list (g.sliced), each group is run in slices of ray-grid rows: a slice is classified, the count of
// (triangle, direction) pairs it wants is read back (the stream is synchronised), and a slice that
// does not fit the hit list is split by its count before any of its hits is summed.  slices
// (optional, in and out): row slices to start from when they cover the run's rows (else the whole
// grid); receives the slices that fitted, so that the next run on the same rays and directions
// takes them directly.  Without Newton refinement, on rays that keep their amplitude bound
// (RaysDev::fmax), the hits are summed per output tile in 64-bit fixed point (the same field bit
// for bit from run to run) and turned into doubles once a group is complete.
int grid_field_run(const ObjDev* h_objs, const ObjDev* d_objs, int nobj, const RaysDev& st, const GridPlan& g,
                   const rtw_dirs* dirs, const DirSet& d, bool per_order, double* out, unsigned char* mask_out,
                   const GridWs& w, int classify_block, int newton, unsigned int* status, unsigned long long* nfail,
                   cudaStream_t s, std::vector<std::pair<long long, long long>>* slices = nullptr);

// per-object feature table of the learned proposal
void object_features(const ObjHost& o, ObjFeat& f);
// bf16 weights of the network of one order
MlpWeights mlp_weights(const rtw_mlp* m, int order);

}  // namespace host
}  // namespace rtw

struct rtw_object {
    int count = 0;
    int device = 0;
    std::vector<rtw::host::ObjHost> h;
};

#define RTW_CUDA(call)                                                    \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return rtw::host::cuda_fail(e_, #call);    \
    } while (0)
