// rtw_launch.h -- host-side launchers of the librtw kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "rtw_internal.h"

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

struct FieldArgs {
    const ObjDev* d_obj;   // this object's entry of the table
    RaysDev st;
    int pmax;
    int per_order;
    double* out;           // [directions][nout][4]
    unsigned int* mask;    // [directions] scratch words
    unsigned int* status;
};

// message returned by rtw_last_error() on the calling thread
void set_last_error(const char* msg);

// trace
cudaError_t launch_trace(const ObjDev* d_objs, int nobj, RaysDev st, int pmax, bool aux, unsigned int* status,
                         cudaStream_t s);
cudaError_t launch_trace_points(const ObjDev* d_obj, const double* xy, long long n, int pmax, double* s_out,
                                double* F_out, double* psi_out, uint32_t* flags_out, cudaStream_t s);
cudaError_t launch_export(RaysDev st, int order, long long first, long long count, double* s_out, double* F_out,
                          double* psi_out, uint32_t* flags_out, cudaStream_t s);

// field
cudaError_t launch_dir_tables(int nt, int nph, double* tab, cudaStream_t s);
cudaError_t launch_field_grid(const FieldArgs& a, long long nx, long long ix0, long long ix1, long long iy0,
                              long long iy1, int nt, int nph, const double* tab, unsigned long long* big,
                              unsigned int* nbig, unsigned int big_cap, unsigned long long* hit_tri,
                              unsigned int* hit_dir, unsigned int* nhit, unsigned int hit_cap, int newton,
                              cudaStream_t s);
cudaError_t launch_field_fan(const FieldArgs& a, long long nrays, double fan_phi, int ndir, double alpha0,
                             double dalpha, PoWindow* d_win, int* d_nwin, double2* d_scratch, long long ap_cap, int po,
                             int newton, cudaStream_t s);
cudaError_t launch_finalize_mask(const unsigned int* words, unsigned char* mask_out, long long ndir, int kind,
                                 int nt, int nph, double alpha0, double dalpha, double axial, cudaStream_t s);

}  // namespace rtw
