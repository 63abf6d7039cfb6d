// rtw_static.cu -- rtw_fan_field_static: the fan trace and far field without any allocation.
//
// Some programs that embed this library may not allocate device memory themselves: a host
// application whose memory manager owns the whole device and forbids direct cudaMalloc calls from
// plug-ins, or a control loop that must never block on the implicit device synchronisation an
// allocation can bring.  For them this entry point runs the 1-D fan path (trace of every ray and
// order, then the interpolated far field and its mask) entirely in caller buffers plus one
// fixed-size scratch array that lives in the library's device image.
//
// The scratch array below is a file-scope __device__ symbol.  On the host its name only stands for
// the symbol; the device address is looked up with cudaGetSymbolAddress, once per device, with that
// device current, on the first call made on it.  Every call on a device shares the array and leaves
// its contents behind, so each call clears what has to start at zero; calls whose work overlaps on
// the GPU (other streams, other host threads) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "rtw.h"
#include "rtw_host.h"
#include "rtw_launch.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// Limits of the scratch: rays times orders of the fan, and observation directions.
constexpr long long kStaticRayOrders = 65536;
constexpr long long kStaticDirs = 65536;
// layout: object entry | ray state (s01, s2psi, Fx, Fy, Fz: 16 B each; flags: 4 B) | mask words
constexpr size_t kObjBytes = 512;
constexpr size_t kStateBytes = (size_t)kStaticRayOrders * (5 * 16 + 4);
constexpr size_t kMaskBytes = (size_t)kStaticDirs * 4;
constexpr size_t kScratchBytes = kObjBytes + kStateBytes + kMaskBytes + 256;

static __device__ __align__(256) unsigned char g_rtw_static_scratch[kScratchBytes];

__global__ void put_object_kernel(rtw::ObjDev o)
{
    // device code may name the array directly
    *reinterpret_cast<rtw::ObjDev*>(g_rtw_static_scratch) = o;
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

int set_error(int code, const char* msg)
{
    rtw::set_last_error(msg);  // reported by rtw_last_error()
    return code;
}

// device address of the scratch array for the current device (looked up once per device)
int scratch_address(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(RTW_ERR_CUDA, "no current CUDA device");
    if (dev < 0 || dev >= kMaxDevices) return set_error(RTW_ERR_UNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rtw_static_scratch);
        if (e != cudaSuccess || !p) return set_error(RTW_ERR_CUDA, cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return RTW_OK;
}

}  // namespace

extern "C" int rtw_fan_field_static(const rtw_object_desc* d, const rtw_incident* w, const rtw_trace_params* tp,
                                    const rtw_dirs* dirs, int flags, void* field_out, uint8_t* mask_out,
                                    void* stream)
{
    if (!d || !w || !tp || !dirs || !field_out) return set_error(RTW_ERR_ARG, "null pointer");
    if (tp->grid != RTW_GRID_FAN || dirs->kind != RTW_DIRS_PLANE)
        return set_error(RTW_ERR_ARG, "needs a fan grid and in-plane directions");
    if (tp->precision != RTW_FP64) return set_error(RTW_ERR_UNSUPPORTED, "FP64 only");
    if (tp->observe_radius != 0.0) return set_error(RTW_ERR_ARG, "far field only (observe_radius 0)");
    if ((flags & ~RTW_FIELD_PER_ORDER) != 0) return set_error(RTW_ERR_UNSUPPORTED, "only RTW_FIELD_PER_ORDER");
    if (tp->p_max < 0 || tp->p_max >= rtw::kMaxOrders) return set_error(RTW_ERR_ARG, "p_max out of [0, 15]");
    if (tp->n_rays < 2) return set_error(RTW_ERR_ARG, "fan needs n_rays >= 2");
    const int np = tp->p_max + 1;
    if (tp->n_rays * np > kStaticRayOrders)
        return set_error(RTW_ERR_CAPACITY, "n_rays * (p_max + 1) exceeds the static scratch limit of 65536");
    if (dirs->n_theta < 1 || dirs->n_theta > kStaticDirs)
        return set_error(RTW_ERR_CAPACITY, "direction count outside [1, 65536]");
    if (!(std::fabs(dirs->dalpha) > 0.0) || std::fabs(dirs->dalpha) > 0.5 ||
        std::fabs(dirs->dalpha) * dirs->n_theta > 2.0 * kPi + 1e-9)
        return set_error(RTW_ERR_ARG, "plane grid needs 0 < |dalpha| <= 0.5 and a span <= 2 pi");
    // object validation and tables: the same host helpers as rtw_create_object and rtw_trace
    if (w->kind != RTW_INCIDENT_PLANE) return set_error(RTW_ERR_UNSUPPORTED, "plane waves only");
    if (d->shape_e != 0.0 && d->shape_e != 1.0) return set_error(RTW_ERR_UNSUPPORTED, "ellipsoids only");
    rtw::host::ObjHost oh;
    int rc = rtw::host::make_object_host(*d, *w, 0, oh);
    if (rc != RTW_OK) return rc;
    rtw::ObjDev o;
    if ((rc = rtw::host::object_device_entry(oh, tp, 0, o)) != RTW_OK) return rc;

    unsigned char* base = nullptr;
    if ((rc = scratch_address(&base)) != RTW_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const long long R_ = tp->n_rays, n = R_ * np;
    rtw::RaysDev st{};
    st.R = R_;
    st.np = np;
    st.precision = RTW_FP64;
    unsigned char* p = base + kObjBytes;
    st.s01 = reinterpret_cast<double2*>(p);
    st.s2psi = reinterpret_cast<double2*>(p + 16 * n);
    st.Fx = reinterpret_cast<double2*>(p + 32 * n);
    st.Fy = reinterpret_cast<double2*>(p + 48 * n);
    st.Fz = reinterpret_cast<double2*>(p + 64 * n);
    st.flags = reinterpret_cast<uint32_t*>(p + 80 * n);
    st.aux = nullptr;
    st.frec = nullptr;
    st.fval = nullptr;
    unsigned int* mask_words = reinterpret_cast<unsigned int*>(base + kObjBytes + kStateBytes);
    rtw::ObjDev* d_obj = reinterpret_cast<rtw::ObjDev*>(base);

    put_object_kernel<<<1, 1, 0, s>>>(o);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(RTW_ERR_CUDA, cudaGetErrorString(e));
    // the trace writes every (ray, order) slot it owns, valid or not; the mask words and the output
    // are accumulated and start from zero
    const int nout = (flags & RTW_FIELD_PER_ORDER) ? np : 1;
    const long long ndir = dirs->n_theta;
    if ((e = cudaMemsetAsync(mask_words, 0, sizeof(unsigned int) * (size_t)ndir, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(field_out, 0, sizeof(double) * 4 * (size_t)nout * (size_t)ndir, s)) != cudaSuccess)
        return set_error(RTW_ERR_CUDA, cudaGetErrorString(e));
    if ((e = rtw::launch_trace(d_obj, 1, st, tp->p_max, false, nullptr, s)) != cudaSuccess)
        return set_error(RTW_ERR_CUDA, cudaGetErrorString(e));
    rtw::FieldArgs a;
    a.d_obj = d_obj;
    a.st = st;
    a.pmax = tp->p_max;
    a.per_order = (flags & RTW_FIELD_PER_ORDER) ? 1 : 0;
    a.out = static_cast<double*>(field_out);
    a.mask = mask_words;
    a.status = nullptr;  // no kernel of the plain fan path raises an error bit
    a.nfail = nullptr;
    if ((e = rtw::launch_field_fan(a, R_, tp->fan_phi, (int)ndir, dirs->alpha0, dirs->dalpha, nullptr, nullptr,
                                   nullptr, 0, 0, 0, s)) != cudaSuccess)
        return set_error(RTW_ERR_CUDA, cudaGetErrorString(e));
    if (mask_out) {
        if ((e = rtw::launch_finalize_mask(mask_words, mask_out, d_obj, 1, ndir, 0, dirs->n_theta, 0, dirs->alpha0,
                                           dirs->dalpha, s)) != cudaSuccess)
            return set_error(RTW_ERR_CUDA, cudaGetErrorString(e));
    }
    return RTW_OK;
}
