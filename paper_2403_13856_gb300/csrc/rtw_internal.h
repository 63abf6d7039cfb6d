// rtw_internal.h -- device-side data layout shared by the CUDA translation units of librtw.
//
// One object table entry per ellipsoid (ObjDev) and one structure-of-arrays ray state (RaysDev)
// per rtw_rays handle.  Ray state index: i = p * R + j, p the order, j the global ray index
// (objects laid out one after the other, square grids row-major with x fastest), R the number of
// rays per order, so that consecutive threads (consecutive j) touch consecutive 16-byte vectors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rtw {

constexpr int kMaxOrders = 16;

enum : uint32_t {
    kFlagValid = 1u,
    kFlagOrient = 2u,   // set: the map (x, y) -> s preserves orientation (z up, s outward)
    kFlagCaustic = 4u,  // dA/dOmega above the caustic cap
};
__host__ __device__ inline uint32_t flag_nf(uint32_t f) { return (f >> 8) & 0xffu; }

enum : int { kGridFan = 0, kGridSquare = 1 };

struct ObjDev {
    double W[6];  // symmetric quadric matrix: xx xy xz yy yz zz; surface (x-c)^T W (x-c) = 1
    double c[3];  // centre
    double m;     // n_object / n_host
    double k0;    // 2 pi / lambda
    double lambda;
    double jre[2], jim[2];  // incident Jones vector on (x, y)
    double zstart;          // plane where the incident rays start
    double S[3];            // projected ellipse xx xy yy
    double cap;             // caustic cap on dA/dOmega (um^2)
    double lmin, lmax;
    // ray grid
    int grid;
    int pad0;
    double h;               // square: spacing; fan: 2 w / n
    double fan_w, fan_ex, fan_ey;
    long long nx, ny;       // square: grid size; fan: (n, 1)
    long long ray_offset;   // first global ray index of this object
    long long item_first;   // first work item (kRaysPerItem rays) of this object in a batched trace
    double gc[2];           // centre of the square ray grid (plane wave: c_x, c_y)
    double src[3];          // point source (src_mode 1): rays leave it through c + x e1 + y e2
    double e1[3], e2[3];
    int src_mode;
    int shape_n;            // 2 shape_e when that is an integer in [3, 32] (powers by products), else 0
    // superellipsoid sum_i |u_i|^(2e) = 1, u_i = inv_a[i] (Rb^T (x - c))_i, for shape_e > 1 (1: the
    // quadric W above); the body lies inside the ellipsoid sum_i u_i^2 = bound2 = 3^(1 - 1/e)
    double Rb[9];           // body -> world rotation, row-major (columns are the body axes)
    double inv_a[3];
    double shape_e;
    double bound2;
};
static_assert(sizeof(ObjDev) == 464, "object table entries are 464 bytes");

// rays per work item of the persistent batched trace
constexpr int kRaysPerItem = 256;

// Double-precision ray state.  Aux arrays (exit-wave data for the PO integral) are allocated for
// fan grids traced with RTW_TRACE_APERTURE only.
enum AuxField : int {
    kAuxRx = 0, kAuxRy, kAuxRz,              // exit point
    kAuxExr, kAuxExi, kAuxEyr, kAuxEyi, kAuxEzr, kAuxEzi,  // exit field vector (Fresnel chain only)
    kAuxQ11, kAuxQ12, kAuxQ22,               // exit WFC in (e_perp, e_perp x s)
    kAuxEpx, kAuxEpy, kAuxEpz,               // e_perp of the exit interaction
    kAuxDlegs, kAuxPath, kAuxNfLegs,
    kAuxCount
};

struct RaysDev {
    long long R;      // rays per order
    int np;           // number of orders
    int precision;    // RTW_FP64 / RTW_MIXED / RTW_DFLOAT
    double near_r;    // > 0: records at the points where the rays cross the sphere |M| = near_r
    // FP64 state
    double2* s01;     // (s_x, s_y)
    double2* s2psi;   // (s_z, Psi)
    double2* Fx;      // F_x (re, im)
    double2* Fy;
    double2* Fz;
    uint32_t* flags;
    // single-precision field records of every (ray, order) for the square-grid field, two 32-byte
    // halves in two arrays: the geometry that the classification reads, frec[2 i], frec[2 i + 1] =
    // (theta, phi, s_x, s_y hi), (s_z hi, s_x, s_y, s_z lo); the values that a hit reads, fval[2 i],
    // fval[2 i + 1] = (Psi_hi, Psi_lo, F_x), (F_y, F_z) -- direction and phase as hi + lo pairs (about
    // 48 bits), F, theta and phi to single precision; null when not kept
    float4* frec;
    float4* fval;
    double* aux;      // kAuxCount x (np R) or null
    unsigned int* fmax;  // per object: bits of the largest |F|^2 (float) of a valid record that is not
                         //   near-caustic (the scale of the field's fixed-point sums); null when not kept
};

// Double to single precision in the integer pipe (the double-precision pipe, which also converts
// between the precisions, issues 1.6 operations per clock per SM on GB300, the integer pipe 64):
// the exponent is rebiased and the 52-bit significand rounded to 23 bits, half away from zero.
// Normal results only: magnitudes below 2^-126 give a signed zero, above the single range infinity.
__device__ __forceinline__ float f64_to_f32_int(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
    const unsigned int sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    // top 23 significand bits and the rounding bit below them
    const unsigned int m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned int r = (lo >> 28) & 1u;
    return __uint_as_float(sign | (((unsigned int)e << 23) + m + r));  // a carry rounds into the exponent
}

// Single to double precision in the integer pipe (exact for normal numbers; subnormals give 0).
__device__ __forceinline__ double f32_to_f64_int(float v)
{
    const unsigned int u = __float_as_uint(v);
    const unsigned int e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

// error bits of the device status word
enum : unsigned int { kStatusCapacity = 1u, kStatusTimeout = 2u, kStatusNumeric = 4u };

}  // namespace rtw
