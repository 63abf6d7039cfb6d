// rtw_field.cu -- the second half of the RTW hot path: the ray map interpolated onto the
// observation directions and all rays summed ("Strategy of Ray Theory of Waves", principle iii),
// and the physical-optics integral around in-plane folds ("Diffraction effect correction based
// on VCRM").
//
// Square grids: one thread per (order, cell) of the ray grid.  A cell is split along its diagonal
// into two triangles of neighbouring rays; the image triangle on the unit sphere of directions
// owns the grid directions inside it (sign tests of the edge planes s_lo x s_hi, evaluated with the
// endpoints in ray-index order so both triangles of an edge compute the same product: a direction
// on a shared edge is owned exactly once).  The candidate directions come from a single-precision
// cap around the triangle (conservative, 1e-5 rad margin); the tests, the interpolation and the
// phase are double precision.  Hits are few (about one per direction, branch and order), so the
// accumulation is a double-precision atomicAdd into the output.
#include <math_constants.h>

#include "rtw_launch.h"
#include "rtw_device.cuh"
#include "rtw_trace.cuh"

namespace rtw {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr unsigned int kMaskCaustic = 1u, kMaskAxial = 2u, kMaskPo = 4u;
constexpr double kFoldNewtonWindow = 2.0 * 3.14159265358979323846 / 180.0;  // 2 deg around a fold

__device__ __forceinline__ double wrap_angle(double a)
{
    if (!(fabs(a) < 1e6)) return a;  // non-finite input: no wrapping loop
    while (a > kPi) a -= 2.0 * kPi;
    while (a <= -kPi) a += 2.0 * kPi;
    return a;
}

__device__ __forceinline__ double ramp(double x, double x0, double x1)
{
    if (x <= x0) return 1.0;
    if (x >= x1) return 0.0;
    double c = cos(0.5 * kPi * (x - x0) / (x1 - x0));
    return c * c;
}

__device__ __forceinline__ bool edge_in(double e, long long ia, long long ib, int sigma)
{
    const double se = sigma > 0 ? e : -e;
    if (se > 0.0) return true;
    if (se < 0.0) return false;
    return (ia < ib) == (sigma > 0);
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void load_dir(const RaysDev& st, long long i, double* s)
{
    const double2 a = st.s01[i];
    const double2 b = st.s2psi[i];
    s[0] = a.x;
    s[1] = a.y;
    s[2] = b.x;
}

// F e^{i Psi} projected on (e_theta, e_phi) and added into acc (4 doubles)
__device__ __forceinline__ void add_contribution(const double* F, double psi, const double* eth, const double* eph,
                                                 double w, double* dst)
{
    double sp, cp;
    sincos(psi, &sp, &cp);
    double tr = 0.0, ti = 0.0, pr = 0.0, pi = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double re = F[2 * c] * cp - F[2 * c + 1] * sp;
        const double im = F[2 * c] * sp + F[2 * c + 1] * cp;
        tr += re * eth[c];
        ti += im * eth[c];
        pr += re * eph[c];
        pi += im * eph[c];
    }
    atomicAdd(dst + 0, w * tr);
    atomicAdd(dst + 1, w * ti);
    atomicAdd(dst + 2, w * pr);
    atomicAdd(dst + 3, w * pi);
}


// ---------------------------------------------------------------------------------------------
// direction tables: cos(theta_i), sin(theta_i), cos(phi_j), sin(phi_j)
// ---------------------------------------------------------------------------------------------
// double tables (4 x n) followed by single-precision copies (4 x n floats) and the remainders of
// those copies (4 x n floats: value = copy + remainder to about 2^-48)
__global__ void dir_tables_kernel(int nt, int nph, double* tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float* ftab = reinterpret_cast<float*>(tab + 2 * (nt + nph));
    float* ltab = ftab + 2 * (nt + nph);
    if (i < nt) {
        double s, c;
        sincos((i + 0.5) * (kPi / nt), &s, &c);
        tab[i] = c;
        tab[nt + i] = s;
        ftab[i] = (float)c;
        ftab[nt + i] = (float)s;
        ltab[i] = (float)(c - (double)(float)c);
        ltab[nt + i] = (float)(s - (double)(float)s);
    }
    if (i < nph) {
        double s, c;
        sincos(-kPi + (i + 0.5) * (2.0 * kPi / nph), &s, &c);
        tab[2 * nt + i] = c;
        tab[2 * nt + nph + i] = s;
        ftab[2 * nt + i] = (float)c;
        ftab[2 * nt + nph + i] = (float)s;
        ltab[2 * nt + i] = (float)(c - (double)(float)c);
        ltab[2 * nt + nph + i] = (float)(s - (double)(float)s);
    }
}

// ---------------------------------------------------------------------------------------------
// square grid.  Phase 1: one thread per (order, cell) boxes the cell's two triangles; a triangle
// whose candidate box holds few grid directions is queued in the block and finished there by one
// thread, a larger one (rim rays near grazing incidence map onto wide image triangles) goes to a
// list.  Phase 2: the listed triangles a warp at a time, the lanes taking their candidate directions
// in turn, so that no thread serialises thousands of tests.  Phase 3: the hits summed.
// ---------------------------------------------------------------------------------------------
constexpr int kInlineCandidates = 32;  // measured best of 4..64 with the block queue (ellipsoid, spheroid)
constexpr unsigned int kHitClose = 0x80000000u;  // hit entry flag: needs the double-precision test

struct TriGeom {
    long long id[3];  // local ray indices, counter-clockwise in the ray grid
    uint32_t f[3];
    float s[3][3];    // single-precision (hi) exit directions
    float l[3][3];    //   and their lo parts
    float th[3], ph[3];  // theta and phi of the corners' directions (phi unwrapped by tri_box)
    float c[3];       // unit vector at the centre of the image triangle (local origin)
    int it0, it1, jp0, jcount;
    float mt;         // tri_box: the theta margin of the edges' bulge; 0 for a cap (tri_setup)
    float cth, cph, crho;  // tri_setup: the cap's centre (theta, phi) and radius
};

// the single-precision candidate cap of a triangle whose corners are loaded; returns the number of
// candidates
__device__ __forceinline__ long long tri_setup(TriGeom& g, const DirSet& d)
{
    const int nt = d.nt, nph = d.nph;
    if (!(g.f[0] & g.f[1] & g.f[2] & kFlagValid)) return 0;
    float cmx = g.s[0][0] + g.s[1][0] + g.s[2][0];
    float cmy = g.s[0][1] + g.s[1][1] + g.s[2][1];
    float cmz = g.s[0][2] + g.s[1][2] + g.s[2][2];
    const float cn = rsqrtf(cmx * cmx + cmy * cmy + cmz * cmz);
    cmx *= cn;
    cmy *= cn;
    cmz *= cn;
    g.c[0] = cmx;
    g.c[1] = cmy;
    g.c[2] = cmz;
    float ch = 0.0f;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const float dx = g.s[v][0] - cmx, dy = g.s[v][1] - cmy, dz = g.s[v][2] - cmz;
        ch = fmaxf(ch, sqrtf(dx * dx + dy * dy + dz * dz));
    }
    // corners more than 90 deg (chord sqrt 2) from their mean do not lie in one hemisphere: the
    // edge planes bound no proper spherical triangle, and the cell is skipped
    if (!(ch < 1.41421356f)) return 0;
    // a list's bins are candidates when their centre lies within the cap widened by a bin radius
    const float rho = 2.0f * asinf(fminf(1.0f, 0.5f * ch)) + 1e-5f + d.pad;
    const float thc = atan2f(sqrtf(cmx * cmx + cmy * cmy), cmz), phc = atan2f(cmy, cmx);
    g.mt = 0.0f;
    g.cth = thc;
    g.cph = phc;
    g.crho = rho;
    const float dth = 3.14159265358979f / nt, dph = 6.28318530717959f / nph;
    g.it0 = max((int)ceilf((thc - rho) / dth - 0.5f), 0);
    g.it1 = min((int)floorf((thc + rho) / dth - 0.5f), nt - 1);
    bool allphi = (thc - rho <= 0.0f) || (thc + rho >= 3.14159265358979f);
    g.jp0 = 0;
    g.jcount = nph;
    if (!allphi) {
        const float sr = sinf(rho) / sinf(thc);
        if (sr < 0.9f) {  // close to a pole the phi extent is ill-conditioned: take every phi
            const float dphi = asinf(sr) + 1e-5f;
            g.jp0 = (int)ceilf((phc - dphi + 3.14159265358979f) / dph - 0.5f);
            const int jp1 = (int)floorf((phc + dphi + 3.14159265358979f) / dph - 0.5f);
            g.jcount = min(max(jp1 - g.jp0 + 1, 0), nph);
            if (jp1 - g.jp0 + 1 > nph) g.jp0 = 0;
        }
    }
    if (g.it1 < g.it0 || g.jcount <= 0) return 0;
    return (long long)(g.it1 - g.it0 + 1) * g.jcount;
}

__device__ __forceinline__ void cross3f(const float* a, const float* b, float* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Single-precision tests in a local frame.  With c the unit vector at the triangle's centre and
// d_v = s_v - c (from the hi + lo split of s_v, relative error below 1.2e-7), an edge plane is
// s_a x s_b = c x (d_b - d_a) + d_a x d_b and its value at a direction x = c + dx is
// e = (d_a x d_b) . c + (s_a x s_b) . dx.  Every term scales with the triangle, so the rounding of
// the inputs, of the table direction (3.1e-7) and of the arithmetic stays below
// 2e-6 (|d_a| + |d_b|); signs beyond that bound are the double-precision signs.  The triangle's
// orientation c . ((d_1 - d_0) x (d_2 - d_0)) + d_0 . (d_1 x d_2) is decided the same way.  Closer
// calls go to the double-precision rule.
struct TriFrame {
    float n[3][3], k[3], tol[3], sg[3];
    int sig32;
    bool ok;  // corners agree in focal lines, orientation and carry no caustic flag, image not folded
};

__device__ __forceinline__ void tri_frame(const TriGeom& g, TriFrame& fr)
{
    const float* c = g.c;
    float d[3][3], dn[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        d[v][0] = (g.s[v][0] - c[0]) + g.l[v][0];
        d[v][1] = (g.s[v][1] - c[1]) + g.l[v][1];
        d[v][2] = (g.s[v][2] - c[2]) + g.l[v][2];
        dn[v] = sqrtf(d[v][0] * d[v][0] + d[v][1] * d[v][1] + d[v][2] * d[v][2]);
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int va = e, vb = (e + 1) % 3;
        const bool fwd = g.id[va] < g.id[vb];
        const float* dl = fwd ? d[va] : d[vb];
        const float* dh = fwd ? d[vb] : d[va];
        fr.sg[e] = fwd ? 1.0f : -1.0f;
        const float dd[3] = {dh[0] - dl[0], dh[1] - dl[1], dh[2] - dl[2]};
        float cx[3], dx[3];
        cross3f(c, dd, cx);
        cross3f(dl, dh, dx);
        fr.n[e][0] = cx[0] + dx[0];
        fr.n[e][1] = cx[1] + dx[1];
        fr.n[e][2] = cx[2] + dx[2];
        fr.k[e] = dx[0] * c[0] + dx[1] * c[1] + dx[2] * c[2];
        fr.tol[e] = 2e-6f * (dn[va] + dn[vb]);
    }
    const float u[3] = {d[1][0] - d[0][0], d[1][1] - d[0][1], d[1][2] - d[0][2]};
    const float w[3] = {d[2][0] - d[0][0], d[2][1] - d[0][1], d[2][2] - d[0][2]};
    float uw[3], d12[3];
    cross3f(u, w, uw);
    cross3f(d[1], d[2], d12);
    const float vol =
        c[0] * uw[0] + c[1] * uw[1] + c[2] * uw[2] + d[0][0] * d12[0] + d[0][1] * d12[1] + d[0][2] * d12[2];
    const float un = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const float wn = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    const float tv = 2e-6f * (un * wn + dn[0] * dn[1] * dn[2]);
    fr.sig32 = vol > tv ? 1 : (vol < -tv ? -1 : 0);
    const uint32_t* f = g.f;
    fr.ok = flag_nf(f[0]) == flag_nf(f[1]) && flag_nf(f[1]) == flag_nf(f[2]) && ((f[0] ^ f[1]) & kFlagOrient) == 0 &&
            ((f[1] ^ f[2]) & kFlagOrient) == 0 && ((f[0] | f[1] | f[2]) & kFlagCaustic) == 0 &&
            fr.sig32 == ((f[0] & kFlagOrient) ? 1 : -1);
}

// 0: outside; 1: inside (sure); 2: close call
__device__ __forceinline__ int tri_classify(const TriFrame& fr, float dx0, float dx1, float dx2)
{
    int npos = 0, nneg = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ef = fr.sg[k] * (fr.k[k] + fr.n[k][0] * dx0 + fr.n[k][1] * dx1 + fr.n[k][2] * dx2);
        npos += ef > fr.tol[k];
        nneg += ef < -fr.tol[k];
    }
    if (npos > 0 && nneg > 0) return 0;
    if ((npos == 3 || nneg == 3) && fr.sig32 != 0) return ((npos == 3 ? 1 : -1) == fr.sig32) ? 1 : 0;
    return 2;
}

struct HitArgs {
    unsigned long long* tri;  // (order-cell index << 1) | triangle
    unsigned int* dir;        // direction index | kHitClose
    unsigned int* n;
    unsigned int cap;
    int raise;                // 1: an overflow is an error; 0: the host reads *n and splits the run
};

// warp-aggregated append of one (triangle, direction) pair
__device__ __forceinline__ void push_hit(const HitArgs& h, unsigned int* status, unsigned long long code,
                                         unsigned int dir)
{
    const unsigned int m = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned int b = 0;
    if (lane == leader) b = atomicAdd(h.n, (unsigned int)__popc(m));
    b = __shfl_sync(m, b, leader) + __popc(m & ((1u << lane) - 1u));
    if (b < h.cap) {
        h.tri[b] = code;
        h.dir[b] = dir;
    } else if (h.raise) {
        atomicOr(status, kStatusCapacity);
    }
}

// caustic bits of a direction covered by a triangle of order p that is not consistent: bit 0, and bit
// 8 + p that tells the orders apart (the caustic correction reads it; the byte mask keeps bit 0)
__device__ __forceinline__ unsigned int caustic_bits(int p) { return kMaskCaustic | (0x100u << p); }

__device__ __forceinline__ void candidate(const FieldArgs& a, const HitArgs& h, const TriFrame& fr,
                                          unsigned long long code, unsigned int* mask, unsigned int cbit,
                                          unsigned int dk, float dx0, float dx1, float dx2)
{
    const int cls = tri_classify(fr, dx0, dx1, dx2);
    if (cls == 0) return;
    if (cls == 2) {
        push_hit(h, a.status, code, dk | kHitClose);
    } else if (!fr.ok) {  // singular or folded cell: mark, add nothing
        if ((mask[dk] & cbit) != cbit) atomicOr(mask + dk, cbit);
    } else {
        push_hit(h, a.status, code, dk);
    }
}

// The cells of one launch: objects [obj0, obj0 + nobj) of the table, each with its cell window
// and the first thread index of its (order, cell) range.
__device__ __forceinline__ CellRef decode_cell(const FieldArgs& a, const GridBatch& b, long long t)
{
    int lo = 0, hi = b.nobj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.cells[mid].first <= t) lo = mid;
        else hi = mid - 1;
    }
    const GridCells& gc = b.cells[lo];
    CellRef r;
    r.orel = lo;
    r.o = a.d_obj + lo;
    const long long ncell = gc.ncx * gc.ncy;
    const long long local = t - gc.first;
    if (local <= 0xffffffffll && ncell <= 0xffffffffll) {
        // 32-bit division where the indices fit (every grid here): far cheaper than 64-bit
        const unsigned int l32 = (unsigned int)local, n32 = (unsigned int)ncell, x32 = (unsigned int)gc.ncx;
        const unsigned int p32 = l32 / n32, c32 = l32 - p32 * n32, y32 = c32 / x32;
        r.p = (int)p32;
        r.cx = gc.ix0 + (long long)(c32 - y32 * x32);
        r.cy = gc.iy0 + (long long)y32;
    } else {
        r.p = (int)(local / ncell);
        const long long cell = local - (long long)r.p * ncell;
        r.cx = gc.ix0 + cell % gc.ncx;
        r.cy = gc.iy0 + cell / gc.ncx;
    }
    r.nx = r.o->nx;
    r.base = (long long)r.p * a.st.R + r.o->ray_offset;
    return r;
}

// corners of triangle t (0: c00 c10 c11, 1: c00 c11 c01) of cell (cx, cy)
__device__ __forceinline__ void cell_triangle(const FieldArgs& a, long long base, long long nx, long long cx,
                                              long long cy, int t, TriGeom& g)
{
    const long long l00 = cy * nx + cx;
    g.id[0] = l00;
    g.id[1] = t == 0 ? l00 + 1 : l00 + nx + 1;
    g.id[2] = t == 0 ? l00 + nx + 1 : l00 + nx;
#pragma unroll
    for (int v = 0; v < 3; ++v) g.f[v] = a.st.flags[base + g.id[v]];
}

// theta, phi and the direction's hi parts of corner v from its field record
__device__ __forceinline__ void load_corner_hi(const FieldArgs& a, long long i, TriGeom& g, int v)
{
    const float4 r0 = a.st.frec[2 * i], r1 = a.st.frec[2 * i + 1];
    g.th[v] = r0.x;
    g.ph[v] = r0.y;
    g.s[v][0] = r0.z;
    g.s[v][1] = r0.w;
    g.s[v][2] = r1.x;
    g.l[v][0] = r1.y;
    g.l[v][1] = r1.z;
    g.l[v][2] = r1.w;
}

// (the low parts come with the geometry record)
__device__ __forceinline__ void load_corner_lo(const FieldArgs&, long long, TriGeom&, int) {}

// corners of triangle t with their single-precision directions (hi and lo parts)
__device__ __forceinline__ void load_triangle(const FieldArgs& a, long long base, long long nx, long long cx,
                                              long long cy, int t, TriGeom& g)
{
    cell_triangle(a, base, nx, cx, cy, t, g);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        load_corner_hi(a, base + g.id[v], g, v);
        load_corner_lo(a, base + g.id[v], g, v);
    }
}

// Candidate box of a triangle on a (theta, phi) grid from its corners' theta and phi.  A great
// circle crosses every half-meridian once, so phi along an edge is monotonic and the triangle's phi
// range is its corners' (less a pole inside); theta along an edge bulges toward the nearer pole by
// less than L^2 |cot theta| / 8 (L the edge's chord), taken four times over.  Triangles near a pole,
// wide in phi or long use the cap of tri_setup; so do lists (their bins widen every cap).  Returns
// the number of candidates (0: none).
__device__ __forceinline__ long long tri_box(TriGeom& g, const DirSet& d)
{
    g.mt = 0.0f;
    if (!(g.f[0] & g.f[1] & g.f[2] & kFlagValid)) return 0;
    if (d.list) return tri_setup(g, d);
    float l2 = 0.0f, cmax = 0.0f, s2min = 1.0f;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const int w = (v + 1) % 3;
        const float dx = g.s[v][0] - g.s[w][0], dy = g.s[v][1] - g.s[w][1], dz = g.s[v][2] - g.s[w][2];
        l2 = fmaxf(l2, dx * dx + dy * dy + dz * dz);
        // sin^2 theta and |cos theta| of a unit direction
        s2min = fminf(s2min, g.s[v][0] * g.s[v][0] + g.s[v][1] * g.s[v][1]);
        cmax = fmaxf(cmax, fabsf(g.s[v][2]));
    }
    // the margins below exceed the rounding of these approximate forms (relative 1e-6) many times
    const float smin = s2min * rsqrtf(fmaxf(s2min, 1e-30f));
    float p0 = g.ph[0], p1 = g.ph[1], p2 = g.ph[2];
    if (fmaxf(p0, fmaxf(p1, p2)) - fminf(p0, fminf(p1, p2)) > 3.14159265f) {  // across phi = +-pi
        p0 += p0 < 0.0f ? 6.28318531f : 0.0f;
        p1 += p1 < 0.0f ? 6.28318531f : 0.0f;
        p2 += p2 < 0.0f ? 6.28318531f : 0.0f;
    }
    const float pmin = fminf(p0, fminf(p1, p2)), pmax = fmaxf(p0, fmaxf(p1, p2));
    if (l2 > 0.25f || smin < 0.05f || pmax - pmin > 1.0f) return tri_setup(g, d);
    const float mt = 0.5f * l2 * (__fdividef(cmax, smin) + 1.0f) + 2e-6f, mp = 1e-5f;
    g.ph[0] = p0;
    g.ph[1] = p1;
    g.ph[2] = p2;
    g.mt = mt;
    const float tmin = fminf(g.th[0], fminf(g.th[1], g.th[2])), tmax = fmaxf(g.th[0], fmaxf(g.th[1], g.th[2]));
    const int nt = d.nt, nph = d.nph;
    // rows and columns by multiplication with the reciprocal spacing: the rounding, 1.5 ulp of index
    // values up to 2 nph (0.006 of a column at 36000 columns), stays below a tenth of the margins
    const float ith = nt * 0.318309886f, iph = nph * 0.159154943f;
    g.it0 = max((int)ceilf((tmin - mt) * ith - 0.5f), 0);
    g.it1 = min((int)floorf((tmax + mt) * ith - 0.5f), nt - 1);
    g.jp0 = (int)ceilf((pmin - mp + 3.14159265358979f) * iph - 0.5f);
    const int jp1 = (int)floorf((pmax + mp + 3.14159265358979f) * iph - 0.5f);
    g.jcount = min(max(jp1 - g.jp0 + 1, 0), nph);
    if (g.it1 < g.it0 || g.jcount <= 0) return 0;
    // the local origin of the single-precision tests
    float cx = g.s[0][0] + g.s[1][0] + g.s[2][0], cy = g.s[0][1] + g.s[1][1] + g.s[2][1];
    float cz = g.s[0][2] + g.s[1][2] + g.s[2][2];
    const float cn = rsqrtf(cx * cx + cy * cy + cz * cz);
    g.c[0] = cx * cn;
    g.c[1] = cy * cn;
    g.c[2] = cz * cn;
    return (long long)(g.it1 - g.it0 + 1) * g.jcount;
}

struct DirTabF {
    const float *ct, *st, *cp, *sp;
};

__device__ __forceinline__ DirTabF dir_tab_f(const double* tab, int nt, int nph)
{
    const float* f = reinterpret_cast<const float*>(tab + 2 * (nt + nph));
    return DirTabF{f, f + nt, f + 2 * nt, f + 2 * nt + nph};
}

// every candidate direction of one (bin) grid point (it, jp): the point itself, or a bin's list
__device__ __forceinline__ void candidates_at(const FieldArgs& a, const HitArgs& h, const DirSet& d,
                                              const DirTabF& T, const TriFrame& fr, const TriGeom& g,
                                              unsigned long long code, unsigned int* mask, unsigned int cbit, int it,
                                              int jp)
{
    if (!d.list) {
        const float sth = T.st[it];
        candidate(a, h, fr, code, mask, cbit, (unsigned int)it * (unsigned int)d.nph + (unsigned int)jp,
                  sth * T.cp[jp] - g.c[0], sth * T.sp[jp] - g.c[1], T.ct[it] - g.c[2]);
        return;
    }
    const int bn = it * d.nph + jp;
    for (int m = d.bin_first[bn]; m < d.bin_first[bn + 1]; ++m) {
        const unsigned int dk = (unsigned int)d.bin_dir[m];
        const float4 x = d.ldir_f[dk];
        candidate(a, h, fr, code, mask, cbit, dk, x.x - g.c[0], x.y - g.c[1], x.z - g.c[2]);
    }
}

// Triangles with at most kInlineCandidates candidates are queued in shared memory by the first pass and taken
// one per thread by the second, so that the few threads whose triangles hold candidates (about one
// triangle in ten on dense ray grids) work in full warps instead of a few lanes of every warp.
constexpr int kClassifyMaxThreads = 256;

__global__ void __launch_bounds__(kClassifyMaxThreads) field_grid_kernel(FieldArgs a, GridBatch b, DirSet d,
                                                                         unsigned long long* big, unsigned int* nbig,
                                                                         unsigned int big_cap, HitArgs h)
{
    __shared__ unsigned long long queue[2 * kClassifyMaxThreads];
    __shared__ unsigned int nqueue;
    if (threadIdx.x == 0) nqueue = 0u;
    __syncthreads();
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    if (tid < b.total) {
        const CellRef c = decode_cell(a, b, tid);
        for (int t = 0; t < 2; ++t) {
            TriGeom g;
            cell_triangle(a, c.base, c.nx, c.cx, c.cy, t, g);
            if (!(g.f[0] & g.f[1] & g.f[2] & kFlagValid)) continue;
#pragma unroll
            for (int v = 0; v < 3; ++v) load_corner_hi(a, c.base + g.id[v], g, v);
            const long long nc = tri_box(g, d);
            if (nc == 0) continue;
            const unsigned long long code = ((unsigned long long)tid << 1) | (unsigned long long)t;
            if (nc > kInlineCandidates) {
                // warp-aggregated append to the list of the large-triangle kernel
                const unsigned int m = __activemask();
                const int leader = __ffs(m) - 1;
                unsigned int slot = 0;
                if (lane == leader) slot = atomicAdd(nbig, (unsigned int)__popc(m));
                slot = __shfl_sync(m, slot, leader) + __popc(m & ((1u << lane) - 1u));
                if (slot < big_cap) {
                    big[slot] = code;
                    continue;
                }
            }
            // the block's queue (two entries per thread at most: it cannot overflow)
            const unsigned int m = __activemask();
            const int leader = __ffs(m) - 1;
            unsigned int slot = 0;
            if (lane == leader) slot = atomicAdd(&nqueue, (unsigned int)__popc(m));
            slot = __shfl_sync(m, slot, leader) + __popc(m & ((1u << lane) - 1u));
            queue[slot] = code;
        }
    }
    __syncthreads();
    const unsigned int nq = nqueue;
    const int nph = d.nph;
    const DirTabF T = dir_tab_f(d.tab, d.nt, nph);
    for (unsigned int e = threadIdx.x; e < nq; e += blockDim.x) {
        // the triangle again (its corners are in this SM's cache), its candidate box and edge frame
        const unsigned long long code = queue[e];
        const CellRef c = decode_cell(a, b, (long long)(code >> 1));
        TriGeom g;
        load_triangle(a, c.base, c.nx, c.cx, c.cy, (int)(code & 1ull), g);
        tri_box(g, d);
        TriFrame fr;
        tri_frame(g, fr);
        unsigned int* mask = a.mask + (long long)c.orel * b.ndir;
        const unsigned int cbit = caustic_bits(c.p);
        for (int it = g.it0; it <= g.it1; ++it) {
            for (int jj = 0; jj < g.jcount; ++jj) {
                int jp = g.jp0 + jj;
                jp = jp >= nph ? jp - nph : (jp < 0 ? jp + nph : jp);
                candidates_at(a, h, d, T, fr, g, code, mask, cbit, it, jp);
            }
        }
    }
}

// Phase 2: the listed triangles in batches of 32 per warp.  First every lane sets up one triangle
// of the batch (cell, corners, candidate cap, edge frame) into shared memory; then the warp takes
// the batch's triangles in turn, the lanes walking a triangle's candidate grid points (row-major
// over the candidate rows and columns) 32 apart, so that narrow triangles spanning many rows keep
// every lane busy and no lane repeats another's set-up.
struct BigRec {
    TriFrame fr;
    float c[3];
    int it0, it1, jp0, jcount;
    // the rows' spans: a boxed triangle's corners (theta 3, phi 3 unwrapped) and bulge margin (> 0),
    // or a cap's centre theta, phi and radius (sp[6] = 0)
    float sp[7];
    unsigned long long code;
    int orel, valid;  // valid: 1 + the order of the cell, 0 for an empty entry
};
constexpr int kBigWarps = 8;  // warps per block of the large-triangle kernel
constexpr int kSpanMin = 128;  // boxes of more candidates take the rows' spans (big_row_span)

// Candidate columns of row it of a large triangle, inside its box: [*j0, *j0 + count), unwrapped
// (taken modulo nph).  A boxed triangle's points on the row lie, at the same phi, within its bulge
// margin in theta of the plane triangle of its corners' (theta, phi) (the margin that widens its box),
// so their phi lies in the phi extent of that plane triangle clipped to the strip of that half-width
// about the row.  A cap's points on the row lie within the cap's phi half-width there,
// cos dphi = (cos rho - cos theta cos theta_c) / (sin theta sin theta_c), taken wider by the
// rounding of the single-precision terms.  The margins cover the rounding of the box's own bounds.
__device__ __forceinline__ int big_row_span(const BigRec& r, int it, float dth, float dph, int nph, int* j0)
{
    const float tr = (it + 0.5f) * dth;
    float pmin, pmax;
    bool all = false;
    if (r.sp[6] > 0.0f) {
        const float lo = tr - r.sp[6], hi = tr + r.sp[6];
        pmin = 1e30f;
        pmax = -1e30f;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const float t0 = r.sp[v], p0 = r.sp[3 + v];
            if (t0 >= lo && t0 <= hi) {
                pmin = fminf(pmin, p0);
                pmax = fmaxf(pmax, p0);
            }
            const int w = v == 2 ? 0 : v + 1;
            const float t1 = r.sp[w], p1 = r.sp[3 + w];
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float y = b ? hi : lo;
                if ((t0 - y) * (t1 - y) < 0.0f) {
                    const float pc = p0 + (y - t0) / (t1 - t0) * (p1 - p0);
                    pmin = fminf(pmin, pc);
                    pmax = fmaxf(pmax, pc);
                }
            }
        }
        if (!(pmin <= pmax)) return 0;
    } else {
        const float thc = r.sp[0], phc = r.sp[1], rho = r.sp[2];
        float st, ct, sc, cc;
        sincosf(tr, &st, &ct);
        sincosf(thc, &sc, &cc);
        const float den = st * sc;
        if (den < 1e-4f) {
            all = true;
            pmin = pmax = 0.0f;
        } else {
            const float arg = (cosf(rho) - ct * cc) / den - 4e-6f / den - 1e-5f;
            if (arg <= -1.0f) {
                all = true;
                pmin = pmax = 0.0f;
            } else {
                const float dphi = acosf(fminf(arg, 1.0f)) + 1e-4f;
                pmin = phc - dphi;
                pmax = phc + dphi;
            }
        }
    }
    const bool full_box = r.jcount >= nph;
    if (all) {
        *j0 = r.jp0;
        return r.jcount;
    }
    const float mp = 2e-5f;
    int jlo = (int)ceilf((pmin - mp + 3.14159265358979f) / dph - 0.5f);
    int jhi = (int)floorf((pmax + mp + 3.14159265358979f) / dph - 0.5f);
    if (full_box) {  // a box of every column: the row's span may cross the seam; modulo nph later
        if (jhi - jlo + 1 >= nph) {
            *j0 = 0;
            return nph;
        }
    } else {
        jlo = max(jlo, r.jp0);
        jhi = min(jhi, r.jp0 + r.jcount - 1);
    }
    *j0 = jlo;
    return jhi >= jlo ? jhi - jlo + 1 : 0;
}

__global__ void __launch_bounds__(32 * kBigWarps) field_grid_big_kernel(FieldArgs a, GridBatch b, DirSet d,
                                                                      const unsigned long long* big,
                                                                      const unsigned int* nbig, unsigned int big_cap,
                                                                      HitArgs h)
{
    __shared__ BigRec rec[kBigWarps][32];
    const unsigned int n = min(*nbig, big_cap);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long warps = (long long)gridDim.x * kBigWarps;
    const int nph = d.nph;
    const DirTabF T = dir_tab_f(d.tab, d.nt, nph);
    const float dth = 3.14159265358979f / d.nt, dph = 6.28318530717959f / nph;
    // lane l of warp w takes list entries w + warps (32 i + l): consecutive entries (neighbouring,
    // alike triangles) are spread over all warps
    const long long w = blockIdx.x * (long long)kBigWarps + wib;
    for (long long i0 = 0; w + warps * i0 < n; i0 += 32) {
        BigRec& mine = rec[wib][lane];
        mine.valid = 0;
        const long long e = w + warps * (i0 + lane);
        if (e < n) {
            const unsigned long long code = big[e];
            const CellRef c = decode_cell(a, b, (long long)(code >> 1));
            TriGeom g;
            load_triangle(a, c.base, c.nx, c.cx, c.cy, (int)(code & 1ull), g);
            if (tri_box(g, d) != 0) {
                tri_frame(g, mine.fr);
                mine.c[0] = g.c[0];
                mine.c[1] = g.c[1];
                mine.c[2] = g.c[2];
                mine.it0 = g.it0;
                mine.it1 = g.it1;
                mine.jp0 = g.jp0;
                mine.jcount = g.jcount;
                if (g.mt > 0.0f) {
#pragma unroll
                    for (int v = 0; v < 3; ++v) {
                        mine.sp[v] = g.th[v];
                        mine.sp[3 + v] = g.ph[v];
                    }
                    mine.sp[6] = g.mt;
                } else {
                    mine.sp[0] = g.cth;
                    mine.sp[1] = g.cph;
                    mine.sp[2] = g.crho;
                    mine.sp[6] = 0.0f;
                }
                mine.code = code;
                mine.orel = c.orel;
                mine.valid = 1 + c.p;
            }
        }
        __syncwarp();
        // the batch's boxes of at most kSpanMin candidates as one list: lane l's triangle holds
        // candidates [before_l, incl_l) of it (a warp scan of the box sizes); each lane finds the
        // triangle of candidate q by a binary search over the scan (shuffles), and its row and column
        // from the index inside the box, so that small boxes keep every lane busy
        {
            const BigRec& mr = rec[wib][lane];
            const long long box = (long long)(mr.it1 - mr.it0 + 1) * mr.jcount;
            const int cnt = (mr.valid && box <= kSpanMin) ? (int)box : 0;
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                int L = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int v = __shfl_sync(0xffffffffu, incl, L + step - 1);
                    if (v <= q) L += step;
                }
                const int before = __shfl_sync(0xffffffffu, incl, L > 0 ? L - 1 : 0);
                if (q < total) {
                    const BigRec& r = rec[wib][L];
                    const int e = q - (L > 0 ? before : 0);
                    const int row = e / r.jcount;
                    int jp = r.jp0 + (e - row * r.jcount);
                    jp = jp >= nph ? jp - nph : (jp < 0 ? jp + nph : jp);
                    TriGeom g;
                    g.c[0] = r.c[0];
                    g.c[1] = r.c[1];
                    g.c[2] = r.c[2];
                    candidates_at(a, h, d, T, r.fr, g, r.code, a.mask + (long long)r.orel * b.ndir,
                                  caustic_bits(r.valid - 1), r.it0 + row, jp);
                }
            }
        }
        // the boxes of more candidates one by one, their rows' spans taken
        for (int k = 0; k < 32; ++k) {
            const BigRec& r = rec[wib][k];
            if (!r.valid || (long long)(r.it1 - r.it0 + 1) * r.jcount <= kSpanMin) continue;
            const TriFrame fr = r.fr;
            TriGeom g;
            g.c[0] = r.c[0];
            g.c[1] = r.c[1];
            g.c[2] = r.c[2];
            const unsigned long long code = r.code;
            unsigned int* mask = a.mask + (long long)r.orel * b.ndir;
            const unsigned int cbit = caustic_bits(r.valid - 1);
            // 32 rows at a time: lane l takes the span of row r0 + l; the warp's inclusive scan of
            // the spans numbers the candidates, and each lane finds the row of candidate q by a
            // binary search over the scan (shuffles), the column from the row's first one
            for (int r0 = r.it0; r0 <= r.it1; r0 += 32) {
                int j0 = r.jp0, jn = 0;
                if (r0 + lane <= r.it1) jn = big_row_span(r, r0 + lane, dth, dph, nph, &j0);
                int incl = jn;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += y;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                for (int q0 = 0; q0 < total; q0 += 32) {
                    const int q = q0 + lane;
                    int L = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int v = __shfl_sync(0xffffffffu, incl, L + step - 1);
                        if (v <= q) L += step;
                    }
                    const int before = __shfl_sync(0xffffffffu, incl, L > 0 ? L - 1 : 0);
                    const int first = __shfl_sync(0xffffffffu, j0, L);
                    if (q < total) {
                        int jp = first + (q - (L > 0 ? before : 0));
                        jp %= nph;
                        jp = jp < 0 ? jp + nph : jp;
                        candidates_at(a, h, d, T, fr, g, code, mask, cbit, r0 + L, jp);
                    }
                }
            }
        }
        __syncwarp();
    }
}

// Phase 3: one thread per (triangle, direction) pair: the double-precision rule for close calls,
// then the barycentric weights of the central projection, F, Psi and F e^{i Psi}.  kNewton: replace
// the interpolated hit by the exact ray found by Newton steps (a separate instantiation, so that the
// dense mode does not carry the exact trace's registers).
template <bool kNewton>
__global__ void __launch_bounds__(256) field_grid_hit_kernel(FieldArgs a, GridBatch b, DirSet d, HitArgs h)
{
    const unsigned int n = min(*h.n, h.cap);
    const int nt = d.nt, nph = d.nph;
    const double* ctab = d.tab;
    const double* stab = d.tab + nt;
    const double* cptab = d.tab + 2 * nt;
    const double* sptab = d.tab + 2 * nt + nph;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const unsigned long long code = h.tri[q];
        const unsigned int dw = h.dir[q];
        const bool close = (dw & kHitClose) != 0;
        const unsigned int dk = dw & ~kHitClose;
        const int t = (int)(code & 1ull);
        const CellRef c = decode_cell(a, b, (long long)(code >> 1));
        const int p = c.p;
        const long long base = c.base;
        TriGeom g;
        cell_triangle(a, base, c.nx, c.cx, c.cy, t, g);
        double s[3][3];
#pragma unroll
        for (int v = 0; v < 3; ++v) load_dir(a.st, base + g.id[v], s[v]);
        double nrm[3][3], sg[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int va = e, vb = (e + 1) % 3;
            if (g.id[va] < g.id[vb]) {
                cross3(s[va], s[vb], nrm[e]);
                sg[e] = 1.0;
            } else {
                cross3(s[vb], s[va], nrm[e]);
                sg[e] = -1.0;
            }
        }
        double ct, sth, cp, sp;
        if (d.list) {
            const double* q = d.ldir + 4 * (long long)dk;
            ct = q[0];
            sth = q[1];
            cp = q[2];
            sp = q[3];
        } else {
            const int it = (int)(dk / (unsigned int)nph), jp = (int)(dk % (unsigned int)nph);
            ct = ctab[it];
            sth = stab[it];
            cp = cptab[jp];
            sp = sptab[jp];
        }
        const double x[3] = {sth * cp, sth * sp, ct};
        double e[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) e[k] = sg[k] * (nrm[k][0] * x[0] + nrm[k][1] * x[1] + nrm[k][2] * x[2]);
        if (close) {
            double c12[3];
            cross3(s[1], s[2], c12);
            const double vol = s[0][0] * c12[0] + s[0][1] * c12[1] + s[0][2] * c12[2];
            const int sigma = vol > 0.0 ? 1 : (vol < 0.0 ? -1 : 0);
            if (sigma == 0) continue;
            if (!edge_in(e[0], g.id[0], g.id[1], sigma) || !edge_in(e[1], g.id[1], g.id[2], sigma) ||
                !edge_in(e[2], g.id[2], g.id[0], sigma))
                continue;
            const uint32_t* f = g.f;
            const bool ok = flag_nf(f[0]) == flag_nf(f[1]) && flag_nf(f[1]) == flag_nf(f[2]) &&
                            ((f[0] ^ f[1]) & kFlagOrient) == 0 && ((f[1] ^ f[2]) & kFlagOrient) == 0 &&
                            ((f[0] | f[1] | f[2]) & kFlagCaustic) == 0 && sigma == ((f[0] & kFlagOrient) ? 1 : -1);
            if (!ok) {
                atomicOr(a.mask + (long long)c.orel * b.ndir + dk, caustic_bits(c.p));
                continue;
            }
        }
        double F[3][6], psi[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const long long i = base + g.id[v];
            const double2 fx = a.st.Fx[i], fy = a.st.Fy[i], fz = a.st.Fz[i];
            F[v][0] = fx.x; F[v][1] = fx.y; F[v][2] = fy.x;
            F[v][3] = fy.y; F[v][4] = fz.x; F[v][5] = fz.y;
            psi[v] = a.st.s2psi[i].y;
        }
        const double inv = 1.0 / (e[0] + e[1] + e[2]);
        const double l0 = e[1] * inv, l1 = e[2] * inv, l2 = e[0] * inv;
        double Fi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Fi[k] = l0 * F[0][k] + l1 * F[1][k] + l2 * F[2][k];
        double ps = l0 * psi[0] + l1 * psi[1] + l2 * psi[2];
        if constexpr (kNewton) {
            // exact ray of this branch from the interpolated impact point (the same weights)
            double xs = 0.0, ys = 0.0;
            const double lw[3] = {l0, l1, l2};
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                double xv, yv;
                ray_origin(*c.o, g.id[v], xv, yv);
                xs += lw[v] * xv;
                ys += lw[v] * yv;
            }
            FarRecord fr;
            if (newton_point(*c.o, p, x, xs, ys, 8.0 * c.o->h, fr)) {
#pragma unroll
                for (int k = 0; k < 6; ++k) Fi[k] = fr.F[k];
                ps = fr.psi;
            } else if (a.nfail) {
                atomicAdd(a.nfail, 1ull);
            }
        }
        const double eth[3] = {ct * cp, ct * sp, -sth};
        const double eph[3] = {-sp, cp, 0.0};
        if (a.st.near_r > 0.0) {
            double* dst = a.out + (((long long)c.orel * b.ndir + dk) * b.nout + (a.per_order ? p : 0)) * 6;
            add_contribution_reduced3(Fi, ps, x, eth, eph, dst);
        } else {
            double* dst = a.out + (((long long)c.orel * b.ndir + dk) * b.nout + (a.per_order ? p : 0)) * 4;
            add_contribution_reduced(Fi, ps, eth, eph, dst);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// fan: in-plane exit angles, folds, physical-optics windows
// ---------------------------------------------------------------------------------------------
struct FanScales {
    double po_full, po_end, ap_full, ap_end;
};

__device__ __forceinline__ FanScales fan_scales(const ObjDev& o)
{
    // Airy width (lambda/L)^(2/3) and Fresnel width 1/sqrt(k0 L) of the centre aperture plane
    const double aw = pow(o.lambda / o.lmax, 2.0 / 3.0), fw = 1.0 / sqrt(o.k0 * o.lmax);
    FanScales s;
    s.po_full = 1.5 * aw;
    s.po_end = 3.0 * aw;
    s.ap_full = 3.0 * aw + 3.0 * fw;
    s.ap_end = 3.0 * aw + 6.0 * fw;
    return s;
}

__device__ __forceinline__ double fan_alpha(const RaysDev& st, long long i, double efx, double efy)
{
    double s[3];
    load_dir(st, i, s);
    return atan2(s[0] * efx + s[1] * efy, s[2]);
}

// alpha of every (order, ray) of the fan, NaN where invalid
__global__ void fan_alpha_kernel(FieldArgs a, long long nrays, double efx, double efy, double* alpha)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nrays * (a.pmax + 1)) return;
    const int p = (int)(t / nrays);
    const long long j = t - (long long)p * nrays;
    const long long i = (long long)p * a.st.R + a.d_obj->ray_offset + j;
    alpha[t] = (a.st.flags[i] & kFlagValid) ? fan_alpha(a.st, i, efx, efy) : CUDART_NAN;
}

__global__ void fan_fold_kernel(FieldArgs a, long long nrays, const double* alpha, PoWindow* win, int* nwin)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nrays * (a.pmax + 1)) return;
    const int p = (int)(t / nrays);
    const long long j = t - (long long)p * nrays;
    if (p < 1 || j < 1 || j + 1 >= nrays) return;
    const double am = alpha[t - 1], a0 = alpha[t], ap = alpha[t + 1];
    if (isnan(am) || isnan(a0) || isnan(ap)) return;
    const double d0 = wrap_angle(a0 - am), d1 = wrap_angle(ap - a0);
    if (!(d0 * d1 < 0.0)) return;
    const int slot = atomicAdd(nwin, 1);
    if (slot >= kMaxPoWindows) {
        atomicOr(a.status, kStatusCapacity);
        return;
    }
    win[slot].p = p;
    win[slot].jc = j;
}

// one block: sort the folds by (order, ray) and walk every window along the fan
__global__ void fan_walk_kernel(FieldArgs a, long long nrays, const double* alpha, PoWindow* win, int* nwin)
{
    const ObjDev& o = *a.d_obj;
    const int n = min(*nwin, kMaxPoWindows);
    if (threadIdx.x == 0) {
        for (int i = 1; i < n; ++i) {
            PoWindow w = win[i];
            int k = i - 1;
            while (k >= 0 && (win[k].p > w.p || (win[k].p == w.p && win[k].jc > w.jc))) {
                win[k + 1] = win[k];
                --k;
            }
            win[k + 1] = w;
        }
        *nwin = n;
    }
    __syncthreads();
    const FanScales sc = fan_scales(o);
    for (int w = threadIdx.x; w < n; w += blockDim.x) {
        PoWindow& wv = win[w];
        const double* al = alpha + (long long)wv.p * nrays;
        const long long j = wv.jc;
        const double d0 = wrap_angle(al[j] - al[j - 1]), d1 = wrap_angle(al[j + 1] - al[j]);
        wv.alpha_c = al[j];
        long long lo = j, hi = j;
        while (lo - 1 >= 0 && !isnan(al[lo - 1]) && fabs(wrap_angle(al[lo - 1] - wv.alpha_c)) < sc.ap_end &&
               fabs(al[lo - 1] - al[lo]) < kPi && (al[lo - 1] - al[lo]) * d0 < 0.0)
            --lo;
        while (hi + 1 < nrays && !isnan(al[hi + 1]) && fabs(wrap_angle(al[hi + 1] - wv.alpha_c)) < sc.ap_end &&
               fabs(al[hi + 1] - al[hi]) < kPi && (al[hi + 1] - al[hi]) * d1 > 0.0)
            ++hi;
        wv.jlo = lo;
        wv.jhi = hi;
        wv.ok = (hi - lo + 1) >= 3;
        const long long i = (long long)wv.p * a.st.R + o.ray_offset + j;
        load_dir(a.st, i, wv.sc);
    }
}

// aperture field of every window ray: x_i (3) and U_i |dxi_i| (3 complex) -> ap[off + i] (9 slots)
__device__ bool aperture_point(const FieldArgs& a, const ObjDev& o, const PoWindow& wv, long long j, double efx,
                               double efy, double* x, double* xi)
{
    const long long n = (long long)a.st.np * a.st.R;
    const long long i = (long long)wv.p * a.st.R + o.ray_offset + j;
    const double* aux = a.st.aux + i;
    double s[3];
    load_dir(a.st, i, s);
    const double r[3] = {aux[kAuxRx * n], aux[kAuxRy * n], aux[kAuxRz * n]};
    const double dd[3] = {o.c[0] - r[0], o.c[1] - r[1], o.c[2] - r[2]};
    const double tau = (wv.sc[0] * dd[0] + wv.sc[1] * dd[1] + wv.sc[2] * dd[2]) /
                       (wv.sc[0] * s[0] + wv.sc[1] * s[1] + wv.sc[2] * s[2]);
    for (int c = 0; c < 3; ++c) x[c] = r[c] + tau * s[c];
    const double ca = cos(wv.alpha_c), sa = sin(wv.alpha_c);
    const double exi[3] = {ca * efx, ca * efy, -sa};
    *xi = exi[0] * (x[0] - o.c[0]) + exi[1] * (x[1] - o.c[1]) + exi[2] * (x[2] - o.c[2]);
    return true;
}

__global__ void fan_aperture_kernel(FieldArgs a, double efx, double efy, const double* alpha, long long nrays,
                                    const PoWindow* win, const int* nwin, const long long* offs, double* ap,
                                    long long ap_cap)
{
    const int w = blockIdx.y;
    if (w >= *nwin) return;
    const PoWindow wv = win[w];
    if (!wv.ok) return;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nw = wv.jhi - wv.jlo + 1;
    if (t >= nw) return;
    const long long slot = offs[w] + t;
    if (slot >= ap_cap) {
        atomicOr(a.status, kStatusCapacity);
        return;
    }
    const ObjDev& o = *a.d_obj;
    const FanScales sc = fan_scales(o);
    const long long j = wv.jlo + t;
    const long long n = (long long)a.st.np * a.st.R;
    const long long i = (long long)wv.p * a.st.R + o.ray_offset + j;
    const double* aux = a.st.aux + i;
    double x[3], xi, xn[3], xim = 0.0, xip = 0.0;
    aperture_point(a, o, wv, j, efx, efy, x, &xi);
    if (t > 0) aperture_point(a, o, wv, j - 1, efx, efy, xn, &xim);
    if (t + 1 < nw) aperture_point(a, o, wv, j + 1, efx, efy, xn, &xip);
    double dxi;
    if (t == 0) dxi = 0.5 * (xip - xi);
    else if (t == nw - 1) dxi = 0.5 * (xi - xim);
    else dxi = 0.5 * (xip - xim);
    // exit wave carried to the aperture line
    double s[3];
    load_dir(a.st, i, s);
    const double r[3] = {aux[kAuxRx * n], aux[kAuxRy * n], aux[kAuxRz * n]};
    const double tau = (x[0] - r[0]) * s[0] + (x[1] - r[1]) * s[1] + (x[2] - r[2]) * s[2];
    const double q11 = aux[kAuxQ11 * n], q12 = aux[kAuxQ12 * n], q22 = aux[kAuxQ22 * n];
    const double A11 = 1.0 + tau * q11, A22 = 1.0 + tau * q22, A12 = tau * q12;
    const double detA = A11 * A22 - A12 * A12;
    double* out = ap + 9 * slot;
    if (detA == 0.0) {
        for (int c = 0; c < 9; ++c) out[c] = 0.0;
        atomicOr(a.status, kStatusNumeric);
        return;
    }
    const int nfl = neg_eigs_sym(A11, A12, A22);
    const int nf_ap = (int)aux[kAuxNfLegs * n] + (tau > 0.0 ? nfl : -nfl);
    const double dq = q11 * q22 - q12 * q12;
    const double qa11 = (q11 + tau * dq) / detA, qa12 = q12 / detA, qa22 = (q22 + tau * dq) / detA;
    const double ep[3] = {aux[kAuxEpx * n], aux[kAuxEpy * n], aux[kAuxEpz * n]};
    const double v2[3] = {ep[1] * s[2] - ep[2] * s[1], ep[2] * s[0] - ep[0] * s[2], ep[0] * s[1] - ep[1] * s[0]};
    const double npl[3] = {efy, -efx, 0.0};  // normal of the fan plane
    const double c1 = npl[0] * ep[0] + npl[1] * ep[1] + npl[2] * ep[2];
    const double c2 = npl[0] * v2[0] + npl[1] * v2[1] + npl[2] * v2[2];
    const double qs = c1 * c1 * qa11 + 2.0 * c1 * c2 * qa12 + c2 * c2 * qa22;
    const double Rs = 1.0 / qs;
    const double dap = aux[kAuxDlegs * n] / fabs(detA);
    // amplitude sqrt(D) (-i)^nf e^{i k0 (L + tau)} times the sagittal factor sqrt|Rs| e^{i pi/4 sgn Rs}
    double ph = o.k0 * (aux[kAuxPath * n] + tau) - 0.5 * kPi * (double)nf_ap + (Rs > 0.0 ? 0.25 : -0.25) * kPi;
    double sph, cph;
    sincos(ph, &sph, &cph);
    const double tap = ramp(fabs(wrap_angle(alpha[(long long)wv.p * nrays + j] - wv.alpha_c)), sc.ap_full, sc.ap_end);
    const double mag = tap * sqrt(dap) * sqrt(fabs(Rs)) * fabs(dxi);
    const double E[6] = {aux[kAuxExr * n], aux[kAuxExi * n], aux[kAuxEyr * n],
                         aux[kAuxEyi * n], aux[kAuxEzr * n], aux[kAuxEzi * n]};
    out[0] = x[0];
    out[1] = x[1];
    out[2] = x[2];
    for (int c = 0; c < 3; ++c) {
        out[3 + 2 * c] = mag * (E[2 * c] * cph - E[2 * c + 1] * sph);
        out[4 + 2 * c] = mag * (E[2 * c] * sph + E[2 * c + 1] * cph);
    }
}

// target direction of an in-plane angle alpha and its (e_theta, e_phi)
__device__ __forceinline__ void plane_dir(double alk, double efx, double efy, double* d, double* eth, double* eph)
{
    const double th = fabs(alk);
    const double cph = alk >= 0.0 ? efx : -efx, sph = alk >= 0.0 ? efy : -efy;
    double st, ct;
    sincos(th, &st, &ct);
    d[0] = st * cph;
    d[1] = st * sph;
    d[2] = ct;
    eth[0] = ct * cph;
    eth[1] = ct * sph;
    eth[2] = -st;
    eph[0] = -sph;
    eph[1] = cph;
    eph[2] = 0.0;
}

// one block per (window, target direction): sum over the window's aperture samples
__global__ void __launch_bounds__(256) fan_po_kernel(FieldArgs a, double efx, double efy, int ndir, double alpha0,
                                                     double dalpha, const PoWindow* win, const int* nwin,
                                                     const long long* offs, const double* ap, long long ap_cap)
{
    const int w = blockIdx.y;
    if (w >= *nwin) return;
    const PoWindow wv = win[w];
    if (!wv.ok) return;
    if (offs[w] + (wv.jhi - wv.jlo + 1) > ap_cap) return;  // samples beyond capacity were not written
    const int k = blockIdx.x;
    const double alk = alpha0 + k * dalpha;
    const ObjDev& o = *a.d_obj;
    const FanScales sc = fan_scales(o);
    const double sblend = ramp(fabs(wrap_angle(alk - wv.alpha_c)), sc.po_full, sc.po_end);
    if (sblend == 0.0) return;
    double d[3], eth[3], eph[3];
    plane_dir(alk, efx, efy, d, eth, eph);
    const long long nw = wv.jhi - wv.jlo + 1;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long t = threadIdx.x; t < nw; t += blockDim.x) {
        const double* q = ap + 9 * (offs[w] + t);
        double sp, cp;
        sincos(-o.k0 * (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]), &sp, &cp);
        double tr = 0.0, ti = 0.0, pr = 0.0, pi = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double re = q[3 + 2 * c] * cp - q[4 + 2 * c] * sp;
            const double im = q[3 + 2 * c] * sp + q[4 + 2 * c] * cp;
            tr += re * eth[c];
            ti += im * eth[c];
            pr += re * eph[c];
            pi += im * eph[c];
        }
        acc[0] += tr;
        acc[1] += ti;
        acc[2] += pr;
        acc[3] += pi;
    }
    // warp shuffle reduction, then one partial per warp in shared memory
    __shared__ double red[4][32];
    for (int c = 0; c < 4; ++c) {
        double v = acc[c];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < 4; ++c)
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot[c] += red[c][i];
        // sqrt(k0 / 2 pi) (-i) times the blend weight
        const double pre = sqrt(o.k0 / (2.0 * kPi)) * sblend;
        const double r0 = pre * tot[1], i0 = -pre * tot[0];
        const double r1 = pre * tot[3], i1 = -pre * tot[2];
        double* dst = a.out + ((long long)k * (a.per_order ? (a.pmax + 1) : 1) + (a.per_order ? wv.p : 0)) * 4;
        atomicAdd(dst + 0, r0);
        atomicAdd(dst + 1, i0);
        atomicAdd(dst + 2, r1);
        atomicAdd(dst + 3, i1);
        atomicOr(a.mask + k, kMaskPo);
    }
}

// Newton on the exact double-precision trace (the definition the interpolation approximates):
// finds the impact parameter b of the fan ray of order p leaving at in-plane angle alpha_t, from
// the interpolated seed.  The derivative d alpha / d b comes from the transfer matrix carried
// through the trace: d s = Q' T (e_x, e_y) db in the exit basis (e_perp, e_perp x s).  At most 40
// steps (quadratic convergence takes 3 to 6), stop at |d alpha| < 1e-13.
__device__ bool newton_fan(const ObjDev& o, int p, double efx, double efy, double alpha_t, double b, FarRecord& out)
{
    for (int it = 0; it < 40; ++it) {
        CaptureSink cs;
        cs.want = p;
        cs.got = false;
        trace_ray<double, true>(o, o.c[0] + b * efx, o.c[1] + b * efy, p, cs);
        if (!cs.got) return false;
        FarRecord r;
        if (!far_record(o, cs.w, r)) return false;
        const double al = atan2(r.s[0] * efx + r.s[1] * efy, r.s[2]);
        const double da = wrap_angle(alpha_t - al);
        if (fabs(da) < 1e-13) {
            out = r;
            return true;
        }
        const ExitWave& w = cs.w;
        const double J00 = w.q11 * w.t11 + w.q12 * w.t21, J01 = w.q11 * w.t12 + w.q12 * w.t22;
        const double J10 = w.q12 * w.t11 + w.q22 * w.t21, J11 = w.q12 * w.t12 + w.q22 * w.t22;
        const double j0 = J00 * efx + J01 * efy, j1 = J10 * efx + J11 * efy;
        const double v2[3] = {w.ep[1] * w.k[2] - w.ep[2] * w.k[1], w.ep[2] * w.k[0] - w.ep[0] * w.k[2],
                              w.ep[0] * w.k[1] - w.ep[1] * w.k[0]};
        double sa, ca;
        sincos(al, &sa, &ca);
        const double ea[3] = {ca * efx, ca * efy, -sa};
        double dadb = 0.0;
        for (int c = 0; c < 3; ++c) dadb += (j0 * w.ep[c] + j1 * v2[c]) * ea[c];
        if (dadb == 0.0) return false;
        b += da / dadb;
    }
    return false;
}

// fan: one thread per (order, segment of neighbouring rays)
__global__ void __launch_bounds__(256) field_fan_kernel(FieldArgs a, long long nrays, double efx, double efy,
                                                        int ndir, double alpha0, double dalpha,
                                                        const PoWindow* win, const int* nwin_p, int po,
                                                        int newton)
{
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nseg = nrays - 1;
    if (nseg <= 0 || tid >= nseg * (a.pmax + 1)) return;
    const int p = (int)(tid / nseg);
    const long long j = tid - (long long)p * nseg;
    const ObjDev& o = *a.d_obj;
    const long long ia = (long long)p * a.st.R + o.ray_offset + j, ib = ia + 1;
    const uint32_t fa = a.st.flags[ia], fb = a.st.flags[ib];
    if (!(fa & fb & kFlagValid)) return;
    const bool consistent = flag_nf(fa) == flag_nf(fb) && ((fa ^ fb) & kFlagOrient) == 0 &&
                            ((fa | fb) & kFlagCaustic) == 0;
    const double al_a = fan_alpha(a.st, ia, efx, efy), al_b = fan_alpha(a.st, ib, efx, efy);
    const double da = wrap_angle(al_b - al_a);
    if (da == 0.0) return;
    int wi = -1;
    const int nwin = nwin_p ? *nwin_p : 0;
    if (po)
        for (int w = 0; w < nwin; ++w)
            if (win[w].ok && win[w].p == p && j >= win[w].jlo && j + 1 <= win[w].jhi) wi = w;
    const FanScales sc = fan_scales(o);
    const double lo = fmin(al_a, al_a + da), hi = fmax(al_a, al_a + da);
    bool loaded = false;
    double Fa[6], Fb[6], pa = 0.0, pb = 0.0;
    for (int sh = -1; sh <= 1; ++sh) {
        const double shift = sh * 2.0 * kPi;
        long long k0 = (long long)ceil((lo + shift - alpha0) / dalpha) - 1;
        long long k1 = (long long)floor((hi + shift - alpha0) / dalpha) + 1;
        if (k0 < 0) k0 = 0;
        if (k1 > ndir - 1) k1 = ndir - 1;
        for (long long k = k0; k <= k1; ++k) {
            const double alk = alpha0 + k * dalpha;
            const double lam = wrap_angle(alk - al_a) / da;
            if (!(lam >= 0.0 && lam < 1.0)) continue;
            if (!consistent) {
                if (wi < 0) atomicOr(a.mask + k, kMaskCaustic);
                continue;
            }
            double wgo = 1.0;
            if (wi >= 0) wgo = 1.0 - ramp(fabs(wrap_angle(alk - win[wi].alpha_c)), sc.po_full, sc.po_end);
            if (wgo == 0.0) continue;
            if (!loaded) {
                const double2 xa = a.st.Fx[ia], ya = a.st.Fy[ia], za = a.st.Fz[ia];
                const double2 xb = a.st.Fx[ib], yb = a.st.Fy[ib], zb = a.st.Fz[ib];
                Fa[0] = xa.x; Fa[1] = xa.y; Fa[2] = ya.x; Fa[3] = ya.y; Fa[4] = za.x; Fa[5] = za.y;
                Fb[0] = xb.x; Fb[1] = xb.y; Fb[2] = yb.x; Fb[3] = yb.y; Fb[4] = zb.x; Fb[5] = zb.y;
                pa = a.st.s2psi[ia].y;
                pb = a.st.s2psi[ib].y;
                loaded = true;
            }
            double F[6];
            for (int c = 0; c < 6; ++c) F[c] = (1.0 - lam) * Fa[c] + lam * Fb[c];
            double ps = (1.0 - lam) * pa + lam * pb;
            // Newton on the exact trace: every hit, or the hits within 2 deg of a fold of this order
            bool exact = newton == 1;
            if (newton == 2)
                for (int w = 0; w < nwin && !exact; ++w)
                    if (win[w].p == p && fabs(wrap_angle(alk - win[w].alpha_c)) < kFoldNewtonWindow) exact = true;
            if (exact) {
                const double bj = -o.fan_w + ((double)j + 0.5) * o.h;
                FarRecord fr;
                if (newton_fan(o, p, efx, efy, alk, bj + lam * o.h, fr)) {
                    for (int c = 0; c < 6; ++c) F[c] = fr.F[c];
                    ps = fr.psi;
                } else {
                    if (a.nfail) atomicAdd(a.nfail, 1ull);
                }
            }
            double d[3], eth[3], eph[3];
            plane_dir(alk, efx, efy, d, eth, eph);
            double* dst = a.out + (k * (a.per_order ? (a.pmax + 1) : 1) + (a.per_order ? p : 0)) * 4;
            add_contribution(F, ps, eth, eph, wgo, dst);
        }
    }
}

__global__ void window_prefix_kernel(const PoWindow* win, const int* nwin, long long* offs)
{
    long long o = 0;
    const int n = *nwin;
    for (int w = 0; w < n; ++w) {
        offs[w] = o;
        o += win[w].ok ? (win[w].jhi - win[w].jlo + 1) : 0;
    }
    offs[n] = o;
}

// per-object cell windows and thread offsets of a grid launch (one thread; the group is small)
__global__ void grid_cells_kernel(const ObjDev* objs, int n, int np, int windowed, long long wx0, long long wx1,
                                  long long wy0, long long wy1, GridCells* cells)
{
    long long first = 0;
    for (int i = 0; i < n; ++i) {
        const ObjDev& o = objs[i];
        long long ix0 = 0, ix1 = o.nx - 1, iy0 = 0, iy1 = o.ny - 1;
        if (windowed) {
            ix0 = wx0 < 0 ? 0 : wx0;
            ix1 = wx1 > o.nx - 1 ? o.nx - 1 : wx1;
            iy0 = wy0 < 0 ? 0 : wy0;
            iy1 = wy1 > o.ny - 1 ? o.ny - 1 : wy1;
        }
        GridCells c;
        c.ix0 = ix0;
        c.iy0 = iy0;
        c.ncx = ix1 - ix0 > 0 ? ix1 - ix0 : 0;
        c.ncy = iy1 - iy0 > 0 ? iy1 - iy0 : 0;
        c.first = first;
        first += c.ncx * c.ncy * np;
        cells[i] = c;
    }
}

__global__ void finalize_mask_kernel(const unsigned int* words, unsigned char* mask_out, const ObjDev* objs, int nobj,
                                     long long ndir, int kind, int nt, int nph, double alpha0, double dalpha,
                                     const double* list)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ndir * nobj) return;
    const int oi = (int)(t / ndir);
    const long long d = t - (long long)oi * ndir;
    const double axial = 2.0 * objs[oi].lambda / objs[oi].lmin;
    double th;
    if (kind == 0) {
        th = fabs(alpha0 + d * dalpha);
    } else if (kind == 1) {
        const int it = (int)(d / nph);
        th = (it + 0.5) * (kPi / nt);
    } else {
        th = acos(fmin(1.0, fmax(-1.0, cos(list[2 * d]))));  // polar angle of the listed direction
    }
    unsigned int m = words[t];
    if (th < axial || th > kPi - axial) m |= kMaskAxial;
    mask_out[t] = (unsigned char)m;
}

// unit vector (double cos/sin pairs and single-precision xyz) and bin of every listed direction
__global__ void list_prep_kernel(const double* __restrict__ list, long long n, int nt, int nph, double* ldir,
                                 float4* ldir_f, int* binid, int* count)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double th = list[2 * i], ph = list[2 * i + 1];
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    ldir[4 * i] = ct;
    ldir[4 * i + 1] = st;
    ldir[4 * i + 2] = cp;
    ldir[4 * i + 3] = sp;
    const double x = st * cp, y = st * sp;
    ldir_f[i] = make_float4((float)x, (float)y, (float)ct, 0.0f);
    // bin of the direction itself (theta in [0, pi], phi in [-pi, pi))
    const double tq = atan2(sqrt(x * x + y * y), ct), pq = atan2(y, x);
    int it = (int)floor(tq * nt / kPi), jp = (int)floor((pq + kPi) * nph / (2.0 * kPi));
    it = it < 0 ? 0 : (it >= nt ? nt - 1 : it);
    jp = jp < 0 ? 0 : (jp >= nph ? nph - 1 : jp);
    const int b = it * nph + jp;
    binid[i] = b;
    atomicAdd(count + b, 1);
}

// exclusive prefix of count[0, n) into first[0, n] (one block; n up to a few million)
__global__ void __launch_bounds__(1024) list_scan_kernel(const int* __restrict__ count, int n, int* __restrict__ first)
{
    __shared__ int part[1024];
    const int t = threadIdx.x, per = (n + 1023) / 1024;
    const int lo = min(t * per, n), hi = min(lo + per, n);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += count[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = lo; i < hi; ++i) {
        first[i] = run;
        run += count[i];
    }
    if (t == 1023) first[n] = part[1023];
}

__global__ void list_fill_kernel(const int* __restrict__ binid, long long n, const int* __restrict__ first,
                                 int* cursor, int* __restrict__ bin_dir)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = binid[i];
    bin_dir[first[b] + atomicAdd(cursor + b, 1)] = (int)i;
}

// ---------------------------------------------------------------------------------------------
// square grid: summing the hits.  One thread per hit, in the order of the hit list (the order of the
// classified cells on the ray grid, so that neighbouring hits share corner records in the caches):
// the hit is decided and interpolated, and its contribution F e^{i Psi} is added to its direction's
// words as 64-bit fixed-point numbers by integer atomics; a last pass turns the words into doubles.
// Integer sums do not depend on their order, so the field is the same bit for bit from run to run.
// (Sorting the hits by tile of 8 x 16 directions and summing each tile in shared memory gives the
// same words and took 0.42 ms longer on the 4e6-ray ellipsoid: the sort's passes cost more than the
// atomics they save, and the tile order scatters the corner reads.)  On GB300 the double-precision
// pipe (which also converts between precisions) issues 1.6 operations per clock per SM, against 128
// for single precision: the edge planes of a hit are double-float (pairs of floats, error-free
// products and sums), F is interpolated in single precision from corner values narrowed in the
// integer pipe (f64_to_f32_int), and double precision is kept for the phase (about ten operations
// per hit).
// ---------------------------------------------------------------------------------------------
// fixed point: a value v with |v| < 2^eB (eB the bound of the object's |F|) is stored as
// round(v 2^(46 - eB)); 2^16 such values add without leaving the 63-bit range
constexpr int kFixBits = 46;

// ---- double-float pieces ----
struct F2 {
    float h, l;
};

// a b as an unevaluated pair: the rounded product, then its error and the products with the low parts
__device__ __forceinline__ F2 df_mul(float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    return F2{p, e};
}

// component k of a x b (a_y b_z - a_z b_y and cyclic), a and b given as hi + lo
__device__ __forceinline__ F2 df_cross_k(const float* ah, const float* al, const float* bh, const float* bl, int k)
{
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    const F2 p = df_mul(ah[i], al[i], bh[j], bl[j]);
    const F2 q = df_mul(ah[j], al[j], bh[i], bl[i]);
    float s, e;
    df_two_sum(p.h, -q.h, s, e);
    e = __fadd_rn(e, __fsub_rn(p.l, q.l));
    df_fast_two_sum(s, e, s, e);
    return F2{s, e};
}

// n . x as a normalised pair (n and x given as hi + lo)
__device__ __forceinline__ F2 df_dot(const float* nh, const float* nl, const float* xh, const float* xl)
{
    float s = 0.0f, t = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const F2 p = df_mul(nh[c], nl[c], xh[c], xl[c]);
        float u, e;
        df_two_sum(s, p.h, u, e);
        s = u;
        t = __fadd_rn(t, __fadd_rn(e, p.l));
    }
    df_fast_two_sum(s, t, s, t);
    return F2{s, t};
}


// v 2^k rounded to an integer (|v| 2^k < 2^62), in the integer pipe
__device__ __forceinline__ unsigned long long to_fixed(float v, int k)
{
    const unsigned int u = __float_as_uint(v);
    const int ex = (int)((u >> 23) & 0xffu);
    if (ex == 0) return 0ull;
    const unsigned long long m = (unsigned long long)((u & 0x7fffffu) | 0x800000u);
    const int sh = ex - 127 - 23 + k;
    long long r;
    if (sh >= 0) r = (long long)(m << sh);
    else if (sh > -26) r = (long long)((m + (1ull << (-sh - 1))) >> -sh);
    else r = 0;
    return (unsigned long long)((u >> 31) ? -r : r);
}

// fixed-point exponent of object orel: kFixBits - e with max |F| < 2^e
__device__ __forceinline__ int fix_exponent(const unsigned int* fmax, int orel)
{
    const float b2 = __uint_as_float(fmax[orel]);
    if (!(b2 > 0.0f)) return 0;
    int eb;
    frexpf(sqrtf(b2) * 1.0000005f, &eb);
    return kFixBits - eb;
}

// One hit: the exact test of a close call, the weights, F and Psi interpolated, F e^{i Psi} added to
// the kNc fixed-point words at dst (scale 2^kfix); a singular cell marks the direction instead.
template <int kNc>
__device__ __forceinline__ void sum_hit(const FieldArgs& a, const GridBatch& b, const DirSet& d, const float* lt,
                                        unsigned long long code, unsigned int dw, int kfix, unsigned long long* dst)
{
    const bool close = (dw & kHitClose) != 0;
    const unsigned int dk = dw & ~kHitClose;
    const CellRef c = decode_cell(a, b, (long long)(code >> 1));
    TriGeom g;
    load_triangle(a, c.base, c.nx, c.cx, c.cy, (int)(code & 1ull), g);
    // the direction (hi + lo) and its e_theta, e_phi
    float xh[3], xl[3], eth[3], eph[3];
    if (d.list) {
        const double* qd = d.ldir + 4 * (long long)dk;
        const double ct = qd[0], st = qd[1], cp = qd[2], sp = qd[3];
        const double x[3] = {st * cp, st * sp, ct};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            xh[k] = f64_to_f32_int(x[k]);
            xl[k] = f64_to_f32_int(x[k] - f32_to_f64_int(xh[k]));
        }
        const float ctf = f64_to_f32_int(ct), stf = f64_to_f32_int(st), cpf = f64_to_f32_int(cp),
                    spf = f64_to_f32_int(sp);
        eth[0] = ctf * cpf;
        eth[1] = ctf * spf;
        eth[2] = -stf;
        eph[0] = -spf;
        eph[1] = cpf;
        eph[2] = 0.0f;
    } else {
        const int nt = d.nt, nph = d.nph;
        const int it = (int)(dk / (unsigned int)nph), jp = (int)(dk - (unsigned int)it * nph);
        const float* ft = reinterpret_cast<const float*>(d.tab + 2 * (nt + nph));
        const float cth = ft[it], sth = ft[nt + it], cph = ft[2 * nt + jp], sph = ft[2 * nt + nph + jp];
        const float ctl = lt[it], stl = lt[nt + it], cpl = lt[2 * nt + jp], spl = lt[2 * nt + nph + jp];
        const F2 xx = df_mul(sth, stl, cph, cpl), xy = df_mul(sth, stl, sph, spl);
        xh[0] = xx.h;
        xl[0] = xx.l;
        xh[1] = xy.h;
        xl[1] = xy.l;
        xh[2] = cth;
        xl[2] = ctl;
        eth[0] = cth * cph;
        eth[1] = cth * sph;
        eth[2] = -sth;
        eph[0] = -sph;
        eph[1] = cph;
        eph[2] = 0.0f;
    }
    // edge planes with their endpoints in index order (both triangles of an edge evaluate the same
    // plane), double-float values at the direction
    F2 e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int va = k, vb = (k + 1) % 3;
        const bool fwd = g.id[va] < g.id[vb];
        float ah[3], al[3], bh[3], bl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            ah[r] = fwd ? g.s[va][r] : g.s[vb][r];
            al[r] = fwd ? g.l[va][r] : g.l[vb][r];
            bh[r] = fwd ? g.s[vb][r] : g.s[va][r];
            bl[r] = fwd ? g.l[vb][r] : g.l[va][r];
        }
        float nh[3], nl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const F2 n = df_cross_k(ah, al, bh, bl, r);
            nh[r] = n.h;
            nl[r] = n.l;
        }
        e[k] = df_dot(nh, nl, xh, xl);
        if (!fwd) {
            e[k].h = -e[k].h;
            e[k].l = -e[k].l;
        }
    }
    if (close) {
        // orientation s0 . (s1 x s2), then the half-open rule (edge_in) in double-float
        float nh[3], nl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const F2 n = df_cross_k(g.s[1], g.l[1], g.s[2], g.l[2], r);
            nh[r] = n.h;
            nl[r] = n.l;
        }
        const F2 v = df_dot(nh, nl, g.s[0], g.l[0]);
        const int sigma = v.h > 0.0f ? 1 : (v.h < 0.0f ? -1 : 0);
        if (sigma == 0) return;
        auto in = [&](const F2& ev, long long ia, long long ib) {
            const float se = sigma > 0 ? ev.h : -ev.h;
            if (se > 0.0f) return true;
            if (se < 0.0f) return false;
            return (ia < ib) == (sigma > 0);
        };
        if (!in(e[0], g.id[0], g.id[1]) || !in(e[1], g.id[1], g.id[2]) || !in(e[2], g.id[2], g.id[0])) return;
        const uint32_t* f = g.f;
        const bool ok = flag_nf(f[0]) == flag_nf(f[1]) && flag_nf(f[1]) == flag_nf(f[2]) &&
                        ((f[0] ^ f[1]) & kFlagOrient) == 0 && ((f[1] ^ f[2]) & kFlagOrient) == 0 &&
                        ((f[0] | f[1] | f[2]) & kFlagCaustic) == 0 && sigma == ((f[0] & kFlagOrient) ? 1 : -1);
        if (!ok) {
            atomicOr(a.mask + (long long)c.orel * b.ndir + dk, caustic_bits(c.p));
            return;
        }
    }
    // weights of the central projection: l0 = e12 / S, l1 = e20 / S, l2 = e01 / S, S their sum
    const df S = df(e[0].h, e[0].l) + df(e[1].h, e[1].l) + df(e[2].h, e[2].l);
    const df w1 = df(e[2].h, e[2].l) / S, w2 = df(e[0].h, e[0].l) / S;
    const float l1 = w1.hi, l2 = w2.hi, l0 = 1.0f - l1 - l2;
    // corner F and Psi from the field records
    float Fi[6];
    df P[3];
    {
        float F[3][6];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const long long i = c.base + g.id[v];
            const float4 r0 = a.st.fval[2 * i], r1 = a.st.fval[2 * i + 1];
            F[v][0] = r0.z;
            F[v][1] = r0.w;
            F[v][2] = r1.x;
            F[v][3] = r1.y;
            F[v][4] = r1.z;
            F[v][5] = r1.w;
            P[v] = df(r0.x, r0.y);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) Fi[k] = l0 * F[0][k] + l1 * F[1][k] + l2 * F[2][k];
    }
    // Psi_0 + l1 (Psi_1 - Psi_0) + l2 (Psi_2 - Psi_0), reduced modulo 2 pi, in double-float
    const df psi = P[0] + w1 * (P[1] - P[0]) + w2 * (P[2] - P[0]);
    const float nturn = rintf(psi.hi * 0.159154943f);
    const df red = psi - df_mul_f(df(6.28318548f, -1.74845553e-7f), nturn);
    float sp, cp;
    sincosf(red.hi + red.lo, &sp, &cp);
    float rr = 0.0f, ri = 0.0f, tr = 0.0f, ti = 0.0f, pr = 0.0f, pi = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float re = Fi[2 * k] * cp - Fi[2 * k + 1] * sp;
        const float im = Fi[2 * k] * sp + Fi[2 * k + 1] * cp;
        tr += re * eth[k];
        ti += im * eth[k];
        pr += re * eph[k];
        pi += im * eph[k];
        if constexpr (kNc == 6) {
            rr += re * xh[k];
            ri += im * xh[k];
        }
    }
    if constexpr (kNc == 6) {
        atomicAdd(dst + 0, to_fixed(rr, kfix));
        atomicAdd(dst + 1, to_fixed(ri, kfix));
        dst += 2;
    }
    atomicAdd(dst + 0, to_fixed(tr, kfix));
    atomicAdd(dst + 1, to_fixed(ti, kfix));
    atomicAdd(dst + 2, to_fixed(pr, kfix));
    atomicAdd(dst + 3, to_fixed(pi, kfix));
}

// The hits of the list, a thread each, added to their directions' fixed-point words.
template <int kNc>
__global__ void __launch_bounds__(256, 3) hit_sum_kernel(FieldArgs a, GridBatch b, DirSet d, HitArgs h,
                                                         const unsigned int* fmax)
{
    const unsigned int n = min(*h.n, h.cap);
    const float* lt = reinterpret_cast<const float*>(d.tab + 2 * (d.nt + d.nph)) + 2 * (d.nt + d.nph);
    unsigned long long* out = reinterpret_cast<unsigned long long*>(a.out);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long code = h.tri[i];
        const unsigned int dw = h.dir[i];
        const CellRef c = decode_cell(a, b, (long long)(code >> 1));
        const long long dk = (long long)(dw & ~kHitClose);
        unsigned long long* dst = out + (((long long)c.orel * b.ndir + dk) * b.nout + (a.per_order ? c.p : 0)) * kNc;
        sum_hit<kNc>(a, b, d, lt, code, dw, fix_exponent(fmax, c.orel), dst);
    }
}

// fixed-point words of the launch's objects to doubles, in place
__global__ void tile_convert_kernel(double* out, long long per_obj, long long n, const unsigned int* fmax)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long v = __double_as_longlong(out[i]);
    if (!v) return;
    // 2^-k as a double built from its exponent field (|k| well below 1000)
    const int k = fix_exponent(fmax, (int)(i / per_obj));
    out[i] = (double)v * __longlong_as_double((long long)(1023 - k) << 52);
}

}  // namespace

cudaError_t launch_field_convert(double* out, long long per_obj, int nobj, const unsigned int* fmax, cudaStream_t s)
{
    const long long n = per_obj * nobj;
    if (n <= 0) return cudaSuccess;
    tile_convert_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, per_obj, n, fmax);
    return cudaGetLastError();
}

cudaError_t launch_bin_dirs(const double* list, long long n, int nt, int nph, double* ldir, float4* ldir_f,
                            int* binid, int* count, int* first, int* cursor, int* bin_dir, cudaStream_t s)
{
    const int nb = nt * nph;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(nb + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)(nb + 1), s);
    if (e != cudaSuccess || n <= 0) return e;
    const unsigned g = (unsigned)((n + 255) / 256);
    list_prep_kernel<<<g, 256, 0, s>>>(list, n, nt, nph, ldir, ldir_f, binid, count);
    list_scan_kernel<<<1, 1024, 0, s>>>(count, nb, first);
    list_fill_kernel<<<g, 256, 0, s>>>(binid, n, first, cursor, bin_dir);
    return cudaGetLastError();
}

cudaError_t launch_dir_tables(int nt, int nph, double* tab, cudaStream_t s)
{
    const int n = nt > nph ? nt : nph;
    dir_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(nt, nph, tab);
    return cudaGetLastError();
}

cudaError_t launch_field_grid(const FieldArgs& a, const GridBatch& b, const DirSet& d, unsigned long long* big,
                              unsigned int* nbig, unsigned int big_cap, unsigned long long* hit_tri,
                              unsigned int* hit_dir, unsigned int* nhit, unsigned int hit_cap, int classify_block,
                              int newton, cudaStream_t s, int stage, const unsigned int* fmax)
{
    if (b.total <= 0) return cudaSuccess;
    const int bs = 256;
    const int cb = classify_block > 0 ? classify_block : bs;
    HitArgs h{hit_tri, hit_dir, nhit, hit_cap, stage == kFieldClassify ? 0 : 1};
    // fixed grids walk the lists: 32 blocks per SM for the large triangles, 16 for the hits (8 for the
    // fixed-point sums, measured best of 8 to 64)
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (stage != 2) {
        cudaError_t e = cudaMemsetAsync(nbig, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(nhit, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
        field_grid_kernel<<<(unsigned)((b.total + cb - 1) / cb), cb, 0, s>>>(a, b, d, big, nbig, big_cap, h);
        field_grid_big_kernel<<<(unsigned)(32 * sms), 32 * kBigWarps, 0, s>>>(a, b, d, big, nbig, big_cap, h);
    }
    if (stage != 1) {
        if (newton) {
            field_grid_hit_kernel<true><<<(unsigned)(16 * sms), bs, 0, s>>>(a, b, d, h);
        } else if (!fmax) {
            field_grid_hit_kernel<false><<<(unsigned)(16 * sms), bs, 0, s>>>(a, b, d, h);
        } else if (a.st.near_r > 0.0) {
            // fixed-point sums (the words turn into doubles in launch_field_convert once the launch
            // group is complete)
            hit_sum_kernel<6><<<(unsigned)(8 * sms), 256, 0, s>>>(a, b, d, h, fmax);
        } else {
            hit_sum_kernel<4><<<(unsigned)(8 * sms), 256, 0, s>>>(a, b, d, h, fmax);
        }
    }
    return cudaGetLastError();
}

// the fan path: alpha table, folds and windows (when PO or Newton near folds), aperture fields
// (when PO), the segments, then the PO sums
cudaError_t launch_field_fan(const FieldArgs& a, long long nrays, double fan_phi, int ndir, double alpha0,
                             double dalpha, PoWindow* d_win, int* d_nwin, double2* d_scratch, long long ap_cap, int po,
                             int newton, cudaStream_t s)
{
    const long long nseg = (nrays - 1) * (a.pmax + 1);
    if (nseg <= 0) return cudaSuccess;
    const double efx = cos(fan_phi), efy = sin(fan_phi);
    const int bs = 256;
    const bool folds = po || newton == 2;
    const long long nt = nrays * (a.pmax + 1);
    double* alpha = reinterpret_cast<double*>(d_scratch);
    long long* offs = reinterpret_cast<long long*>(alpha + nt);
    double* ap = reinterpret_cast<double*>(offs + kMaxPoWindows + 1);
    if (folds) {
        cudaError_t e = cudaMemsetAsync(d_nwin, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        fan_alpha_kernel<<<(unsigned)((nt + bs - 1) / bs), bs, 0, s>>>(a, nrays, efx, efy, alpha);
        fan_fold_kernel<<<(unsigned)((nt + bs - 1) / bs), bs, 0, s>>>(a, nrays, alpha, d_win, d_nwin);
        fan_walk_kernel<<<1, 64, 0, s>>>(a, nrays, alpha, d_win, d_nwin);
    }
    if (po) {
        window_prefix_kernel<<<1, 1, 0, s>>>(d_win, d_nwin, offs);
        dim3 g1((unsigned)((nrays + bs - 1) / bs), kMaxPoWindows);
        fan_aperture_kernel<<<g1, bs, 0, s>>>(a, efx, efy, alpha, nrays, d_win, d_nwin, offs, ap, ap_cap);
    }
    field_fan_kernel<<<(unsigned)((nseg + bs - 1) / bs), bs, 0, s>>>(
        a, nrays, efx, efy, ndir, alpha0, dalpha, folds ? d_win : nullptr, folds ? d_nwin : nullptr, po ? 1 : 0, newton);
    if (po) {
        dim3 g2((unsigned)ndir, kMaxPoWindows);
        fan_po_kernel<<<g2, 256, 0, s>>>(a, efx, efy, ndir, alpha0, dalpha, d_win, d_nwin, offs, ap, ap_cap);
    }
    return cudaGetLastError();
}

cudaError_t launch_grid_cells(const ObjDev* objs, int n, int np, bool windowed, const int64_t* win, GridCells* cells,
                              cudaStream_t s)
{
    grid_cells_kernel<<<1, 1, 0, s>>>(objs, n, np, windowed ? 1 : 0, windowed ? win[0] : 0, windowed ? win[1] : 0,
                                      windowed ? win[2] : 0, windowed ? win[3] : 0, cells);
    return cudaGetLastError();
}

cudaError_t launch_finalize_mask(const unsigned int* words, unsigned char* mask_out, const ObjDev* objs, int nobj,
                                 long long ndir, int kind, int nt, int nph, double alpha0, double dalpha, cudaStream_t s,
                                 const double* list)
{
    if (!mask_out || ndir == 0 || nobj == 0) return cudaSuccess;
    const long long n = ndir * nobj;
    finalize_mask_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(words, mask_out, objs, nobj, ndir, kind, nt, nph,
                                                                      alpha0, dalpha, list);
    return cudaGetLastError();
}

}  // namespace rtw
