// rtw_api.cu -- host side of the C ABI declared in include/rtw.h.
//
// Argument validation, object tables, ray-grid layout, device allocations and kernel launches.
// No compute happens on the host: every step of the path runs in the kernels of rtw_trace.cu and
// rtw_field.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "rtw.h"
#include "rtw_host.h"
#include "rtw_launch.h"

using rtw::ObjDev;
using rtw::RaysDev;
using rtw::host::align_up;
using rtw::host::cuda_fail;
using rtw::host::fail;
using rtw::host::ObjHost;
using rtw::host::newton_counter;
using rtw::host::status_word;

namespace {
constexpr double kPi = 3.14159265358979323846;
thread_local std::string g_last_error;
std::mutex g_status_mu;
std::vector<unsigned int*> g_status;
}  // namespace

namespace rtw {

void set_last_error(const char* msg) { g_last_error = msg; }

namespace host {

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) { return fail(RTW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e)); }

// 16 bytes per device: the status word, then (at byte 8) the Newton failure counter
unsigned int* status_word(int dev)
{
    std::lock_guard<std::mutex> lk(g_status_mu);
    if ((int)g_status.size() <= dev) g_status.resize(dev + 1, nullptr);
    if (!g_status[dev]) {
        unsigned int* p = nullptr;
        if (cudaMalloc(&p, 16) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, 16);
        g_status[dev] = p;
    }
    return g_status[dev];
}

unsigned long long* newton_counter(int dev)
{
    unsigned int* p = status_word(dev);
    return p ? reinterpret_cast<unsigned long long*>(p + 2) : nullptr;
}

void fill_objdev(const ObjHost& o, ObjDev& d)
{
    std::memset(&d, 0, sizeof(d));
    d.W[0] = o.W[0][0];
    d.W[1] = o.W[0][1];
    d.W[2] = o.W[0][2];
    d.W[3] = o.W[1][1];
    d.W[4] = o.W[1][2];
    d.W[5] = o.W[2][2];
    for (int i = 0; i < 3; ++i) d.c[i] = o.c[i];
    d.m = o.m;
    d.lambda = o.lambda;
    d.k0 = 2.0 * kPi / o.lambda;
    d.jre[0] = o.jre[0];
    d.jre[1] = o.jre[1];
    d.jim[0] = o.jim[0];
    d.jim[1] = o.jim[1];
    d.zstart = o.c[2] - 2.0 * o.lmax - 1.0;
    d.S[0] = o.S[0][0];
    d.S[1] = o.S[0][1];
    d.S[2] = o.S[1][1];
    d.cap = o.lmax * o.lmax * std::cbrt(o.lmax / o.lambda);
    d.lmin = o.lmin;
    d.lmax = o.lmax;
    d.gc[0] = o.gc[0];
    d.gc[1] = o.gc[1];
    d.src_mode = o.src;
    for (int i = 0; i < 3; ++i) {
        d.src[i] = o.src_pos[i];
        d.e1[i] = o.e1[i];
        d.e2[i] = o.e2[i];
        d.inv_a[i] = 1.0 / o.a[i];
        for (int j = 0; j < 3; ++j) d.Rb[3 * i + j] = o.R[i][j];
    }
    d.shape_e = o.shape_e;
    d.bound2 = std::pow(3.0, 1.0 - 1.0 / o.shape_e);
    const double n2 = 2.0 * o.shape_e;
    d.shape_n = (n2 == std::floor(n2) && n2 >= 3.0 && n2 <= 32.0) ? (int)n2 : 0;
}

// ray grid of one object (host arithmetic only)
int grid_of(const ObjHost& o, const rtw_trace_params* tp, double* h, long long* nx, long long* ny, double* fan_w)
{
    if (tp->grid == RTW_GRID_FAN) {
        if (tp->n_rays < 2) return fail(RTW_ERR_ARG, "fan needs n_rays >= 2");
        const double e0 = std::cos(tp->fan_phi), e1 = std::sin(tp->fan_phi);
        const double q = e0 * (o.S[0][0] * e0 + o.S[0][1] * e1) + e1 * (o.S[1][0] * e0 + o.S[1][1] * e1);
        const double w = 1.0 / std::sqrt(q);
        *fan_w = w;
        *h = 2.0 * w / (double)tp->n_rays;
        *nx = tp->n_rays;
        *ny = 1;
        return RTW_OK;
    }
    if (tp->grid != RTW_GRID_SQUARE) return fail(RTW_ERR_ARG, "unknown grid kind %d", tp->grid);
    double hh = tp->spacing;
    if (!(hh > 0.0)) {
        if (tp->n_rays < 1) return fail(RTW_ERR_ARG, "square grid needs n_rays >= 1 or spacing > 0");
        const double detS = o.S[0][0] * o.S[1][1] - o.S[0][1] * o.S[1][0];
        hh = std::sqrt(kPi / (std::sqrt(detS) * (double)tp->n_rays));
    }
    const double X = std::sqrt(o.Sinv[0][0]), Y = std::sqrt(o.Sinv[1][1]);
    const long long kx = (long long)std::ceil(X / hh), ky = (long long)std::ceil(Y / hh);
    *h = hh;
    *nx = 2 * kx + 2;
    *ny = 2 * ky + 2;
    *fan_w = 0.0;
    return RTW_OK;
}

// Validates one object description and its incident wave and fills the host description (no
// device work, no allocation beyond the error message); i numbers the object in messages.
int make_object_host(const rtw_object_desc& d, const rtw_incident& w, int i, ObjHost& o)
{
    if (!(d.a > 0.0 && d.b > 0.0 && d.c > 0.0) || !std::isfinite(d.a + d.b + d.c))
        return fail(RTW_ERR_ARG, "object %d: semi-axes must be positive", i);
    const double qn = std::sqrt(d.quat[0] * d.quat[0] + d.quat[1] * d.quat[1] + d.quat[2] * d.quat[2] +
                                d.quat[3] * d.quat[3]);
    if (!(std::fabs(qn - 1.0) <= 1e-9)) return fail(RTW_ERR_ARG, "object %d: |quat| = %.17g != 1", i, qn);
    if (!(d.m_re > 0.0) || d.m_re == 1.0 || !std::isfinite(d.m_re))
        return fail(RTW_ERR_ARG, "object %d: m must be positive and != 1", i);
    if (d.m_im != 0.0) return fail(RTW_ERR_UNSUPPORTED, "object %d: absorbing objects (m_im != 0)", i);
    if (!(w.wavelength_um > 0.0) || !std::isfinite(w.wavelength_um))
        return fail(RTW_ERR_ARG, "object %d: wavelength must be positive", i);
    if (w.kind != RTW_INCIDENT_PLANE && w.kind != RTW_INCIDENT_POINT)
        return fail(RTW_ERR_ARG, "object %d: incident kind %d", i, w.kind);
    if (w.kind == RTW_INCIDENT_PLANE && (w.dir[0] != 0.0 || w.dir[1] != 0.0 || w.dir[2] != 1.0))
        return fail(RTW_ERR_UNSUPPORTED, "object %d: incident direction must be (0, 0, 1)", i);
    if (w.kind == RTW_INCIDENT_POINT && !std::isfinite(w.source[0] + w.source[1] + w.source[2]))
        return fail(RTW_ERR_ARG, "object %d: source position must be finite", i);
    const double se = d.shape_e == 0.0 ? 1.0 : d.shape_e;
    if (!(se >= 1.0) || !std::isfinite(se))
        return fail(RTW_ERR_ARG, "object %d: shape exponent %g (0 or 1: ellipsoid, > 1: superellipsoid)", i,
                    d.shape_e);
    o.shape_e = se;
    o.a[0] = d.a;
    o.a[1] = d.b;
    o.a[2] = d.c;
    const double qw = d.quat[0] / qn, qx = d.quat[1] / qn, qy = d.quat[2] / qn, qz = d.quat[3] / qn;
    o.R[0][0] = 1 - 2 * (qy * qy + qz * qz);
    o.R[0][1] = 2 * (qx * qy - qw * qz);
    o.R[0][2] = 2 * (qx * qz + qw * qy);
    o.R[1][0] = 2 * (qx * qy + qw * qz);
    o.R[1][1] = 1 - 2 * (qx * qx + qz * qz);
    o.R[1][2] = 2 * (qy * qz - qw * qx);
    o.R[2][0] = 2 * (qx * qz - qw * qy);
    o.R[2][1] = 2 * (qy * qz + qw * qx);
    o.R[2][2] = 1 - 2 * (qx * qx + qy * qy);
    for (int k = 0; k < 3; ++k) o.c[k] = d.center[k];
    o.m = d.m_re;
    o.lambda = w.wavelength_um;
    o.jre[0] = w.jones_re[0];
    o.jre[1] = w.jones_re[1];
    o.jim[0] = w.jones_im[0];
    o.jim[1] = w.jones_im[1];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += o.R[r][k] * o.R[c][k] / (o.a[k] * o.a[k]);
            o.W[r][c] = s;
        }
    o.lmax = std::fmax(d.a, std::fmax(d.b, d.c));
    o.lmin = std::fmin(d.a, std::fmin(d.b, d.c));
    o.S[0][0] = o.W[0][0] - o.W[0][2] * o.W[0][2] / o.W[2][2];
    o.S[0][1] = o.W[0][1] - o.W[0][2] * o.W[1][2] / o.W[2][2];
    o.S[1][0] = o.S[0][1];
    o.S[1][1] = o.W[1][1] - o.W[1][2] * o.W[1][2] / o.W[2][2];
    // a superellipsoid lies inside the ellipsoid of semi-axes a_i 3^((1 - 1/e) / 2) (power-mean
    // inequality), Wb = W / g2; the rays that meet it bound the ray grid (Wb = W for e = 1)
    const double g2 = se != 1.0 ? std::pow(3.0, 1.0 - 1.0 / se) : 1.0;
    double Wb[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Wb[r][c] = o.W[r][c] / g2;
    if (se != 1.0)
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) o.S[r][c] /= g2;
    o.gc[0] = o.c[0];
    o.gc[1] = o.c[1];
    o.src = w.kind == RTW_INCIDENT_POINT;
    if (o.src) {
        // rays from the source s through X = c + x e1 + y e2 (v = X - s = g + x e1 + y e2, g = c - s)
        // hit where (v.W g)^2 - (v.W v)(g.W g - 1) > 0: v^T K v > 0 with K = W g g^T W - (g.W g - 1) W,
        // an ellipse (w - w0)^T S (w - w0) < 1 of the plane
        double g[3], Wg[3];
        for (int k = 0; k < 3; ++k) {
            o.src_pos[k] = w.source[k];
            g[k] = o.c[k] - w.source[k];
        }
        for (int r = 0; r < 3; ++r) Wg[r] = Wb[r][0] * g[0] + Wb[r][1] * g[1] + Wb[r][2] * g[2];
        const double gWg = g[0] * Wg[0] + g[1] * Wg[1] + g[2] * Wg[2];
        if (!(gWg > 1.0))
            return fail(RTW_ERR_ARG, "object %d: the source lies inside the object (its bounding ellipsoid)", i);
        const double gd = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const double ax[3] = {g[0] / gd, g[1] / gd, g[2] / gd};
        const double ref[3] = {std::fabs(ax[0]) > 0.9 ? 0.0 : 1.0, std::fabs(ax[0]) > 0.9 ? 1.0 : 0.0, 0.0};
        const double ra = ref[0] * ax[0] + ref[1] * ax[1] + ref[2] * ax[2];
        double n1 = 0.0;
        for (int k = 0; k < 3; ++k) {
            o.e1[k] = ref[k] - ra * ax[k];
            n1 += o.e1[k] * o.e1[k];
        }
        n1 = std::sqrt(n1);
        for (int k = 0; k < 3; ++k) o.e1[k] /= n1;
        o.e2[0] = ax[1] * o.e1[2] - ax[2] * o.e1[1];
        o.e2[1] = ax[2] * o.e1[0] - ax[0] * o.e1[2];
        o.e2[2] = ax[0] * o.e1[1] - ax[1] * o.e1[0];
        double K[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) K[r][c] = Wg[r] * Wg[c] - (gWg - 1.0) * Wb[r][c];
        auto Kv = [&](const double* v, double* out3) {
            for (int r = 0; r < 3; ++r) out3[r] = K[r][0] * v[0] + K[r][1] * v[1] + K[r][2] * v[2];
        };
        auto dot = [](const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
        double Kg[3], K1[3], K2[3];
        Kv(g, Kg);
        Kv(o.e1, K1);
        Kv(o.e2, K2);
        const double M00 = dot(o.e1, K1), M01 = dot(o.e1, K2), M11 = dot(o.e2, K2);
        const double b0 = dot(o.e1, Kg), b1 = dot(o.e2, Kg);
        const double dM = M00 * M11 - M01 * M01;
        if (!(dM > 0.0)) return fail(RTW_ERR_ARG, "object %d: degenerate view from the source", i);
        const double w0x = -(M11 * b0 - M01 * b1) / dM, w0y = -(M00 * b1 - M01 * b0) / dM;
        const double f0 = dot(g, Kg) + b0 * w0x + b1 * w0y;
        if (!(f0 > 0.0)) return fail(RTW_ERR_ARG, "object %d: degenerate view from the source", i);
        o.S[0][0] = -M00 / f0;
        o.S[0][1] = o.S[1][0] = -M01 / f0;
        o.S[1][1] = -M11 / f0;
        o.gc[0] = w0x;
        o.gc[1] = w0y;
    }
    const double det = o.S[0][0] * o.S[1][1] - o.S[0][1] * o.S[1][0];
    o.Sinv[0][0] = o.S[1][1] / det;
    o.Sinv[0][1] = -o.S[0][1] / det;
    o.Sinv[1][0] = -o.S[1][0] / det;
    o.Sinv[1][1] = o.S[0][0] / det;
    return RTW_OK;
}

// The device table entry of object o for the ray grid of tp: the object's tables and its grid
// (spacing, size, fan half-width and axis), its rays starting at ray_offset.
int object_device_entry(const ObjHost& o, const rtw_trace_params* tp, long long ray_offset, ObjDev& d)
{
    double h = 0.0, w = 0.0;
    long long nx = 0, ny = 0;
    int rc = grid_of(o, tp, &h, &nx, &ny, &w);
    if (rc != RTW_OK) return rc;
    fill_objdev(o, d);
    d.grid = tp->grid == RTW_GRID_FAN ? rtw::kGridFan : rtw::kGridSquare;
    d.h = h;
    d.fan_w = w;
    d.fan_ex = std::cos(tp->fan_phi);
    d.fan_ey = std::sin(tp->fan_phi);
    d.nx = nx;
    d.ny = ny;
    d.ray_offset = ray_offset;
    return RTW_OK;
}

long long dir_count(const rtw_dirs* dirs)
{
    return dirs->kind == RTW_DIRS_LIST ? (long long)dirs->n_list : (long long)dirs->n_theta * dirs->n_phi;
}

// a list is binned on about one bin per direction: nt x 2 nt bins, nt up to 1024
void dir_grid(const rtw_dirs* dirs, int* nt, int* nph)
{
    if (dirs->kind == RTW_DIRS_LIST) {
        const long long want = (long long)std::ceil(std::sqrt(0.5 * (double)dirs->n_list));
        const int b = (int)std::min<long long>(1024, std::max<long long>(1, want));
        *nt = b;
        *nph = 2 * b;
    } else {
        *nt = dirs->n_theta;
        *nph = dirs->n_phi;
    }
}

int check_grid_dirs(const rtw_dirs* dirs, bool window_allowed, const char* who)
{
    if (dirs->kind == RTW_DIRS_GRID) {
        if (dirs->n_theta < 1 || dirs->n_phi < 2) return fail(RTW_ERR_ARG, "%s: n_theta >= 1, n_phi >= 2", who);
    } else if (dirs->kind == RTW_DIRS_LIST) {
        if (!dirs->list || dirs->n_list < 1 || dirs->n_list >= (1ll << 31))
            return fail(RTW_ERR_ARG, "%s: a direction list needs a device pointer and 1 <= n_list < 2^31", who);
    } else {
        return fail(RTW_ERR_ARG, "%s: a (theta, phi) grid or list of directions is required", who);
    }
    const int64_t* win = dirs->cell_window;
    const bool windowed = !(win[0] == -1 && win[1] == -1 && win[2] == -1 && win[3] == -1);
    if (windowed && !window_allowed) return fail(RTW_ERR_ARG, "%s: cell windows are not taken", who);
    return RTW_OK;
}

GridPlan plan_grid(const ObjDev* objs, int nobj, int np, const rtw_dirs* dirs)
{
    GridPlan g;
    const int64_t* win = dirs->cell_window;
    g.windowed = !(win[0] == -1 && win[1] == -1 && win[2] == -1 && win[3] == -1);
    const long long ndir = dir_count(dirs);
    g.group = (int)std::max<long long>(1, std::min<long long>(nobj, (1ll << 28) / std::max(1ll, 4 * ndir * np)));
    for (int oi = 0; oi < nobj; ++oi) g.super_shapes = g.super_shapes || objs[oi].shape_e != 1.0;
    // sliced runs: superellipsoids (hundreds of branches per direction), or direction grids so fine
    // that four pairs per direction and order no longer fit the largest hit list
    g.sliced = g.super_shapes || 4 * ndir * np * (long long)g.group + (1 << 20) > (1ll << 29);
    for (int g0 = 0; g0 < nobj; g0 += g.group) {
        long long cells = 0;
        for (int oi = g0; oi < std::min(nobj, g0 + g.group); ++oi) {
            const ObjDev& o = objs[oi];
            long long ix0 = 0, ix1 = o.nx - 1, iy0 = 0, iy1 = o.ny - 1;
            if (g.windowed) {
                ix0 = win[0] < 0 ? 0 : win[0];
                ix1 = win[1] > o.nx - 1 ? o.nx - 1 : win[1];
                iy0 = win[2] < 0 ? 0 : win[2];
                iy1 = win[3] > o.ny - 1 ? o.ny - 1 : win[3];
            }
            cells += std::max(0ll, ix1 - ix0) * std::max(0ll, iy1 - iy0) * np;
        }
        g.max_group_cells = std::max(g.max_group_cells, cells);
    }
    return g;
}

size_t grid_ws(const GridPlan& g, int np, const rtw_dirs* dirs, char* base, GridWs* w)
{
    const long long ndir = dir_count(dirs);
    int nt = 0, nph = 0;
    dir_grid(dirs, &nt, &nph);
    const bool list = dirs->kind == RTW_DIRS_LIST;
    const size_t nl = list ? (size_t)ndir : 0, nb = list ? (size_t)nt * (size_t)nph + 1 : 0;
    // list of large triangles: room for every triangle of a group (coarse ray grids make most of them
    // large), up to 2^29 entries; a triangle beyond the list is classified by its own thread
    const unsigned int big_cap =
        (unsigned int)std::min<long long>(std::max<long long>(65536, 2 * g.max_group_cells), 1ll << 29);
    // hit list: 4 pairs per direction and order (ellipsoids: one to a few branches each); 32 with
    // superellipsoids, whose runs are sliced to fit
    const long long per_dir = g.super_shapes ? 32 : 4;
    const unsigned int hit_cap =
        (unsigned int)std::min<long long>(per_dir * ndir * np * g.group + (1 << 20), 1ll << 29);
    size_t off_mask = 0;
    size_t off_tab = align_up(off_mask + sizeof(unsigned int) * (size_t)ndir * (size_t)g.group, 256);
    // double tables then their single-precision copies
    size_t off_cells = align_up(off_tab + sizeof(double) * 4 * ((size_t)nt + (size_t)nph), 256);
    size_t off_ldir = align_up(off_cells + sizeof(GridCells) * (size_t)g.group, 256);
    size_t off_ldirf = align_up(off_ldir + sizeof(double) * 4 * nl, 256);
    size_t off_binid = align_up(off_ldirf + sizeof(float4) * nl, 256);
    size_t off_count = align_up(off_binid + sizeof(int) * nl, 256);
    size_t off_first = align_up(off_count + sizeof(int) * nb, 256);
    size_t off_cursor = align_up(off_first + sizeof(int) * nb, 256);
    size_t off_bindir = align_up(off_cursor + sizeof(int) * nb, 256);
    size_t off_big = align_up(off_bindir + sizeof(int) * nl, 256);
    size_t off_cnt = align_up(off_big + 8 * (size_t)big_cap, 256);
    size_t off_hit_tri = align_up(off_cnt + 256, 256);
    size_t off_hit_dir = align_up(off_hit_tri + 8 * (size_t)hit_cap, 256);
    size_t total = align_up(off_hit_dir + 4 * (size_t)hit_cap, 256);
    if (base && w) {
        w->mask_words = (unsigned int*)(base + off_mask);
        w->tab = (double*)(base + off_tab);
        w->cells = (GridCells*)(base + off_cells);
        w->ldir = list ? (double*)(base + off_ldir) : nullptr;
        w->ldir_f = list ? (float4*)(base + off_ldirf) : nullptr;
        w->binid = list ? (int*)(base + off_binid) : nullptr;
        w->count = list ? (int*)(base + off_count) : nullptr;
        w->first = list ? (int*)(base + off_first) : nullptr;
        w->cursor = list ? (int*)(base + off_cursor) : nullptr;
        w->bin_dir = list ? (int*)(base + off_bindir) : nullptr;
        w->big = (unsigned long long*)(base + off_big);
        w->nbig = (unsigned int*)(base + off_cnt);
        w->nhit = w->nbig + 1;
        w->hit_tri = (unsigned long long*)(base + off_hit_tri);
        w->hit_dir = (unsigned int*)(base + off_hit_dir);
        w->big_cap = big_cap;
        w->hit_cap = hit_cap;
    }
    return total;
}

int dirs_prepare(const rtw_dirs* dirs, const GridWs& w, DirSet* d, cudaStream_t s)
{
    std::memset(d, 0, sizeof(*d));
    dir_grid(dirs, &d->nt, &d->nph);
    d->tab = w.tab;
    d->ndir = dir_count(dirs);
    RTW_CUDA(launch_dir_tables(d->nt, d->nph, w.tab, s));
    if (dirs->kind == RTW_DIRS_LIST) {
        d->list = 1;
        d->bin_first = w.first;
        d->bin_dir = w.bin_dir;
        d->ldir = w.ldir;
        d->ldir_f = w.ldir_f;
        d->lsrc = dirs->list;
        // a bin spans pi / nt in theta and at most as much in arc along phi: its points lie within
        // sqrt(2) / 2 pi / nt of its centre
        d->pad = (float)(0.75 * kPi / d->nt + 1e-6);
        RTW_CUDA(launch_bin_dirs(dirs->list, d->ndir, d->nt, d->nph, w.ldir, w.ldir_f, w.binid, w.count, w.first,
                                 w.cursor, w.bin_dir, s));
    }
    return RTW_OK;
}

int grid_field_run(const ObjDev* h_objs, const ObjDev* d_objs, int nobj, const RaysDev& st, const GridPlan& g,
                   const rtw_dirs* dirs, const DirSet& d, bool per_order, double* out, unsigned char* mask_out,
                   const GridWs& w, int classify_block, int newton, unsigned int* status, unsigned long long* nfail,
                   cudaStream_t s, std::vector<std::pair<long long, long long>>* slices)
{
    const bool fixed = !newton && st.fmax && st.frec && st.fval;
    const int np = st.np;
    const long long ndir = d.ndir;
    const int nout = per_order ? np : 1;
    const size_t ncomp = st.near_r > 0.0 ? 6 : 4;  // (E_r,) theta, phi components, re and im
    const size_t out_obj = ncomp * (size_t)nout * (size_t)ndir;  // doubles per object
    const int64_t* win = dirs->cell_window;
    for (int g0 = 0; g0 < nobj; g0 += g.group) {
        const int gn = std::min(g.group, nobj - g0);
        RTW_CUDA(cudaMemsetAsync(w.mask_words, 0, sizeof(unsigned int) * (size_t)ndir * (size_t)gn, s));
        FieldArgs a;
        a.d_obj = d_objs + g0;
        a.st = st;
        a.pmax = np - 1;
        a.per_order = per_order ? 1 : 0;
        a.out = out + out_obj * (size_t)g0;
        a.mask = w.mask_words;
        a.status = status;
        a.nfail = nfail;
        // cells [ix0, ix1) x [iy0, iy1) of every object of the group, window wv (when windowed)
        auto batch = [&](bool windowed, const int64_t* wv, GridBatch& b) -> int {
            RTW_CUDA(launch_grid_cells(d_objs + g0, gn, np, windowed, wv, w.cells, s));
            b.cells = w.cells;
            b.nobj = gn;
            b.total = 0;
            for (int oi = g0; oi < g0 + gn; ++oi) {
                const ObjDev& o = h_objs[oi];
                long long ix0 = 0, ix1 = o.nx - 1, iy0 = 0, iy1 = o.ny - 1;
                if (windowed) {
                    ix0 = wv[0] < 0 ? 0 : wv[0];
                    ix1 = wv[1] > o.nx - 1 ? o.nx - 1 : wv[1];
                    iy0 = wv[2] < 0 ? 0 : wv[2];
                    iy1 = wv[3] > o.ny - 1 ? o.ny - 1 : wv[3];
                }
                b.total += std::max(0ll, ix1 - ix0) * std::max(0ll, iy1 - iy0) * np;
            }
            b.ndir = ndir;
            b.nout = nout;
            return RTW_OK;
        };
        const unsigned int* fmax = fixed ? st.fmax + g0 : nullptr;
        if (!g.sliced) {
            GridBatch b;
            int rc = batch(g.windowed, win, b);
            if (rc != RTW_OK) return rc;
            RTW_CUDA(launch_field_grid(a, b, d, w.big, w.nbig, w.big_cap, w.hit_tri, w.hit_dir, w.nhit, w.hit_cap,
                                       classify_block, newton, s, kFieldAll, fmax));
        } else {
            long long rows = 0, cols = 0;
            for (int oi = g0; oi < g0 + gn; ++oi) {
                rows = std::max(rows, h_objs[oi].ny - 1);
                cols = std::max(cols, h_objs[oi].nx - 1);
            }
            const long long x0 = g.windowed ? win[0] : 0, x1 = g.windowed ? win[1] : cols;
            const long long y0 = g.windowed ? std::max<long long>(0, win[2]) : 0;
            const long long y1 = g.windowed ? std::min<long long>(rows, win[3]) : rows;
            std::vector<std::pair<long long, long long>> todo, fitted;
            if (y1 > y0) {
                if (slices && !slices->empty() && slices->front().first == y0 && slices->back().second == y1) {
                    // the slices that fitted last time, taken from the stack in increasing row order
                    todo.assign(slices->rbegin(), slices->rend());
                } else {
                    todo.emplace_back(y0, y1);
                }
            }
            while (!todo.empty()) {
                const auto sl = todo.back();
                todo.pop_back();
                const int64_t wv[4] = {x0, x1, sl.first, sl.second};
                GridBatch b;
                int rc = batch(true, wv, b);
                if (rc != RTW_OK) return rc;
                RTW_CUDA(launch_field_grid(a, b, d, w.big, w.nbig, w.big_cap, w.hit_tri, w.hit_dir, w.nhit, w.hit_cap,
                                           classify_block, newton, s, kFieldClassify));
                unsigned int want = 0;
                RTW_CUDA(cudaMemcpyAsync(&want, w.nhit, sizeof(want), cudaMemcpyDeviceToHost, s));
                RTW_CUDA(cudaStreamSynchronize(s));
                if (b.total > 0 && want > w.hit_cap) {
                    const long long h = sl.second - sl.first;
                    if (h <= 1)
                        return fail(RTW_ERR_CAPACITY, "rtw_field: one row of the ray grid wants %u (triangle, "
                                    "direction) pairs, more than the %u of the hit list", want, w.hit_cap);
                    // the count is exact: split into enough equal slices for three quarters of the list
                    // each (uneven rows split again), taken in increasing row order
                    const long long k = std::min(h, std::max(2ll, (long long)(want / (0.75 * w.hit_cap)) + 1));
                    for (long long q = k - 1; q >= 0; --q)
                        todo.emplace_back(sl.first + h * q / k, sl.first + h * (q + 1) / k);
                    continue;
                }
                RTW_CUDA(launch_field_grid(a, b, d, w.big, w.nbig, w.big_cap, w.hit_tri, w.hit_dir, w.nhit, w.hit_cap,
                                           classify_block, newton, s, kFieldSum, fmax));
                fitted.push_back(sl);
            }
            if (slices) {
                std::sort(fitted.begin(), fitted.end());
                *slices = fitted;
            }
        }
        if (fixed) RTW_CUDA(launch_field_convert(a.out, (long long)out_obj, gn, fmax, s));
        if (mask_out)
            RTW_CUDA(launch_finalize_mask(w.mask_words, mask_out + (size_t)g0 * (size_t)ndir, d_objs + g0, gn, ndir,
                                          d.list ? 2 : 1, d.nt, d.nph, 0.0, 0.0, s, d.lsrc));
    }
    return RTW_OK;
}

}  // namespace host
}  // namespace rtw

struct rtw_rays {
    int device = 0;
    int np = 0;
    int precision = 0;
    int grid = 0;
    int flags = 0;
    int nobj = 0;
    long long R = 0;
    double fan_phi = 0.0;
    std::vector<ObjDev> objs;
    ObjDev* d_objs = nullptr;
    size_t d_objs_cap = 0;
    RaysDev st{};
    // sliced field runs: the row slices that fitted the hit list, for the directions of slice_key
    std::vector<std::pair<long long, long long>> slices;
    long long slice_key = -1;
    void* block = nullptr;
    size_t block_bytes = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
};

namespace {

using rtw::host::fill_objdev;
using rtw::host::grid_of;

int ensure_device(int* dev)
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return fail(RTW_ERR_CUDA, "no usable CUDA device (%s)", cudaGetErrorString(e));
    RTW_CUDA(cudaGetDevice(dev));
    return RTW_OK;
}

// The plan, workspace (grown in the rays' block when too small) and prepared directions of a
// square-grid field of rays on dirs; the row slices kept from an earlier run are dropped when the
// directions or the window changed.
int grid_prepare(rtw_rays* rays, const rtw_dirs* dirs, rtw::host::GridPlan* g, rtw::host::GridWs* w,
                 rtw::DirSet* d, cudaStream_t s)
{
    *g = rtw::host::plan_grid(rays->objs.data(), rays->nobj, rays->np, dirs);
    const size_t total = rtw::host::grid_ws(*g, rays->np, dirs, nullptr, nullptr);
    if (rays->ws_bytes < total) {
        if (rays->ws) cudaFree(rays->ws);
        rays->ws = nullptr;
        rays->ws_bytes = 0;
        cudaError_t e = cudaMalloc(&rays->ws, total);
        if (e != cudaSuccess) return fail(RTW_ERR_NOMEM, "rtw_field: workspace of %zu bytes", total);
        rays->ws_bytes = total;
    }
    rtw::host::grid_ws(*g, rays->np, dirs, (char*)rays->ws, w);
    int rc = rtw::host::dirs_prepare(dirs, *w, d, s);
    if (rc != RTW_OK) return rc;
    const long long ndir = rtw::host::dir_count(dirs);
    const int64_t* cw = dirs->cell_window;
    const long long key = (ndir * 64 + rays->np) ^ (cw[0] * 7919 + cw[1] * 104729 + cw[2] * 1299709 + cw[3] * 15485863);
    if (rays->slice_key != key) {
        rays->slice_key = key;
        rays->slices.clear();
    }
    return RTW_OK;
}

}  // namespace

extern "C" {

const char* rtw_version(void) { return "rtw-gb300 0.1 (sm_103a)"; }

const char* rtw_last_error(void) { return g_last_error.c_str(); }

const char* rtw_status_string(int status)
{
    switch (status) {
    case RTW_OK: return "ok";
    case RTW_ERR_ARG: return "invalid argument";
    case RTW_ERR_UNSUPPORTED: return "unsupported";
    case RTW_ERR_CUDA: return "CUDA error";
    case RTW_ERR_CAPACITY: return "capacity exceeded";
    case RTW_ERR_TIMEOUT: return "bounded iteration gave up";
    case RTW_ERR_NUMERIC: return "non-finite value";
    case RTW_ERR_NOMEM: return "out of memory";
    default: return "unknown status";
    }
}

int rtw_create_object(const rtw_object_desc* desc, int count, const rtw_incident* inc, rtw_object** out)
{
    if (!desc || !inc || !out || count < 1) return fail(RTW_ERR_ARG, "rtw_create_object: null pointer or count < 1");
    *out = nullptr;
    std::vector<ObjHost> hs((size_t)count);
    for (int i = 0; i < count; ++i) {
        const int rc = rtw::host::make_object_host(desc[i], inc[i], i, hs[(size_t)i]);
        if (rc != RTW_OK) return rc;
    }
    int dev = 0;
    int rc = ensure_device(&dev);
    if (rc != RTW_OK) return rc;
    rtw_object* obj = new (std::nothrow) rtw_object();
    if (!obj) return fail(RTW_ERR_NOMEM, "rtw_create_object: host allocation");
    obj->count = count;
    obj->device = dev;
    obj->h = std::move(hs);
    *out = obj;
    return RTW_OK;
}

void rtw_destroy_object(rtw_object* obj) { delete obj; }

int rtw_object_grid(const rtw_object* obj, int index, const rtw_trace_params* tp, double* h, int64_t* nx,
                    int64_t* ny)
{
    if (!obj || !tp || !h || !nx || !ny) return fail(RTW_ERR_ARG, "rtw_object_grid: null pointer");
    if (index < 0 || index >= obj->count) return fail(RTW_ERR_ARG, "rtw_object_grid: index out of range");
    long long a = 0, b = 0;
    double w = 0.0;
    int rc = grid_of(obj->h[(size_t)index], tp, h, &a, &b, &w);
    *nx = a;
    *ny = b;
    return rc;
}

int rtw_trace(rtw_object* obj, const rtw_trace_params* tp, void* stream, rtw_rays** inout)
{
    if (!obj || !tp || !inout) return fail(RTW_ERR_ARG, "rtw_trace: null pointer");
    if (tp->p_max < 0 || tp->p_max >= rtw::kMaxOrders) return fail(RTW_ERR_ARG, "rtw_trace: p_max out of [0, 15]");
    if (tp->precision != RTW_FP64 && tp->precision != RTW_MIXED && tp->precision != RTW_DFLOAT)
        return fail(RTW_ERR_ARG, "rtw_trace: precision %d", tp->precision);
    bool super_shapes = false;
    for (int i = 0; i < obj->count; ++i) {
        if (obj->h[(size_t)i].src && (tp->grid != RTW_GRID_SQUARE || tp->precision != RTW_FP64))
            return fail(RTW_ERR_UNSUPPORTED, "rtw_trace: a point source takes a square grid in double precision");
        if (obj->h[(size_t)i].shape_e != 1.0) {
            if (tp->grid != RTW_GRID_SQUARE || tp->precision != RTW_FP64)
                return fail(RTW_ERR_UNSUPPORTED, "rtw_trace: a superellipsoid takes a square grid in double precision");
            super_shapes = true;
        }
    }
    if (!(tp->observe_radius >= 0.0) || !std::isfinite(tp->observe_radius))
        return fail(RTW_ERR_ARG, "rtw_trace: observe_radius must be finite and >= 0");
    if (tp->observe_radius > 0.0) {
        if (tp->grid != RTW_GRID_SQUARE) return fail(RTW_ERR_ARG, "rtw_trace: observe_radius needs a square grid");
        if (tp->precision != RTW_FP64)
            return fail(RTW_ERR_UNSUPPORTED, "rtw_trace: observe_radius is traced in double precision only");
        if (tp->flags & RTW_TRACE_APERTURE)
            return fail(RTW_ERR_ARG, "rtw_trace: observe_radius excludes RTW_TRACE_APERTURE");
        for (int i = 0; i < obj->count; ++i) {
            const rtw::host::ObjHost& h = obj->h[(size_t)i];
            const double rc = std::sqrt(h.c[0] * h.c[0] + h.c[1] * h.c[1] + h.c[2] * h.c[2]);
            // radius about the centre that holds the body: the largest semi-axis, times 3^((1 - 1/e) / 2)
            // for a superellipsoid (its bounding ellipsoid)
            const double rb = h.lmax * std::sqrt(std::pow(3.0, 1.0 - 1.0 / h.shape_e));
            if (!(tp->observe_radius > rc + rb))
                return fail(RTW_ERR_ARG, "rtw_trace: observe_radius %g does not enclose object %d (|c| + %g)",
                            tp->observe_radius, i, rb);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int np = tp->p_max + 1;
    std::vector<ObjDev> objs((size_t)obj->count);
    long long R = 0;
    for (int i = 0; i < obj->count; ++i) {
        ObjDev& d = objs[(size_t)i];
        int rc = rtw::host::object_device_entry(obj->h[(size_t)i], tp, R, d);
        if (rc != RTW_OK) return rc;
        R += d.nx * d.ny;
    }
    // aperture data: fans (the 1-D PO of rtw_field) and square grids in double precision (rtw_field_po2d)
    if ((tp->flags & RTW_TRACE_APERTURE) && tp->grid == RTW_GRID_SQUARE && tp->precision != RTW_FP64)
        return fail(RTW_ERR_UNSUPPORTED, "rtw_trace: RTW_TRACE_APERTURE on a square grid needs RTW_FP64");
    const bool aux = (tp->flags & RTW_TRACE_APERTURE) != 0;
    // one allocation carved into 256-byte aligned arrays
    const size_t n = (size_t)np * (size_t)R;
    size_t off[9], total = 0;
    const bool sf = tp->grid == RTW_GRID_SQUARE;  // single-precision field records for the grid field
    const size_t sizes[9] = {n * 16, n * 16, n * 16, n * 16, n * 16, n * 4, aux ? n * 8 * rtw::kAuxCount : 0,
                             sf ? n * 64 : 0, sf ? 4 * (size_t)obj->count : 0};
    for (int k = 0; k < 9; ++k) {
        off[k] = total;
        total = align_up(total + sizes[k], 256);
    }
    rtw_rays* r = *inout;
    bool fresh = false;
    if (!r) {
        r = new (std::nothrow) rtw_rays();
        if (!r) return fail(RTW_ERR_NOMEM, "rtw_trace: host allocation");
        fresh = true;
    }
    RTW_CUDA(cudaGetDevice(&r->device));
    if (r->block_bytes < total) {
        if (r->block) cudaFree(r->block);
        r->block = nullptr;
        r->block_bytes = 0;
        cudaError_t e = cudaMalloc(&r->block, total);
        if (e != cudaSuccess) {
            if (fresh) delete r;
            else *inout = r;
            return fail(RTW_ERR_NOMEM, "rtw_trace: cudaMalloc of %zu bytes: %s", total, cudaGetErrorString(e));
        }
        r->block_bytes = total;
    }
    if (r->d_objs_cap < objs.size()) {
        if (r->d_objs) cudaFree(r->d_objs);
        r->d_objs = nullptr;
        r->d_objs_cap = 0;
        if (cudaMalloc(&r->d_objs, sizeof(ObjDev) * objs.size()) != cudaSuccess) {
            if (fresh) delete r;
            return fail(RTW_ERR_NOMEM, "rtw_trace: object table");
        }
        r->d_objs_cap = objs.size();
    }
    *inout = r;
    if (r->R != R || r->np != np || r->grid != tp->grid) r->slices.clear();  // another ray grid
    r->np = np;
    r->precision = tp->precision;
    r->grid = tp->grid;
    r->flags = tp->flags;
    r->nobj = obj->count;
    r->R = R;
    r->fan_phi = tp->fan_phi;
    r->objs = objs;
    char* b = (char*)r->block;
    r->st.R = R;
    r->st.np = np;
    r->st.precision = tp->precision;
    r->st.near_r = tp->observe_radius;
    r->st.s01 = (double2*)(b + off[0]);
    r->st.s2psi = (double2*)(b + off[1]);
    r->st.Fx = (double2*)(b + off[2]);
    r->st.Fy = (double2*)(b + off[3]);
    r->st.Fz = (double2*)(b + off[4]);
    r->st.flags = (uint32_t*)(b + off[5]);
    r->st.aux = aux ? (double*)(b + off[6]) : nullptr;
    r->st.frec = sf ? (float4*)(b + off[7]) : nullptr;
    r->st.fval = sf ? (float4*)(b + off[7] + n * 32) : nullptr;
    r->st.fmax = sf ? (unsigned int*)(b + off[8]) : nullptr;
    RTW_CUDA(cudaMemcpyAsync(r->d_objs, r->objs.data(), sizeof(ObjDev) * objs.size(), cudaMemcpyHostToDevice, s));
    if (sf) RTW_CUDA(cudaMemsetAsync(r->st.fmax, 0, 4 * (size_t)obj->count, s));
    unsigned int* status = status_word(r->device);
    RTW_CUDA(rtw::launch_trace(r->d_objs, r->nobj, r->st, tp->p_max, aux, status, s, super_shapes));
    return RTW_OK;
}

int rtw_rays_info(const rtw_rays* rays, int64_t* rays_per_order, int* n_orders, int* n_objects)
{
    if (!rays) return fail(RTW_ERR_ARG, "rtw_rays_info: null handle");
    if (rays_per_order) *rays_per_order = rays->R;
    if (n_orders) *n_orders = rays->np;
    if (n_objects) *n_objects = rays->nobj;
    return RTW_OK;
}

int rtw_rays_export(const rtw_rays* rays, int order, int64_t first, int64_t count, double* s_out, double* F_out,
                    double* psi_out, uint32_t* flags_out, void* stream)
{
    if (!rays) return fail(RTW_ERR_ARG, "rtw_rays_export: null handle");
    if (order < 0 || order >= rays->np) return fail(RTW_ERR_ARG, "rtw_rays_export: order out of range");
    if (first < 0 || count < 0 || first + count > rays->R) return fail(RTW_ERR_ARG, "rtw_rays_export: range");
    RTW_CUDA(rtw::launch_export(rays->st, order, first, count, s_out, F_out, psi_out, flags_out,
                                (cudaStream_t)stream));
    return RTW_OK;
}

void rtw_destroy_rays(rtw_rays* rays)
{
    if (!rays) return;
    if (rays->block) cudaFree(rays->block);
    if (rays->d_objs) cudaFree(rays->d_objs);
    if (rays->ws) cudaFree(rays->ws);
    delete rays;
}

int rtw_trace_points(const rtw_object* obj, int index, const double* xy, int64_t n, int p_max, double* s_out,
                     double* F_out, double* psi_out, uint32_t* flags_out, void* stream)
{
    if (!obj || (!xy && n > 0)) return fail(RTW_ERR_ARG, "rtw_trace_points: null pointer");
    if (index < 0 || index >= obj->count) return fail(RTW_ERR_ARG, "rtw_trace_points: index out of range");
    if (p_max < 0 || p_max >= rtw::kMaxOrders) return fail(RTW_ERR_ARG, "rtw_trace_points: p_max out of range");
    if (n < 0) return fail(RTW_ERR_ARG, "rtw_trace_points: n < 0");
    if (obj->h[(size_t)index].shape_e != 1.0) return fail(RTW_ERR_UNSUPPORTED, "rtw_trace_points: ellipsoids only");
    cudaStream_t s = (cudaStream_t)stream;
    ObjDev d;
    fill_objdev(obj->h[(size_t)index], d);
    // a per-call object entry: a tiny device buffer freed after the launch has been ordered
    ObjDev* d_obj = nullptr;
    RTW_CUDA(cudaMallocAsync(&d_obj, sizeof(ObjDev), s));
    RTW_CUDA(cudaMemcpyAsync(d_obj, &d, sizeof(ObjDev), cudaMemcpyHostToDevice, s));
    cudaError_t e = rtw::launch_trace_points(d_obj, xy, n, p_max, s_out, F_out, psi_out, flags_out, s);
    cudaFreeAsync(d_obj, s);
    if (e != cudaSuccess) return cuda_fail(e, "trace_points launch");
    return RTW_OK;
}

int rtw_field_po2d(const rtw_rays* rays, const rtw_po2d_params* pp, const double* dirs, int64_t n_dirs,
                   void* field_out, int64_t* n_used, void* stream)
{
    if (!rays || !pp || !dirs || !field_out) return fail(RTW_ERR_ARG, "rtw_field_po2d: null pointer");
    if (rays->grid != RTW_GRID_SQUARE || rays->nobj != 1 || !rays->st.aux || rays->st.near_r != 0.0)
        return fail(RTW_ERR_ARG, "rtw_field_po2d: one object on a square grid traced with RTW_TRACE_APERTURE "
                                 "(far field) is required");
    if (pp->order < 0 || pp->order >= rays->np) return fail(RTW_ERR_ARG, "rtw_field_po2d: order out of range");
    const ObjDev& o = rays->objs[0];
    const int64_t* w = pp->window;
    if (w[0] < 0 || w[2] < 0 || w[1] >= o.nx || w[3] >= o.ny || w[1] - w[0] < 2 || w[3] - w[2] < 2)
        return fail(RTW_ERR_ARG, "rtw_field_po2d: window must hold at least 3 x 3 vertices of the %lld x %lld grid",
                    o.nx, o.ny);
    if ((w[1] - w[0] + 1) * (w[3] - w[2] + 1) >= (1ll << 31))
        return fail(RTW_ERR_ARG, "rtw_field_po2d: more than 2^31 rays in the window");
    if (!(pp->cone_full >= 0.0 && pp->cone_end > pp->cone_full && pp->cone_end <= 0.5 * kPi))
        return fail(RTW_ERR_ARG, "rtw_field_po2d: 0 <= cone_full < cone_end <= pi/2");
    if (!std::isfinite(pp->axis_theta + pp->axis_phi)) return fail(RTW_ERR_ARG, "rtw_field_po2d: axis");
    if (n_dirs < 1 || n_dirs >= (1ll << 31)) return fail(RTW_ERR_ARG, "rtw_field_po2d: 1 <= n_dirs < 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    const long long win[4] = {w[0], w[1], w[2], w[3]};
    const long long nwin = (win[1] - win[0] + 1) * (win[3] - win[2] + 1);
    const double axis[3] = {std::sin(pp->axis_theta) * std::cos(pp->axis_phi),
                            std::sin(pp->axis_theta) * std::sin(pp->axis_phi), std::cos(pp->axis_theta)};
    // a per-call scratch block, freed once the launches have been ordered
    void* scratch = nullptr;
    RTW_CUDA(cudaMallocAsync(&scratch, rtw::po2d_scratch_bytes(nwin, n_dirs), s));
    const size_t bytes = rtw::po2d_scratch_bytes(nwin, n_dirs);
    cudaError_t e = rtw::launch_po2d(rays->st, pp->order, o.nx, win, o.c, axis, o.k0, pp->cone_full, pp->cone_end,
                                     dirs, n_dirs, (double2*)field_out, scratch, s);
    unsigned int used = 0;
    if (e == cudaSuccess && n_used) {
        // the count sits in the last 256 bytes of the scratch block
        e = cudaMemcpyAsync(&used, (char*)scratch + bytes - 256, sizeof(used), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "po2d launch");
    if (n_used) *n_used = (int64_t)used;
    return RTW_OK;
}

int rtw_field(const rtw_rays* rays_c, const rtw_dirs* dirs, int mode, int flags, void* field_out, uint8_t* mask_out,
              void* stream)
{
    rtw_rays* rays = const_cast<rtw_rays*>(rays_c);
    if (!rays || !dirs || !field_out) return fail(RTW_ERR_ARG, "rtw_field: null pointer");
    if (mode != RTW_DENSE && mode != RTW_NEWTON) return fail(RTW_ERR_ARG, "rtw_field: mode %d", mode);
    if (mode == RTW_NEWTON && (flags & RTW_FIELD_NEAR_FOLDS) && rays->grid != RTW_GRID_FAN)
        return fail(RTW_ERR_ARG, "rtw_field: RTW_FIELD_NEAR_FOLDS needs a fan grid");
    cudaStream_t s = (cudaStream_t)stream;
    const bool per_order = (flags & RTW_FIELD_PER_ORDER) != 0;
    const bool po = (flags & RTW_FIELD_PO) != 0;
    const int newton = mode == RTW_NEWTON ? ((flags & RTW_FIELD_NEAR_FOLDS) ? 2 : 1) : 0;
    if (po && newton) return fail(RTW_ERR_ARG, "rtw_field: RTW_FIELD_PO and RTW_NEWTON exclude each other");
    if (rays->st.near_r > 0.0 && (newton || po))
        return fail(RTW_ERR_ARG, "rtw_field: rays traced to a finite radius take the dense mode without PO");
    if (newton || po)
        for (int i = 0; i < rays->nobj; ++i)
            if (rays->objs[(size_t)i].shape_e != 1.0)
                return fail(RTW_ERR_UNSUPPORTED, "rtw_field: a superellipsoid takes the dense mode without PO");
    const bool folds = po || newton == 2;
    const int nout = per_order ? rays->np : 1;
    long long ndir = 0;
    if (dirs->kind == RTW_DIRS_PLANE) {
        if (rays->grid != RTW_GRID_FAN) return fail(RTW_ERR_ARG, "rtw_field: plane directions need a fan grid");
        if (dirs->n_theta < 1 || !(std::fabs(dirs->dalpha) > 0.0) || std::fabs(dirs->dalpha) > 0.5 ||
            std::fabs(dirs->dalpha) * dirs->n_theta > 2.0 * kPi + 1e-9)
            return fail(RTW_ERR_ARG, "rtw_field: plane grid needs n >= 1, 0 < |dalpha| <= 0.5, span <= 2 pi");
        ndir = dirs->n_theta;
    } else if (dirs->kind == RTW_DIRS_GRID || dirs->kind == RTW_DIRS_LIST) {
        if (rays->grid != RTW_GRID_SQUARE)
            return fail(RTW_ERR_ARG, "rtw_field: (theta, phi) grids and lists need a square grid");
        int rc = rtw::host::check_grid_dirs(dirs, true, "rtw_field");
        if (rc != RTW_OK) return rc;
        ndir = rtw::host::dir_count(dirs);
    } else {
        return fail(RTW_ERR_ARG, "rtw_field: unknown direction kind %d", dirs->kind);
    }
    if (po && (rays->grid != RTW_GRID_FAN || !rays->st.aux))
        return fail(RTW_ERR_ARG, "rtw_field: RTW_FIELD_PO needs a fan traced with RTW_TRACE_APERTURE");
    unsigned int* status = status_word(rays->device);
    if (dirs->kind != RTW_DIRS_PLANE) {
        rtw::host::GridPlan g;
        rtw::host::GridWs w;
        rtw::DirSet d;
        int rc = grid_prepare(rays, dirs, &g, &w, &d, s);
        if (rc != RTW_OK) return rc;
        const size_t ncomp = rays->st.near_r > 0.0 ? 6 : 4;
        RTW_CUDA(cudaMemsetAsync(field_out, 0,
                                 sizeof(double) * ncomp * (size_t)nout * (size_t)ndir * (size_t)rays->nobj, s));
        // the slices found for these directions and this window are kept for the next call
        return rtw::host::grid_field_run(rays->objs.data(), rays->d_objs, rays->nobj, rays->st, g, dirs, d,
                                         per_order, (double*)field_out, mask_out, w, 0, newton, status,
                                         newton_counter(rays->device), s, &rays->slices);
    }
    // fan: workspace of mask words, PO windows and scratch
    const long long nfan = rays->objs[0].nx;
    const long long ap_cap = po ? 2 * (long long)rays->np * nfan : 0;
    size_t off_mask = 0;
    size_t off_win = align_up(off_mask + sizeof(unsigned int) * (size_t)ndir, 256);
    size_t off_nwin = align_up(off_win + sizeof(rtw::PoWindow) * rtw::kMaxPoWindows, 256);
    size_t off_po = align_up(off_nwin + 256, 256);
    size_t po_bytes = folds ? sizeof(double) * ((size_t)rays->np * (size_t)nfan + rtw::kMaxPoWindows + 1 +
                                                9 * (size_t)ap_cap)
                            : 0;
    size_t total = align_up(off_po + po_bytes, 256);
    if (rays->ws_bytes < total) {
        if (rays->ws) cudaFree(rays->ws);
        rays->ws = nullptr;
        rays->ws_bytes = 0;
        cudaError_t e = cudaMalloc(&rays->ws, total);
        if (e != cudaSuccess) return fail(RTW_ERR_NOMEM, "rtw_field: workspace of %zu bytes", total);
        rays->ws_bytes = total;
    }
    char* ws = (char*)rays->ws;
    unsigned int* mask_words = (unsigned int*)(ws + off_mask);
    rtw::PoWindow* d_win = (rtw::PoWindow*)(ws + off_win);
    int* d_nwin = (int*)(ws + off_nwin);
    double2* d_po = (double2*)(ws + off_po);
    const size_t out_bytes_obj = sizeof(double) * 4 * (size_t)nout * (size_t)ndir;
    RTW_CUDA(cudaMemsetAsync(field_out, 0, out_bytes_obj * (size_t)rays->nobj, s));
    for (int oi = 0; oi < rays->nobj; ++oi) {
        RTW_CUDA(cudaMemsetAsync(mask_words, 0, sizeof(unsigned int) * (size_t)ndir, s));
        rtw::FieldArgs a;
        a.d_obj = rays->d_objs + oi;
        a.st = rays->st;
        a.pmax = rays->np - 1;
        a.per_order = per_order ? 1 : 0;
        a.out = (double*)((char*)field_out + out_bytes_obj * (size_t)oi);
        a.mask = mask_words;
        a.status = status;
        a.nfail = newton_counter(rays->device);
        const ObjDev& o = rays->objs[(size_t)oi];
        RTW_CUDA(rtw::launch_field_fan(a, o.nx, rays->fan_phi, dirs->n_theta, dirs->alpha0, dirs->dalpha, d_win,
                                       d_nwin, d_po, ap_cap, po ? 1 : 0, newton, s));
        if (mask_out)
            RTW_CUDA(rtw::launch_finalize_mask(mask_words, mask_out + (size_t)oi * (size_t)ndir, rays->d_objs + oi, 1,
                                               ndir, 0, dirs->n_theta, 0, dirs->alpha0, dirs->dalpha, s));
    }
    return RTW_OK;
}

int rtw_field_caustic(const rtw_rays* rays_c, const rtw_dirs* dirs, const rtw_caustic_params* cp, int flags,
                      void* field_out, uint8_t* mask_out, double* weights_out, void* stream)
{
    rtw_rays* rays = const_cast<rtw_rays*>(rays_c);
    if (!rays || !dirs || !cp || !field_out) return fail(RTW_ERR_ARG, "rtw_field_caustic: null pointer");
    if (rays->grid != RTW_GRID_SQUARE || rays->nobj != 1 || !rays->st.aux || rays->st.near_r != 0.0 ||
        rays->precision != RTW_FP64)
        return fail(RTW_ERR_ARG, "rtw_field_caustic: one object on a square grid traced in RTW_FP64 with "
                                 "RTW_TRACE_APERTURE (far field) is required");
    const ObjDev& o = rays->objs[0];
    if (o.src_mode != 0 || o.shape_e != 1.0)
        return fail(RTW_ERR_ARG, "rtw_field_caustic: an ellipsoid in a plane wave is required");
    if (flags & ~RTW_FIELD_PER_ORDER) return fail(RTW_ERR_ARG, "rtw_field_caustic: flags 0 or RTW_FIELD_PER_ORDER");
    if (dirs->kind != RTW_DIRS_GRID) return fail(RTW_ERR_ARG, "rtw_field_caustic: a (theta, phi) grid is required");
    int rc = rtw::host::check_grid_dirs(dirs, false, "rtw_field_caustic");
    if (rc != RTW_OK) return rc;
    const int tt = cp->tile_theta ? cp->tile_theta : 16, tp = cp->tile_phi ? cp->tile_phi : 16;
    if (tt < 1 || tp < 1 || tt * tp > 256)
        return fail(RTW_ERR_ARG, "rtw_field_caustic: tiles of 1 to 256 directions (%d x %d)", tt, tp);
    const double aw = std::pow(o.lambda / o.lmax, 2.0 / 3.0), fw = 1.0 / std::sqrt(o.k0 * o.lmax);
    const bool po_default = cp->po_full == 0.0 && cp->po_end == 0.0;
    const bool cone_default = cp->cone_full == 0.0 && cp->cone_end == 0.0;
    const double po_full = po_default ? 1.5 * aw : cp->po_full, po_end = po_default ? 3.0 * aw : cp->po_end;
    const double cone_full = cone_default ? 3.0 * aw + 3.0 * fw : cp->cone_full;
    const double cone_end = cone_default ? 3.0 * aw + 6.0 * fw : cp->cone_end;
    if (!(po_full >= 0.0 && po_end > po_full && cone_full >= 0.0 && cone_end > cone_full))
        return fail(RTW_ERR_ARG, "rtw_field_caustic: 0 <= po_full < po_end and 0 <= cone_full < cone_end");
    const int nt = dirs->n_theta, nph = dirs->n_phi;
    const double rho_bound = 0.5 * (tt * kPi / nt + tp * kPi / nph);
    if (!(rho_bound + cone_end < 0.5 * kPi))
        return fail(RTW_ERR_ARG, "rtw_field_caustic: a tile's cone reaches pi/2 (radius bound %g + cone_end %g)",
                    rho_bound, cone_end);
    const int np = rays->np;
    const int p_min = cp->p_min ? cp->p_min : 1;
    if (p_min < 0 || p_min > np) return fail(RTW_ERR_ARG, "rtw_field_caustic: p_min %d beyond the orders", p_min);
    const bool per_order = (flags & RTW_FIELD_PER_ORDER) != 0;
    cudaStream_t s = (cudaStream_t)stream;
    rtw::host::GridPlan g;
    rtw::host::GridWs w;
    rtw::DirSet d;
    rc = grid_prepare(rays, dirs, &g, &w, &d, s);
    if (rc != RTW_OK) return rc;
    const long long ndir = (long long)nt * nph;
    const long long ntiles = (long long)((nt + tt - 1) / tt) * ((nph + tp - 1) / tp);
    const long long nblocks = ((o.nx + 15) / 16) * ((o.ny + 15) / 16);
    const size_t per_bytes = sizeof(double) * 4 * (size_t)np * (size_t)ndir;
    const size_t sc_bytes = rtw::caustic_scratch_bytes(ndir, ntiles, nblocks);
    // the per-order field (the caller's output with RTW_FIELD_PER_ORDER) and the correction's scratch
    char* block = nullptr;
    const size_t off_sc = per_order ? 0 : align_up(per_bytes, 256);
    if (cudaMallocAsync((void**)&block, off_sc + sc_bytes, s) != cudaSuccess)
        return fail(RTW_ERR_NOMEM, "rtw_field_caustic: scratch of %zu bytes", off_sc + sc_bytes);
    double* per = per_order ? (double*)field_out : (double*)block;
    void* scratch = block + off_sc;
    auto run = [&]() -> int {
        RTW_CUDA(cudaMemsetAsync(per, 0, per_bytes, s));
        int r = rtw::host::grid_field_run(rays->objs.data(), rays->d_objs, 1, rays->st, g, dirs, d, true, per,
                                          nullptr, w, 0, 0, status_word(rays->device),
                                          newton_counter(rays->device), s, &rays->slices);
        if (r != RTW_OK) return r;
        if (weights_out) RTW_CUDA(cudaMemsetAsync(weights_out, 0, sizeof(double) * (size_t)np * (size_t)ndir, s));
        for (int p = p_min; p < np; ++p)
            RTW_CUDA(rtw::launch_caustic_order(rays->st, o, p, nt, nph, tt, tp, po_full, po_end, cone_full, cone_end,
                                               w.mask_words, per, weights_out, scratch, s));
        RTW_CUDA(rtw::launch_caustic_finish(w.mask_words, ndir, per, per_order ? nullptr : (double*)field_out, np, s));
        if (mask_out)
            RTW_CUDA(rtw::launch_finalize_mask(w.mask_words, mask_out, rays->d_objs, 1, ndir, 1, nt, nph, 0.0, 0.0, s,
                                               nullptr));
        return RTW_OK;
    };
    rc = run();
    cudaFreeAsync(block, s);
    return rc;
}

int rtw_newton_failures(void* stream, int64_t* count)
{
    if (!count) return fail(RTW_ERR_ARG, "rtw_newton_failures: null pointer");
    int dev = 0;
    RTW_CUDA(cudaGetDevice(&dev));
    RTW_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned long long* p = newton_counter(dev);
    if (!p) return fail(RTW_ERR_CUDA, "rtw_newton_failures: counter");
    unsigned long long v = 0;
    RTW_CUDA(cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost));
    RTW_CUDA(cudaMemset(p, 0, sizeof(v)));
    *count = (int64_t)v;
    return RTW_OK;
}

int rtw_sync_status(void* stream)
{
    int dev = 0;
    RTW_CUDA(cudaGetDevice(&dev));
    RTW_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned int* p = status_word(dev);
    if (!p) return fail(RTW_ERR_CUDA, "rtw_sync_status: status word");
    unsigned int v = 0;
    RTW_CUDA(cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost));
    RTW_CUDA(cudaMemset(p, 0, sizeof(v)));
    if (v & rtw::kStatusCapacity) return fail(RTW_ERR_CAPACITY, "a device buffer or bounded loop ran out");
    if (v & rtw::kStatusTimeout) return fail(RTW_ERR_TIMEOUT, "a bounded device iteration gave up");
    if (v & rtw::kStatusNumeric) return fail(RTW_ERR_NUMERIC, "a non-finite or singular value was met");
    return RTW_OK;
}

}  // extern "C"
