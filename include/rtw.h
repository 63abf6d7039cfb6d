/*
 * rtw.h -- C ABI of the GB300 Ray Theory of Waves (RTW) far-field library (librtw.so).
 *
 * The calls follow the paper's statement of the problem (Ren et al., "Ray Theory of Waves",
 * arXiv:2403.13856): an object (shape and refractive index, Fig. 3 caption), an incident plane
 * wave (wavelength, direction, polarisation), and the complex far field of all rays summed at the
 * observation directions ("Strategy of Ray Theory of Waves": rays traced over intermediate
 * variables t, then interpolated to the directions of interest).
 *
 * Conventions.  Lengths in micrometres.  The host medium has index 1; m is the index of the
 * object relative to it.  The incident wave is E_inc = (jones_x, jones_y, 0) e^{i k0 z} with the
 * time factor e^{-i w t}.  The scattered far field is E(r s) = F(s) e^{i k0 r} / r, F in um, given
 * as the complex pair (F_theta, F_phi) on the unit vectors e_theta, e_phi of s = (theta, phi)
 * (theta from +z, phi from +x).  |F|^2 is the differential cross-section in um^2.
 *
 * Memory.  Handles (rtw_object, rtw_rays) are opaque and owned by the library; their device
 * memory is allocated by the library with cudaMalloc and freed by the destroy functions.
 * Every other pointer argument marked "device" is a caller-owned device buffer (for example a
 * torch tensor) that the library reads or writes but never frees.  Host pointers are read during
 * the call only.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is enqueued
 * asynchronously on it; argument errors are reported synchronously by the return value.  Errors
 * raised inside kernels (bounded loops that ran out, capacity) set a status word that
 * rtw_sync_status() reads after synchronising the stream.
 *
 * Errors.  Every call returns RTW_OK (0) or a negative RTW_ERR_* code; rtw_last_error() gives a
 * one-line message for the calling thread.  No C++ exception crosses the ABI and no call falls
 * back to a CPU implementation: without a usable CUDA device every compute call fails with
 * RTW_ERR_CUDA.
 */
#ifndef RTW_H
#define RTW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define RTW_OK 0
#define RTW_ERR_ARG (-1)         /* invalid argument (null pointer, size, range)          */
#define RTW_ERR_UNSUPPORTED (-2) /* valid but not implemented (absorbing m, oblique wave)  */
#define RTW_ERR_CUDA (-3)        /* a CUDA runtime call failed or no device is usable       */
#define RTW_ERR_CAPACITY (-4)    /* a bounded device buffer or loop ran out                 */
#define RTW_ERR_TIMEOUT (-5)     /* a bounded device iteration gave up                      */
#define RTW_ERR_NUMERIC (-6)     /* non-finite values where finite ones are required        */
#define RTW_ERR_NOMEM (-7)       /* host or device allocation failed                        */

/* ---- enums and flags ---- */
#define RTW_GRID_FAN 0    /* 1-D fan of impact parameters b_j = -w + (j + 1/2) 2w/n in the plane
                             of azimuth fan_phi through the projected centre (w: half-chord)    */
#define RTW_GRID_SQUARE 1 /* 2-D square grid x_i = cx + (i + 1/2 - nx/2) h (same for y) covering
                             the projected cross-section; points inside it are rays             */

#define RTW_FP64 0  /* every step in double precision                                          */
#define RTW_MIXED 1 /* geometry, Fresnel and curvature in single precision; intersection points,
                       optical path and phase in double precision                              */
#define RTW_DFLOAT 2 /* every step of the trace in double-float (pairs of single-precision
                        numbers, about 48 significant bits; single-precision exponent range);
                        intersection points and optical path in double precision           */

#define RTW_DENSE 0  /* interpolation of the dense ray map (the paper's RTW strategy)           */
#define RTW_NEWTON 1 /* hits refined by Newton steps on the exact FP64 trace (Eq. WavefrontEqVec
                        gives the Jacobian ds/d(x, y) = Q' T), each step halved until the
                        residual decreases; on square grids the root must lie within 8 h of the
                        interpolated impact point.  A hit whose iteration does not converge
                        keeps its interpolated value and is counted (rtw_newton_failures)        */

#define RTW_DIRS_PLANE 0 /* in-plane angles alpha_k = alpha0 + k dalpha, k < n_theta, measured
                            from +z toward (cos fan_phi, sin fan_phi, 0); fan grids only        */
#define RTW_DIRS_GRID 1  /* cell-centred theta_i = (i + 1/2) pi / n_theta,
                            phi_j = -pi + (j + 1/2) 2 pi / n_phi, index i * n_phi + j           */
#define RTW_DIRS_LIST 2  /* n_list directions (theta, phi) read from list (device, n_list x 2
                            doubles, theta from +z, phi from +x); square grids only            */

#define RTW_FIELD_PER_ORDER 1 /* output one (F_theta, F_phi) pair per order instead of the sum */
#define RTW_FIELD_PO 2        /* fan grids: physical-optics integral around in-plane folds      */
#define RTW_FIELD_NEAR_FOLDS 4 /* with RTW_NEWTON: refine only the hits within 2 deg of an
                                  in-plane fold of their order (rainbow windows)                 */

#define RTW_TRACE_APERTURE 1 /* keep the exit-wave data the PO integrals need (fans; square grids
                                in RTW_FP64 for rtw_field_po2d): 144 B more per (ray, order)      */

#define RTW_MASK_CAUSTIC 1u /* a cell straddling a fold or flagged near-caustic covers it     */
#define RTW_MASK_AXIAL 2u   /* within 2 lambda / min(a, b, c) of the forward or backward axis  */
#define RTW_MASK_PO 4u      /* value replaced (fully or in part) by the PO integral            */

/* ---- descriptors ---- */

/* Object: ellipsoid of semi-axes (a, b, c) along its body axes, rotated body -> world by the unit
 * quaternion quat = (w, x, y, z) (|quat| = 1 within 1e-9), centred at center.  m_re is the
 * refractive index relative to the host; m_im must be 0 (absorbing objects: RTW_ERR_UNSUPPORTED).
 * shape_e: 0 or 1 for the ellipsoid; e > 1 for the superellipsoid |u|^(2e) + |v|^(2e) + |w|^(2e) = 1
 * with (u, v, w) the body coordinates divided by (a, b, c), a smooth convex body between the
 * ellipsoid and the box (the Introduction's principle (iii): the wavefront equation needs of the
 * surface only its normal and curvature matrix at each point, here from the gradient and Hessian
 * of that function).  A superellipsoid takes rtw_trace with a square grid and RTW_FP64 (far field
 * or observe_radius beyond |center| + max(a, b, c) 3^((1 - 1/e) / 2)), a plane wave or a point source
 * outside its bounding ellipsoid of semi-axes (a, b, c) 3^((1 - 1/e) / 2), and rtw_field in
 * RTW_DENSE mode without RTW_FIELD_PO; its ray grid covers the rays that meet that bounding
 * ellipsoid, so n_rays counts those.  Other entry points answer RTW_ERR_UNSUPPORTED. */
typedef struct {
    double a, b, c;
    double quat[4];
    double center[3];
    double m_re, m_im;
    double shape_e;
} rtw_object_desc;

/* Incident wave.  kind RTW_INCIDENT_PLANE: plane wave with direction dir (must be (0, 0, 1)) and
 * Jones vector (E_x, E_y) on the unit vectors x, y.  kind RTW_INCIDENT_POINT (an incident wave that
 * is not plane: Phi_i of Eq. PhaseTotal, Q_i of Eq. WavefrontEqVec, A_0 of Eq. IntVCRM): a point
 * source at `source` (um), outside the object (else RTW_ERR_ARG), field e^{ik rho} p_perp / rho at
 * distance rho with p = jones_x e1 + jones_y e2 made perpendicular to the ray; e1, e2 span the plane
 * through the object's centre perpendicular to a = (center - source) / |center - source| (e1 = x,
 * or y when a is within 26 deg of x, made perpendicular to a; e2 = a x e1).  Rays leave the source
 * through the square grid of that plane (a ray's (x, y) are its coordinates there, from the
 * centre); square grids and RTW_FP64 only; the far field F is then dimensionless.
 * wavelength_um: in the host medium. */
enum { RTW_INCIDENT_PLANE = 0, RTW_INCIDENT_POINT = 1 };
typedef struct {
    double wavelength_um;
    double dir[3];
    double jones_re[2], jones_im[2];
    int kind;
    double source[3];
} rtw_incident;

/* Ray grid and trace options.  n_rays: fan -> exact number of rays; square -> target count inside
 * the projected cross-section (spacing h = sqrt(pi / (sqrt(det S) n_rays)), S the matrix of the
 * projected ellipse), unless spacing > 0 gives h directly.  p_max: orders 0..p_max, p_max <= 15.
 * observe_radius: 0 for the far field; R > 0 (square grids and RTW_FP64 only, R beyond |center| +
 * max semi-axis of every object (of its bounding ellipsoid for a superellipsoid), else RTW_ERR_ARG /
 * RTW_ERR_UNSUPPORTED) records every ray where it
 * crosses the sphere |M| = R about the origin instead: the field at a finite point M (Eqs.
 * IntVCRM, DivFactVCRM with the Gaussian curvature kappa_GM at M, and PhasePath to r_M), whose
 * last leg of length t contributes 1 / det(I + t Q') to the divergence factor, its focal lines to
 * N_f and k t to the phase; the records' directions (rtw_rays_export) are then the unit vectors
 * M / R of the crossing points and their fields the fields at M. */
typedef struct {
    int grid;
    int p_max;
    int precision;
    int flags;
    int64_t n_rays;
    double spacing;
    double fan_phi;
    double observe_radius;
} rtw_trace_params;

/* Observation directions (the paper's "directions of interest"): kind RTW_DIRS_PLANE (n_theta,
 * alpha0, dalpha), RTW_DIRS_GRID (n_theta, n_phi) or RTW_DIRS_LIST (list, n_list; n_list <
 * 2^31; the list is binned on the device for each call and read during the call only).
 * cell_window limits a square-grid field to the cells [ix0, ix1) x [iy0, iy1) of the ray grid
 * (all four -1: every cell); it exists so that a sample of a full-size field can be checked
 * against an independent computation. */
typedef struct {
    int kind;
    int n_theta, n_phi;
    double alpha0, dalpha;
    int64_t cell_window[4];
    const double* list;
    int64_t n_list;
} rtw_dirs;

typedef struct rtw_object rtw_object;
typedef struct rtw_rays rtw_rays;

/* ---- objects ---- */

/* Validates `count` object descriptors and incident waves (inc[i] belongs to desc[i]) and uploads
 * them: quadric matrix W = R diag(a^-2, b^-2, c^-2) R^T, projected ellipse S (Schur complement of
 * W_zz), k0 = 2 pi / lambda.  *out receives a handle owned by the caller until
 * rtw_destroy_object.  Errors: RTW_ERR_ARG (null, count < 1, a, b, c, lambda <= 0, m <= 0,
 * m == 1, |quat| != 1, shape_e neither 0 nor >= 1, a source inside the object or the bounding
 * ellipsoid of a superellipsoid), RTW_ERR_UNSUPPORTED (m_im != 0, dir != (0,0,1)), RTW_ERR_CUDA,
 * RTW_ERR_NOMEM.  Synchronous. */
int rtw_create_object(const rtw_object_desc* desc, int count, const rtw_incident* inc, rtw_object** out);
void rtw_destroy_object(rtw_object* obj);

/* Host query of the ray grid rtw_trace would use for object `index`: spacing h (fan: 2w/n), nx,
 * ny (fan: n, 1).  Pure host arithmetic. */
int rtw_object_grid(const rtw_object* obj, int index, const rtw_trace_params* tp, double* h, int64_t* nx,
                    int64_t* ny);

/* ---- the per-ray trace (the hot path's first half) ---- */

/* Traces every ray of every object through its object and records, for each ray and order p, the
 * exit direction s, the far-field vector amplitude F = A e^{i (Phi_F + Phi_f)} (Eqs. IntVCRM,
 * DivFactVCRM, epsilon_VCRM, Fres, the WFC carried by Eq. WavefrontEqVec), the far-field phase Psi
 * (Eq. PhasePath) and the flags (valid, orientation, near-caustic, focal-line count).
 * If *inout is NULL a new rays handle is allocated; otherwise it is reused when its capacity
 * suffices and reallocated when not.  Asynchronous on `stream`. */
int rtw_trace(rtw_object* obj, const rtw_trace_params* tp, void* stream, rtw_rays** inout);

/* Sizes of a rays handle: rays per order over all objects (square grids count misses), number of
 * orders, number of objects. */
int rtw_rays_info(const rtw_rays* rays, int64_t* rays_per_order, int* n_orders, int* n_objects);

/* Copies the state of rays [first, first + count) of `order` into caller device buffers, any of
 * which may be NULL: s_out (count x 3 double), F_out (count x 6 double: re, im of x, y, z),
 * psi_out (count double), flags_out (count uint32: bit 0 valid, bit 1 orientation +, bit 2
 * near-caustic, bits 8-15 focal-line count).  Asynchronous. */
int rtw_rays_export(const rtw_rays* rays, int order, int64_t first, int64_t count, double* s_out,
                    double* F_out, double* psi_out, uint32_t* flags_out, void* stream);
void rtw_destroy_rays(rtw_rays* rays);

/* Traces n explicit impact points xy (device, n x 2, um, in the plane z = const) of object
 * `index` for orders 0..p_max in double precision and writes the same records as
 * rtw_rays_export, laid out [n][p_max + 1] (s_out n x (p_max+1) x 3, and so on).  Asynchronous. */
int rtw_trace_points(const rtw_object* obj, int index, const double* xy, int64_t n, int p_max,
                     double* s_out, double* F_out, double* psi_out, uint32_t* flags_out, void* stream);

/* ---- the field (the hot path's second half) ---- */

/* Sums the complex amplitudes of all traced rays at the observation directions (principle iii of
 * the paper) by interpolating the ray map over the triangles (square grid) or segments (fan) of
 * neighbouring rays: a direction is owned by the cell whose image contains it (half-open rule),
 * F and Psi are interpolated with the barycentric weights of the central projection, and
 * F e^{i Psi} is added.  Cells whose corners disagree in focal-line count or orientation, or carry
 * the near-caustic flag, add nothing and mark the directions they cover (RTW_MASK_CAUSTIC).  With
 * RTW_FIELD_PO (fan grids traced with RTW_TRACE_APERTURE) the field near every in-plane fold is
 * the physical-optics integral over the exit wave ("Diffraction effect correction based on VCRM").
 * mode RTW_NEWTON replaces each interpolated hit by the exact ray found by Newton steps on the FP64
 * trace from the interpolated impact point (all hits, or, on fans with RTW_FIELD_NEAR_FOLDS, those
 * within 2 deg of a fold).
 * field_out (device): [objects][directions][orders or 1][2] complex128 (F_theta, F_phi), zeroed
 * and written.  For rays traced with observe_radius R > 0 the directions u name the points M = R u
 * and field_out is [objects][directions][orders or 1][3] complex128 (E_r, E_theta, E_phi), the field
 * at M for a unit incident wave (the ray through M need not be radial); mode RTW_DENSE only, no PO.
 * mask_out (device, optional): [objects][directions] uint8.  Asynchronous, except with superellipsoids
 * among the objects (their ray branches per direction multiply with the order: rounded edges fan
 * the rays out again at every internal reflection) or direction grids of more than about 2^27 / (p_max
 * + 1) directions: the field is then summed in slices of ray-grid rows sized to the hit list, each
 * classified first and its pair count read back (the stream is synchronised once per slice);
 * RTW_ERR_CAPACITY when a single row does not fit. */
int rtw_field(const rtw_rays* rays, const rtw_dirs* dirs, int mode, int flags, void* field_out,
              uint8_t* mask_out, void* stream);

/* 2-D physical optics of one order over an aperture of rays ("Diffraction effect correction based
 * on VCRM": near a singularity the field is a diffraction integral of the complex amplitudes the rays
 * carry; this is Kirchhoff's integral over a plane, both directions numerical, where RTW_FIELD_PO
 * integrates one direction of a fan and takes the other by stationary phase).  The rays of the grid
 * vertices [window[0], window[1]] x [window[2], window[3]] carry their exit waves to the plane through
 * the object's centre with normal a = (axis_theta, axis_phi): crossing point x = r + tau s, field
 * U = E' sqrt(D_legs / |det(I + tau Q')|) (-i)^{N_f} e^{i k0 (L + tau)} (focal lines of the last
 * stretch counted forward for tau > 0, undone for tau < 0); dA = the plane's area per grid cell from
 * central differences of the neighbours' crossing points; each ray weighted by the angle g of its
 * exit direction to a: 1 for g <= cone_full, cos^2 to 0 at cone_end (the window should hold every ray
 * within cone_end; its own edges are not tapered).  F(s) = k0 / (2 pi i) sum w U dA e^{-i k0 s.x},
 * the far field of that order (same convention as rtw_field), near the directions of the rays kept.
 * rays: one object, square grid, RTW_FP64, traced with RTW_TRACE_APERTURE, far field.  dirs (device,
 * read during the call): n_dirs (theta, phi) pairs, 1 <= n_dirs < 2^31.  field_out (device):
 * [n_dirs][2] complex128 (F_theta, F_phi), overwritten.  Errors: RTW_ERR_ARG (null, rays not so traced,
 * order outside [0, p_max], a window beyond the grid or under 3 x 3 vertices or over 2^31 rays,
 * not 0 <= cone_full < cone_end <= pi/2), RTW_ERR_CUDA.  Asynchronous; a scratch block of 152 B per
 * window ray and 48 B per direction is allocated and freed in stream order.  n_used (host, optional):
 * receives the number of rays in the sum (the call then synchronises the stream to read it). */
typedef struct {
    int order;
    int64_t window[4];
    double axis_theta, axis_phi;
    double cone_full, cone_end;
} rtw_po2d_params;
int rtw_field_po2d(const rtw_rays* rays, const rtw_po2d_params* pp, const double* dirs, int64_t n_dirs,
                   void* field_out, int64_t* n_used, void* stream);

/* 2-D physical optics at the 3-D caustics of a square-grid far field (the "Diffraction effect
 * correction based on VCRM" carried to three dimensions, where the paper leaves it "under study").
 * The field of rtw_field (RTW_DENSE), and for every order p >= p_min: the directions C_p that cell
 * triangles of order p which are not consistent cover (the directions rtw_field masks for that
 * order) set the weight s_p(u) = ramp(angle from u to the nearest direction of C_p) -- 1 up to
 * po_full, cos^2 down to 0 at po_end -- and the field of that order becomes
 *     (1 - s_p) F_rays + s_p F_PO,
 * F_PO the Kirchhoff integral of the exit waves over a plane, as rtw_field_po2d: for the directions
 * of one tile of tile_theta x tile_phi grid directions the plane passes through the object centre
 * normal to the tile's centre direction a, every ray of order p is weighted by the angle of its exit
 * direction to a (1 up to rho + cone_full, cos^2 to 0 at rho + cone_end, rho the largest angle from a
 * to a direction of the tile), and F_PO(u) = k0 / (2 pi i) (u . a) sum w U dA e^{-i k0 u . x}, the
 * plane's far field (Rayleigh-Sommerfeld).  Widths left 0 take the fan's: with Aw = (lambda / L)^(2/3)
 * and Fw = 1 / sqrt(k0 L), L the largest semi-axis, po_full = 1.5 Aw, po_end = 3 Aw, cone_full =
 * 3 Aw + 3 Fw, cone_end = 3 Aw + 6 Fw.  The integral samples the plane at the rays' crossing points:
 * like rtw_field_po2d it is accurate to about 1e-2 of the field at grid spacings near 0.1 um, and
 * converges as the spacing shrinks.  tile_theta, tile_phi 0 take 16; p_min 0 takes 1 (order 0 of
 * an ellipsoid has no fold).
 * rays: one ellipsoid in a plane wave, square grid, RTW_FP64, traced with RTW_TRACE_APERTURE, far
 * field.  dirs: RTW_DIRS_GRID, cell_window all -1.  flags: 0 or RTW_FIELD_PER_ORDER.  field_out
 * (device): as rtw_field.  mask_out (device, optional): as rtw_field, except that the caustic bit is
 * kept only on the directions of C_p where s_p < 1 (none for po_full > 0) or p < p_min, and every
 * direction with s_p > 0 for some p has RTW_MASK_PO.  weights_out (device, optional):
 * [directions][orders] doubles, s_p (0 for p < p_min).  Errors: RTW_ERR_ARG (rays or directions not
 * as above, tile_theta or tile_phi negative or tile_theta tile_phi above 256, 0 <= po_full < po_end
 * and 0 <= cone_full < cone_end violated, a tile's radius bound (tile_theta pi / n_theta + tile_phi
 * pi / n_phi) / 2 plus cone_end reaching pi / 2, p_min beyond the orders), RTW_ERR_NOMEM, RTW_ERR_CUDA.
 * Asynchronous; scratch (16 bytes per direction, 32 per direction and order without
 * RTW_FIELD_PER_ORDER, 16 per 256 rays) is allocated and freed in stream order.  Cost: per order, the
 * plane crossing of every ray whose 16 x 16 block meets a tile's cone, and one FP32 sincos per
 * (ray in the cone, direction of the tile). */
typedef struct {
    int tile_theta, tile_phi;
    double po_full, po_end;
    double cone_full, cone_end;
    int p_min;
} rtw_caustic_params;
int rtw_field_caustic(const rtw_rays* rays, const rtw_dirs* dirs, const rtw_caustic_params* cp, int flags,
                      void* field_out, uint8_t* mask_out, double* weights_out, void* stream);

/* ---- many objects in one launch sequence ---- */

/* Options of rtw_far_field_batch.  n_rays (host, one entry per object, read during the call) is
 * each object's target ray count inside its projected cross-section, as rtw_trace_params.n_rays
 * for a square grid.  chunk_ray_orders bounds the ray state held at once, counted in
 * (ray, order) pairs over the objects of a chunk (0: 2^29, about 62 GB); an object larger than
 * the bound is a chunk of its own.  trace_variant (0: 2) selects the persistent trace kernel's
 * block size and register cap, 1..5 = (64 threads), (128), (256), (128, 3 CTAs per SM),
 * (256, 2 CTAs per SM); trace_ctas_per_sm (0: as many as fit) its resident CTAs per SM;
 * classify_block (0: 256; 64, 128 or 256) the block size of the grid classification kernel.
 * use_graph = 1 records the whole launch sequence in a CUDA graph on the first call and replays
 * it on later calls whose objects, options, directions and output pointers are the same.
 * timing = 1 records CUDA events around the trace and the field of every chunk (eager runs only,
 * read with rtw_batch_times).  mode: RTW_DENSE, or RTW_NEWTON (every interpolated hit replaced by
 * the exact ray, as in rtw_field). */
typedef struct {
    int p_max;
    int precision;
    const int64_t* n_rays;
    int64_t chunk_ray_orders;
    int trace_variant;
    int trace_ctas_per_sm;
    int classify_block;
    int use_graph;
    int timing;
    int mode;
} rtw_batch_params;

typedef struct rtw_batch rtw_batch;

/* The far field of every object of obj (its own wave, square ray grid) on the same (theta, phi)
 * direction grid: rtw_trace + rtw_field of the square-grid path, object by object, in one
 * sequence of launches.  Objects are split into chunks of at most chunk_ray_orders ray state;
 * each chunk is traced by one persistent kernel that takes work items (object, 256 consecutive
 * rays) from a counter, then its field is accumulated in launch groups of objects.
 * dirs: kind RTW_DIRS_GRID, cell_window all -1.  flags: 0 or RTW_FIELD_PER_ORDER.
 * field_out (device): [objects][directions][orders or 1][2] complex128, zeroed and written;
 * mask_out (device, optional): [objects][directions] uint8.  *inout: NULL on the first call (a
 * handle owning the ray-state block, the workspace and the graph is created) or a handle from an
 * earlier call (reused, grown when needed).  Argument errors return before any work; errors of
 * kernels are read by rtw_sync_status.  Asynchronous on `stream`. */
int rtw_far_field_batch(const rtw_object* obj, const rtw_batch_params* bp, const rtw_dirs* dirs, int flags,
                        void* field_out, uint8_t* mask_out, rtw_batch** inout, void* stream);

/* Sizes of the last call: rays over all objects (square grids count misses), chunks, and 1 when
 * the call replayed a recorded graph. */
int rtw_batch_info(const rtw_batch* b, int64_t* total_rays, int* n_chunks, int* replayed);

/* Trace and field times (ms, summed over chunks) of the last call made with timing = 1;
 * synchronises with its events. */
int rtw_batch_times(const rtw_batch* b, double* trace_ms, double* field_ms);

void rtw_destroy_batch(rtw_batch* b);

/* ---- learned proposal of entry points ----
 * The paper has no learned component.  This part proposes, for an exit direction s and order p,
 * where a ray must enter the object to leave along s, so that Newton steps on the exact trace
 * (Eq. WavefrontEqVec gives their Jacobian) can find the ray without tracing a dense grid.
 * One network per order: 16 features -> 3 hidden layers of 128 (GELU, tanh form) -> 16 outputs.
 * Features: s (3), the rotation body -> lab of the object (9, row-major), its semi-axes over the
 * largest (3), m - 1.  Outputs: 4 candidate entry points uv (outputs 2k, 2k+1) in unit-disk
 * coordinates of the projected section (d = (x - cx, y - cy), S = L L^T the Cholesky factor of
 * the projected ellipse, uv = L^T d), 4 logits (outputs 8..11), 4 unused.  Parameters per network
 * (RTW_MLP_NPARAM floats): W1 (128 x 16), b1, W2 (128 x 128), b2, W3, b3, W4 (16 x 128), b4, each
 * W row-major (out x in).  Products run on the tensor cores in bfloat16 with FP32 accumulation;
 * the master parameters and Adam moments are FP32.  Feature rows X are bfloat16 (16 per row),
 * passed as void*. */
#define RTW_MLP_NPARAM 37264

typedef struct rtw_mlp rtw_mlp;

/* n_orders networks (orders 0..n_orders-1) with initial parameters init (host, n_orders x
 * RTW_MLP_NPARAM floats, or NULL for zeros); Adam state zero.  Synchronous. */
int rtw_mlp_create(int n_orders, const float* init, rtw_mlp** out);
void rtw_mlp_destroy(rtw_mlp* m);
/* Host copies of one network's parameters, Adam moments and step (any pointer may be NULL), and
 * their restoration (checkpoint / resume).  Synchronous. */
int rtw_mlp_get(const rtw_mlp* m, int order, float* theta, float* adam_m, float* adam_v, int64_t* step);
int rtw_mlp_set(rtw_mlp* m, int order, const float* theta, const float* adam_m, const float* adam_v, int64_t step);

/* Training samples from the exact FP64 trace: ray i enters object obj_index[i] (device int32) at
 * unit-disk point uv[i] (device, n x 2 double); for every order p <= p_max, row p n + i of X
 * (device, bf16, 16 per row) gets the features of its exit direction, T (device, 2 floats per row)
 * the target uv and valid (device, uint8) the row's label: 0 when order p does not leave the
 * object (or the index is outside [0, count)), else 1 + (N_f mod 4) with N_f the ray's focal-line
 * count, the head that learns its branch (the branches of one direction and order differ in N_f).
 * Asynchronous. */
int rtw_mlp_samples(const rtw_object* obj, const double* uv, const int32_t* obj_index, int64_t n, int p_max,
                    void* X, float* T, uint8_t* valid, void* stream);
/* Y (device, rows x 16 float) = network `order` applied to X (device, rows x 16 bf16), on the
 * tensor cores.  X and Y must start on 16-byte boundaries (RTW_ERR_ARG otherwise).  Asynchronous; a
 * bounded wait inside the kernel that gives up is reported as RTW_ERR_TIMEOUT by rtw_sync_status. */
int rtw_mlp_forward(const rtw_mlp* m, int order, const void* X, int64_t rows, float* Y, void* stream);
/* The hidden activation of rtw_mlp_forward's kernel on n values (device x, y, float): its GELU (tanh
 * form, single precision, before the kernel rounds it to bfloat16), for tests of the activation
 * against its definition.  Errors: RTW_ERR_ARG.  Asynchronous. */
int rtw_mlp_activation_eval(const float* x, float* y, int64_t n, void* stream);
/* Gradient of the mean loss over the labelled rows (valid != 0) into the network's gradient
 * buffer: for each row head valid - 1 carries the squared distance to the target uv, and beta
 * times the softmax cross-entropy of the logits towards that head is added.  loss_out (device double, may be NULL)
 * receives the loss.  The forward pass (keeping every hidden layer's pre-activations and bf16
 * activations), the backward data pass and the weight gradients run on the tensor cores (tcgen05,
 * bf16 operands, f32 accumulation in tensor memory).  X (rows x 16 bf16) must start on a 16-byte
 * boundary and rows < 2^31 (RTW_ERR_ARG otherwise).  Deterministic (fixed summation order).
 * Asynchronous; a bounded wait inside a kernel that gives up is reported as RTW_ERR_TIMEOUT by
 * rtw_sync_status. */
int rtw_mlp_grad(rtw_mlp* m, int order, const void* X, const float* T, const uint8_t* valid, int64_t rows, float beta,
                 double* loss_out, void* stream);
/* Copies the gradient buffer (RTW_MLP_NPARAM floats) to grad (host or device).  Asynchronous. */
int rtw_mlp_grad_get(const rtw_mlp* m, int order, float* grad, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with learning rate lr on the
 * gradient grad (device, RTW_MLP_NPARAM floats) or, when NULL, the network's own.  Asynchronous. */
int rtw_mlp_adam(rtw_mlp* m, int order, float lr, const float* grad, void* stream);

/* Options of rtw_field_learned: orders 0..p_max (networks 0..p_max of the rtw_mlp handle);
 * heads whose softmax weight is below p_min (0: 0.05) are not tried; at most max_steps
 * double-precision Newton steps per head (0: 3); convergence at |s - target| < tol (0: per object
 * min(1e-6, 1e-4 / (k0 max(a, b, c))), which keeps the phase error of a converged ray below
 * 1e-4 rad); rows (object, direction) per launch sequence chunk_rows (0: 2^24); a step is halved
 * at most max_halvings times (0: 3, range 1..30) before its head is given up.  precision
 * RTW_MIXED first approaches each root on the single-precision trace (at most 6 steps, to
 * |s - target| < 3e-6) and then takes the double-precision steps; RTW_FP64 (0) takes only the
 * latter.  fallback_rays (host, one per object, or NULL): the dense fallback -- every row where a
 * confident head's steps did not converge (root-count bit 7) is redone by the dense path with a
 * square ray grid of fallback_rays[i] rays and its per-order values replace the learned ones of the
 * uncertain orders (needs RTW_FIELD_PER_ORDER; one read-back and a trace per object with such
 * rows). */
typedef struct {
    int p_max;
    float p_min;
    int max_steps;
    double tol;
    int64_t chunk_rows;
    int max_halvings;
    int precision;
    const int64_t* fallback_rays;
} rtw_learned_params;

/* The far field of every object of obj on the (theta, phi) grid of dirs from learned proposals:
 * for each direction s and order p, network p (features of s and the object) proposes 4 entry
 * points (moved onto radius 0.999 of the unit disk when beyond it); each head with softmax
 * weight >= p_min seeds Newton steps on the exact FP64 trace (as RTW_NEWTON, at most max_steps
 * steps of at most max_halvings halvings each, no distance bound); a root within 1e-6 max(a, b, c) of
 * an earlier root of the same direction and order is the same ray and is dropped; every other
 * root adds its exact F e^{i Psi}, except a near-caustic root, which marks the direction
 * (RTW_MASK_CAUSTIC) instead.  A branch that no head finds is missing from the sum: roots_out
 * (device, optional, [objects][directions][orders] uint8) reports the roots found (bits 0..6) and
 * marks with bit 7 the rows where a head the network is confident about did not converge, the rows
 * the dense fallback (lp->fallback_rays) redoes.  field_out and mask_out as
 * rtw_field (flags: 0 or RTW_FIELD_PER_ORDER).  Working memory is allocated stream-ordered and
 * freed before the call's work completes.  Asynchronous. */
int rtw_field_learned(const rtw_object* obj, const rtw_mlp* m, const rtw_learned_params* lp, const rtw_dirs* dirs,
                      int flags, void* field_out, uint8_t* mask_out, uint8_t* roots_out, void* stream);

/* ---- the fan path without allocation ----
 * The paper has no counterpart of this call: it serves programs that may not allocate device
 * memory themselves (a host application whose memory manager owns the device and forbids direct
 * cudaMalloc from plug-ins, or a loop that must not risk the device-wide synchronisation an
 * allocation can cause).  It traces a 1-D fan (tp: grid RTW_GRID_FAN, precision RTW_FP64) of the
 * object described by d and w and writes its far field on in-plane directions (dirs: kind
 * RTW_DIRS_PLANE) exactly as rtw_create_object + rtw_trace + rtw_field would, ray sum only
 * (flags: 0 or RTW_FIELD_PER_ORDER), into the caller's field_out and optional mask_out (device
 * buffers laid out as for rtw_field).  It allocates nothing: its working memory is a fixed array
 * of about 5.8 MB compiled into the library, present on every GPU that loads it until the process
 * exits.  Limits: n_rays * (p_max + 1) <= 65536 and n_theta <= 65536, larger sizes return
 * RTW_ERR_CAPACITY.  The first call on each device looks up the array's device address (with
 * that device current), so make the first call on a device before any stream capture.  All calls
 * on a device share the array: calls whose GPU work overlaps (several streams or host threads)
 * race and must be ordered by the caller.  Asynchronous on `stream`. */
int rtw_fan_field_static(const rtw_object_desc* d, const rtw_incident* w, const rtw_trace_params* tp,
                         const rtw_dirs* dirs, int flags, void* field_out, uint8_t* mask_out, void* stream);

/* ---- measurement ----
 * The paper has no counterpart of this call: it runs a throughput kernel of one floating-point
 * pipe, the denominator of the trace kernels' rooflines.  kind: RTW_PEAK_FP64 (DFMA),
 * RTW_PEAK_FP32 (FFMA) or RTW_PEAK_FP32X2 (packed fma.rn.f32x2); one launch of SMs x blocks_per_sm
 * (1..32) blocks of 256 threads, each thread running 8 independent fused multiply-add chains of
 * 16 iters (1..2^30) steps, no memory traffic.  *flops (host) receives the floating-point
 * operations of the launch (2 per FMA and lane).  sink: device buffer of one double, written only
 * if the chains reach a value they cannot reach (it keeps the compiler from removing them).
 * Asynchronous on `stream`: time it with events on that stream. */
#define RTW_PEAK_FP64 0
#define RTW_PEAK_FP32 1
#define RTW_PEAK_FP32X2 2
int rtw_pipe_peak(int kind, int64_t iters, int blocks_per_sm, void* sink, double* flops, void* stream);

/* ---- status ---- */

/* Synchronises `stream`, reads and clears the device status word of the library: RTW_OK or the
 * first RTW_ERR_* a kernel raised since the last call. */
int rtw_sync_status(void* stream);
/* Synchronises `stream`, then reads and clears the device's count of RTW_NEWTON refinements that
 * did not converge since the last call (their hits kept the interpolated value). */
int rtw_newton_failures(void* stream, int64_t* count);
const char* rtw_status_string(int status);
const char* rtw_last_error(void);
/* Library version string. */
const char* rtw_version(void);

#ifdef __cplusplus
}
#endif
#endif
