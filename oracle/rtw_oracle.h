/*
 * rtw_oracle.h -- plain FP64 CPU oracle of the Ray Theory of Waves (RTW) far field.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check of
 * __graft_entry__ and the CPU-baseline leg of bench.py may load this library.  It shares no
 * code, header, table or constant with the CUDA library under paper_2403_13856_gb300/.
 *
 * Paper: K. F. Ren et al., "Ray Theory of Waves", arXiv:2403.13856.
 *   principle (i)-(iii)           : a ray carries k, E and the WFC matrix Q (Introduction)
 *   Eq. (WavefrontEqVec)          : k' P' Q' P'^T = k_i P_i Q_i P_i^T + C n.(k'-k_i)
 *   Eq. (Theta-r)                 : P_ab = s_a . u_b (Appendix)
 *   Eq. (SnellVec)                : equal tangential wave-vector components
 *   Eq. (IntVCRM), (DivFactVCRM)  : A = A0 |eps| sqrt(D_p), D_p = |prod kappa_G ratios|
 *   Eq. (epsilon_VCRM), (Fres)    : Fresnel factor chain and coefficients from k_in, k_rn
 *   Eq. (PhasePath), (PhaseTotal) : optical path, Fresnel and focal-line phase
 *   "Strategy of RTW"             : trace over intermediate variables t, then interpolate
 *   "Diffraction effect correction": physical-optics integration near caustics
 *
 * Conventions (readings of the paper):
 *   incident plane wave along +z, E_inc = (jones_x, jones_y) e^{i k0 z}, time factor e^{-i w t};
 *   n outward normal of the object; C > 0 for a convex surface; Q = 1/R with R > 0 diverging;
 *   every focal line multiplies the field by e^{-i pi/2};
 *   far field E(r s) = F e^{i Psi} e^{i k0 r} / r with F in micrometres.
 */
#ifndef RTW_ORACLE_H
#define RTW_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Object parameters, flat: a b c qw qx qy qz cx cy cz m lambda jre_x jim_x jre_y jim_y kind sx sy sz e.
 * e >= 1 is the superellipsoid exponent: the surface is sum_i |u_i|^(2e) = 1 with u the body coordinates
 * divided by the semi-axes (a, b, c); e = 1 is the ellipsoid.  For e > 1 the square ray grid covers
 * the silhouette of the bounding ellipsoid of semi-axes (a, b, c) 3^((1 - 1/e) / 2) (with a point source:
 * the ellipse of the source's plane whose rays meet that ellipsoid, the source outside it), and fans
 * are refused.
 * kind 0: plane wave along +z, Jones vector on (x, y).  kind 1: point source at (sx, sy, sz) outside
 * the object, field e^{ik rho} / rho p_perp at distance rho, p = jx e1 + jy e2 projected
 * perpendicular to the ray; rays leave the source through the plane through the centre
 * perpendicular to the axis a = (c - s) / |c - s|, e1 = x (or y when a is along x) made
 * perpendicular to a, e2 = a x e1, and a ray's (x, y) are its coordinates on that plane (from
 * the centre). */
#define OR_NPARAM 21

/* Per-(ray, order) record, flat doubles.  Integers are stored as doubles. */
enum {
    OR_VALID = 0,    /* 1 if this order leaves the object along a traced ray            */
    OR_NF = 1,       /* focal lines crossed, including the last leg to infinity          */
    OR_ORIENT = 2,   /* sign of the Jacobian of (x, y) -> s (oriented by z and by s)     */
    OR_NREFL = 3,    /* reflections on the path                                          */
    OR_S = 4,        /* exit direction s (3)                                             */
    OR_F = 7,        /* far-field vector amplitude, re/im of x, y, z (6), micrometres    */
    OR_PSI = 13,     /* far-field phase Psi (rad)                                        */
    OR_D = 14,       /* divergence factor D_p (um^2), far-field form                     */
    OR_DGEO = 15,    /* dA/dOmega = 1/|det J| (um^2)                                      */
    OR_J = 16,       /* J = ds/d(x, y) in the exit basis (v1, v2), row-major (4)          */
    OR_V1 = 20,      /* exit wavefront basis vector v1 (3)                                */
    OR_V2 = 23,      /* exit wavefront basis vector v2 (3)                                */
    OR_REXIT = 26,   /* exit point (3)                                                    */
    OR_Q = 29,       /* exit WFC matrix in (v1, v2), row-major (4)                         */
    OR_E = 33,       /* exit Jones components along v1, v2: re, im, re, im (4)            */
    OR_DLEGS = 37,   /* product of the internal legs' divergence factors                  */
    OR_NFLEGS = 38,  /* focal lines crossed inside the object                             */
    OR_PATH = 39,    /* optical path from the plane z = 0 to the exit point (um)          */
    OR_POWER = 40,   /* power fraction carried by this order                              */
    OR_COSPROD = 41, /* product of |cos theta'| / |cos theta| over the interactions        */
    OR_CAUSTIC = 42, /* 1 if D_geo exceeds the caustic cap                                */
    OR_NFIELD = 48
};

/* Mask bits of a direction */
#define OR_MASK_CAUSTIC 1u  /* covered by a cell straddling a fold or flagged near-caustic */
#define OR_MASK_AXIAL 2u    /* within 2 lambda / min(a,b,c) of the forward or backward axis */
#define OR_MASK_PO 4u       /* value replaced (fully or partly) by the PO integral          */

/* Field flags */
#define OR_FIELD_PO 1       /* 1-D fan: physical-optics correction around in-plane folds    */
#define OR_FIELD_EXACT 2    /* evaluate every hit by Newton on the exact trace (O3); square
                               grids: root within 8 h of the interpolated impact point      */
#define OR_FIELD_EXACT_FOLDS 4 /* 1-D fan: O3 only for directions within 2 deg of an in-plane
                                  fold of the hit's order (rainbow windows), O2 elsewhere    */

typedef struct or_object or_object;

int or_object_size(void);
/* Fills *o from the flat parameter array; returns 0, or -1 on invalid parameters. */
int or_make_object(const double* p, or_object* o);

/* Helpers describing the ray grids of the oracle. */
double or_fan_halfwidth(const or_object* o, double fan_phi);
void or_square_grid(const or_object* o, int64_t n_target, double h_in, double* h, int64_t* nx,
                    int64_t* ny, double* x0, double* y0);
double or_caustic_cap(const or_object* o);
/* Geometry of the object: rotation body -> lab (row-major 9), semi-axes, centre, projected
 * ellipse S (row-major 4) and index m; any pointer may be NULL. */
void or_object_frame(const or_object* o, double* R9, double* semi, double* center, double* S4, double* m);

/* Traces one incident ray at impact point (x, y); out has (pmax+1)*OR_NFIELD doubles.
 * *p_inside receives the power still travelling inside after the last interaction.
 * Returns 1 if the ray hits the object, 0 otherwise. */
int or_trace_ray(const or_object* o, double x, double y, int pmax, double* out, double* p_inside);
/* Batch form, OpenMP over rays; xy is n x 2. */
void or_trace_rays(const or_object* o, const double* xy, int64_t n, int pmax, double* out,
                   int nthreads);

/* 1-D fan (rays of impact parameter b_j = -w + (j+1/2) 2w/nrays in the plane of azimuth
 * fan_phi).  Target directions are in-plane angles alpha (rad, (-pi, pi]) measured from +z
 * toward (cos fan_phi, sin fan_phi, 0).  out: ndir x (pmax+1) x 4 doubles, per order
 * (F_theta re, im, F_phi re, im).  mask: ndir bytes. */
int or_field_fan(const or_object* o, int64_t nrays, double fan_phi, int pmax,
                 const double* alpha, int64_t ndir, int flags, double* out, uint8_t* mask);

/* 2-D square grid (n_target rays in the projected cross-section, or spacing h_in when
 * h_in > 0) onto the cell-centred (theta, phi) grid.  window = {ix0, ix1, iy0, iy1} limits the
 * cells used (NULL = all).  out: ntheta*nphi x (pmax+1) x 4 doubles.  Returns the number of
 * hits, or a negative value on failure. */
int64_t or_field_grid(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta,
                      int nphi, const int64_t* window, int flags, double* out, uint8_t* mask,
                      int nthreads, int64_t* newton_fail);

/* or_field_grid over every cell, with counts (ndir x (pmax+1) bytes): the number of hits that added
 * to each (direction, order) -- with OR_FIELD_EXACT the number of exact branches found, bit 0x80 set
 * where a hit's Newton refinement did not converge (that hit kept its interpolated value). */
int64_t or_field_grid_counts(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi,
                             int flags, double* out, uint8_t* mask, uint8_t* counts, int nthreads, int64_t* newton_fail);

/* The same field on an arbitrary list of directions: dirs is ndir x (theta, phi) (theta from +z,
 * phi from +x); out: ndir x (pmax+1) x 4, mask: ndir.  Every direction is tested against every
 * cell triangle whose cap contains it. */
int64_t or_field_dirs(const or_object* o, int64_t n_target, double h_in, int pmax, const double* dirs,
                      int64_t ndir, int flags, double* out, uint8_t* mask, int nthreads, int64_t* newton_fail);

/* Record of a traced ray (far, one order's record) at the point where it crosses the sphere
 * |M| = R (R beyond the object): the final leg of length t adds kappa_GM / kappa'_G(p+1) =
 * 1/det(I + t Q') to D_p and its focal lines to N_f, the phase is k0 (path + t), the direction is
 * M / R and the amplitude is the field at M for a unit incident wave.  Returns 1 if valid. */
int or_near_record(const or_object* o, const double* far, double R, double* rec);

/* The field on the sphere |M| = R (R beyond the object's bounding sphere) at the points R u of
 * the cell-centred (theta, phi) grid: the dense-ray interpolation (O2) of the near records.
 * out: ntheta*nphi x (pmax+1) x 6 (E_r re, im, E_theta re, im, E_phi re, im; dimensionless: the
 * ray through M need not be radial), mask as or_field_grid.  Returns the number of hits, or -1 if
 * R does not enclose the object. */
int64_t or_field_sphere(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi, double R,
                        double* out, uint8_t* mask, int nthreads);

/* 2-D physical-optics field of order p over an aperture of rays ("Diffraction effect correction
 * based on VCRM"; Kirchhoff's integral over a plane): the rays of the grid vertices
 * [ix0, ix1] x [iy0, iy1] (window) of the square grid carry their exit waves to the plane through the
 * object centre with normal a = (ap_theta, ap_phi), where each has the field
 * U = E' sqrt(D_legs / |det(I + tau Q')|) (-i)^{N_f} e^{i k0 (L + tau)} and the area dA of the plane
 * per grid cell (central differences of the crossing points); a ray whose exit direction makes the
 * angle g with a has the weight ramp(g): 1 up to cone_full, cos^2 down to 0 at cone_end (the
 * window should hold every ray within cone_end; its own edges are not tapered).
 * F(s) = k0 / (2 pi i) sum w U dA e^{-i k0 s.x}, projected on e_theta, e_phi.  dirs: ndir x
 * (theta, phi); out: ndir x 4.  Returns the number of rays in the sum, or -1 for invalid arguments. */
int64_t or_field_po2d(const or_object* o, int64_t n_target, double h_in, int p, const int64_t* window,
                      double ap_theta, double ap_phi, double cone_full, double cone_end, const double* dirs,
                      int64_t ndir, double* out);

/* Square-grid field with the 2-D physical optics of the caustics (plane wave on an ellipsoid): the
 * ray sum of or_field_grid, and for every order p >= p_min the Kirchhoff integral of the exit waves
 * over a plane blended in around the directions that order's fold cells cover (taper s_p of the
 * angle to them: 1 up to po_full, cos^2 to 0 at po_end); one plane per tile of tile_theta x tile_phi
 * directions, normal to the tile's centre direction a, the rays weighted by the angle of their
 * exit direction to a (1 up to rho + cone_full, 0 from rho + cone_end, rho the tile's radius about a).
 * cp: {tile_theta, tile_phi, po_full, po_end, cone_full, cone_end, p_min}.  out: ndir x (pmax+1) x 4,
 * mask: ndir (caustic bit only where an uncorrected order put it, OR_MASK_PO where s_p > 0).
 * Optional: weights ndir x (pmax+1) (s_p), corders ndir (bit p: covered by an inconsistent cell of
 * order p), l1 ndir x (pmax+1) (s_p k0 / 2 pi |u . a| sum |w U dA|, the size of the summed terms).
 * Returns the hits of the ray sum, -1 for invalid arguments, -2 when a cone reaches 90 deg. */
int64_t or_field_grid_caustic(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi,
                              const double* cp, double* out, uint8_t* mask, double* weights, uint32_t* corders,
                              double* l1, int nthreads);

/* Newton on the exact trace: finds the ray of order p whose exit direction is target, from the
 * seed impact point xy (2), with steps halved until the residual decreases; the root must lie
 * within rmax of the seed (rmax <= 0: no bound).  Returns iterations used, or -1 if it did not
 * converge. */
int or_newton(const or_object* o, int p, const double target[3], double* xy, double rmax, double* rec);
/* The same with at most max_checks evaluations of the residual, convergence at |s - t| < tol and
 * at most max_halvings halvings of a step. */
int or_newton_ex(const or_object* o, int p, const double target[3], double* xy, double rmax, int max_checks,
                 double tol, int max_halvings, double* rec);
/* acc (4) += weight * (F e^{i psi}) . (e_theta, e_phi) as (re, im, re, im) */
void or_project_add(const double F[6], double psi, const double eth[3], const double eph[3], double weight,
                    double* acc);

/* Learned-proposal field on the cell-centred (theta, phi) grid: for every direction s and order
 * p the network of order p (mlp_oracle.h; theta: (pmax+1) x OM_NPARAM doubles, evaluated with
 * bfloat16 rounding as the tensor cores do) proposes 4 entry points (moved onto radius 0.999 of
 * the unit disk when beyond it); each head whose softmax weight is at least p_min seeds
 * or_newton_ex (at most max_steps steps, at most max_halvings halvings of a step, no distance bound,
 * |s - t| < tol, or for tol <= 0 min(1e-6, 1e-4 / (k0 max(a, b, c)))); a root within 1e-6 max(a, b, c) of an earlier root of
 * the same direction and order is the same ray and is dropped; every other root adds
 * F e^{i Psi}, except a near-caustic one, which marks the direction instead.
 * out: ndir x (pmax+1) x 4; mask: ndir (axial as or_field_grid); roots (may be NULL):
 * ndir x (pmax+1) counts, bit 7 set where a head at or above p_min did not converge.  Returns the
 * number of roots. */
int64_t or_field_learned(const or_object* o, const double* theta, int pmax, int ntheta, int nphi, double p_min,
                         int max_steps, double tol, int max_halvings, double* out, uint8_t* mask, uint8_t* roots);
/* The same on a list of directions: dirs is ndir x (theta, phi); out: ndir x (pmax+1) x 4, mask: ndir,
 * roots (may be NULL): ndir x (pmax+1). */
int64_t or_field_learned_dirs(const or_object* o, const double* theta, int pmax, const double* dirs, int64_t ndir,
                              double p_min, int max_steps, double tol, int max_halvings, double* out, uint8_t* mask,
                              uint8_t* roots);

#ifdef __cplusplus
}
#endif
#endif
