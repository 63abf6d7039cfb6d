/*
 * rtw_oracle.c -- plain FP64 CPU oracle of the Ray Theory of Waves far field.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load it.  It shares no code with the CUDA library.
 *
 * Scalar double precision, one ray at a time, compiled with -ffp-contract=off.  OpenMP is
 * used only to run independent rays side by side (and atomics for the accumulation); no
 * step is blocked, fused or reordered.  The steps follow the paper (Ren et al.,
 * arXiv:2403.13856) in its order:
 *   O1  trace of one ray through the object, every interaction by Eq. (SnellVec),
 *       Eq. (Fres), the step-by-step Jones update and Eq. (WavefrontEqVec); every internal leg
 *       by free propagation of Q; amplitude by Eqs. (IntVCRM)/(DivFactVCRM); phase by
 *       Eqs. (PhasePath)/(PhaseTotal).
 *   O2  the RTW strategy ("Strategy of Ray Theory of Waves"): the map t -> (direction, A, Phi)
 *       is interpolated onto the observation directions and all rays are summed (principle iii).
 *   O3  the same hits, each evaluated exactly by Newton on the trace (the definition the
 *       interpolation approximates).
 *   O4  physical-optics "simple integration" over the exit wavefront near an in-plane fold
 *       ("Diffraction effect correction based on VCRM").
 */
#include "rtw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#ifndef OR_OPCOUNT
#include <complex.h>
typedef double complex cplx;
#endif /* else: the counting build (opcount.h) provides cplx */

static const double PI = 3.14159265358979323846;
/* rays whose |cos| of incidence falls below this are dropped (grazing, P' singular) */
static const double GRAZE = 1e-9;

struct or_object {
    double semi[3];
    double R[3][3]; /* body -> world, columns are the body axes */
    double center[3];
    double W[3][3]; /* (x-c)^T W (x-c) = 1 on the surface */
    double m;       /* n_object / n_host */
    double lambda;  /* wavelength in the host medium (um) */
    double k0;
    cplx jones[2];
    double zstart;
    double S[2][2]; /* projected cross-section: (dx,dy) S (dx,dy)^T <= 1 */
    double Sinv[2][2];
    double Lmax, Lmin;
    double gc[2];   /* centre of the ray grid (plane wave: the object's centre x, y) */
    int src;        /* 0: plane wave along +z; 1: point source */
    double src_pos[3], e1[3], e2[3];
    double shape_e; /* superellipsoid exponent e >= 1: sum_i |u_i|^(2e) = 1; e = 1 is the ellipsoid */
    double Rbound;  /* radius about the centre that contains the object */
};

/* ------------------------------------------------------------------------------------- */
/* small linear algebra                                                                  */
/* ------------------------------------------------------------------------------------- */

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double* a) { return sqrt(dot3(a, a)); }

static void matvec3(const double M[3][3], const double* v, double* out)
{
    for (int i = 0; i < 3; ++i) out[i] = M[i][0] * v[0] + M[i][1] * v[1] + M[i][2] * v[2];
}

static double det2(const double A[2][2]) { return A[0][0] * A[1][1] - A[0][1] * A[1][0]; }

static int inv2(const double A[2][2], double B[2][2])
{
    double d = det2(A);
    if (d == 0.0) return 0;
    B[0][0] = A[1][1] / d;
    B[0][1] = -A[0][1] / d;
    B[1][0] = -A[1][0] / d;
    B[1][1] = A[0][0] / d;
    return 1;
}

static void mul2(const double A[2][2], const double B[2][2], double C[2][2])
{
    double t[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) t[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j];
    memcpy(C, t, sizeof(t));
}

static void transpose2(const double A[2][2], double B[2][2])
{
    double t[2][2] = {{A[0][0], A[1][0]}, {A[0][1], A[1][1]}};
    memcpy(B, t, sizeof(t));
}

/* number of negative eigenvalues of a symmetric 2x2 matrix (its symmetric part) */
static int neg_eigs(const double A[2][2])
{
    double off = 0.5 * (A[0][1] + A[1][0]);
    double det = A[0][0] * A[1][1] - off * off;
    double tr = A[0][0] + A[1][1];
    if (det < 0.0) return 1;
    if (det > 0.0 && tr < 0.0) return 2;
    if (det == 0.0 && tr < 0.0) return 1;
    return 0;
}

/* (-i)^n: the phase factor of n focal lines, each e^{-i pi/2} */
static cplx minus_i_pow(int n)
{
    switch (((n % 4) + 4) % 4) {
    case 0: return 1.0;
    case 1: return -I;
    case 2: return -1.0;
    default: return I;
    }
}

static double wrap_angle(double a)
{
    while (a > PI) a -= 2.0 * PI;
    while (a <= -PI) a += 2.0 * PI;
    return a;
}

/* ------------------------------------------------------------------------------------- */
/* object                                                                                */
/* ------------------------------------------------------------------------------------- */

int or_object_size(void) { return (int)sizeof(or_object); }

void or_object_frame(const or_object* o, double* R9, double* semi, double* center, double* S4, double* m)
{
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            if (R9) R9[3 * i + j] = o->R[i][j];
        if (semi) semi[i] = o->semi[i];
        if (center) center[i] = o->center[i];
    }
    if (S4) {
        S4[0] = o->S[0][0];
        S4[1] = o->S[0][1];
        S4[2] = o->S[1][0];
        S4[3] = o->S[1][1];
    }
    if (m) *m = o->m;
}

int or_make_object(const double* p, or_object* o)
{
    memset(o, 0, sizeof(*o));
    for (int i = 0; i < 3; ++i) {
        if (!(p[i] > 0.0)) return -1;
        o->semi[i] = p[i];
    }
    double w = p[3], x = p[4], y = p[5], z = p[6];
    double qn = sqrt(w * w + x * x + y * y + z * z);
    if (!(qn > 0.0)) return -1;
    w /= qn; x /= qn; y /= qn; z /= qn;
    /* rotation matrix of the unit quaternion (w, x, y, z), body -> world */
    o->R[0][0] = 1 - 2 * (y * y + z * z);
    o->R[0][1] = 2 * (x * y - w * z);
    o->R[0][2] = 2 * (x * z + w * y);
    o->R[1][0] = 2 * (x * y + w * z);
    o->R[1][1] = 1 - 2 * (x * x + z * z);
    o->R[1][2] = 2 * (y * z - w * x);
    o->R[2][0] = 2 * (x * z - w * y);
    o->R[2][1] = 2 * (y * z + w * x);
    o->R[2][2] = 1 - 2 * (x * x + y * y);
    for (int i = 0; i < 3; ++i) o->center[i] = p[7 + i];
    o->m = p[10];
    o->lambda = p[11];
    if (!(o->m > 0.0) || o->m == 1.0 || !(o->lambda > 0.0)) return -1;
    o->k0 = 2.0 * PI / o->lambda;
    o->jones[0] = p[12] + I * p[13];
    o->jones[1] = p[14] + I * p[15];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += o->R[i][k] * o->R[j][k] / (o->semi[k] * o->semi[k]);
            o->W[i][j] = s;
        }
    o->shape_e = p[20];
    if (!(o->shape_e >= 1.0) || !isfinite(o->shape_e)) return -1;
    o->Lmax = fmax(o->semi[0], fmax(o->semi[1], o->semi[2]));
    o->Lmin = fmin(o->semi[0], fmin(o->semi[1], o->semi[2]));
    o->zstart = o->center[2] - 2.0 * o->Lmax - 1.0;
    /* a superellipsoid lies inside the ellipsoid of semi-axes a_i 3^((1 - 1/e) / 2): by the power-mean
     * inequality sum u_i^2 / 3 <= (sum |u_i|^(2e) / 3)^(1/e) <= 3^(-1/e) */
    const double grow = sqrt(pow(3.0, 1.0 - 1.0 / o->shape_e));
    o->Rbound = o->Lmax * grow;
    double Wb[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Wb[i][j] = o->W[i][j] / (grow * grow);
    /* silhouette along z (of the bounding ellipsoid for e > 1): the Schur complement of W_zz */
    o->S[0][0] = Wb[0][0] - Wb[0][2] * Wb[0][2] / Wb[2][2];
    o->S[0][1] = Wb[0][1] - Wb[0][2] * Wb[1][2] / Wb[2][2];
    o->S[1][0] = o->S[0][1];
    o->S[1][1] = Wb[1][1] - Wb[1][2] * Wb[1][2] / Wb[2][2];
    o->gc[0] = o->center[0];
    o->gc[1] = o->center[1];
    o->src = p[16] != 0.0;
    if (o->src) {
        /* point source s: rays s + t v through X = c + x e1 + y e2 meet the surface where
         * (v.W g)^2 - (v.W v)(g.W g - 1) > 0 (g = c - s), i.e. v^T K v > 0 with
         * K = W g g^T W - (g^T W g - 1) W; over X this is an ellipse of the plane:
         * (w - w0)^T S (w - w0) < 1 with w = (x, y) */
        double g[3], Wg[3];
        for (int i = 0; i < 3; ++i) {
            o->src_pos[i] = p[17 + i];
            g[i] = o->center[i] - o->src_pos[i];
        }
        /* for a superellipsoid the same construction on its bounding ellipsoid (Wb = W for e = 1) */
        matvec3(Wb, g, Wg);
        double gWg = dot3(g, Wg);
        if (!(gWg > 1.0)) return -1; /* the source must lie outside the object (its bounding ellipsoid) */
        double d = sqrt(dot3(g, g)), a[3] = {g[0] / d, g[1] / d, g[2] / d};
        double ref[3] = {1.0, 0.0, 0.0};
        if (fabs(a[0]) > 0.9) {
            ref[0] = 0.0;
            ref[1] = 1.0;
        }
        double ra = dot3(ref, a);
        for (int i = 0; i < 3; ++i) o->e1[i] = ref[i] - ra * a[i];
        double n1 = sqrt(dot3(o->e1, o->e1));
        for (int i = 0; i < 3; ++i) o->e1[i] /= n1;
        cross3(a, o->e1, o->e2);
        double K[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) K[i][j] = Wg[i] * Wg[j] - (gWg - 1.0) * Wb[i][j];
        const double* E[2] = {o->e1, o->e2};
        double M2[2][2], b2[2], Kg[3], KE[3];
        matvec3(K, g, Kg);
        for (int a2 = 0; a2 < 2; ++a2) {
            b2[a2] = dot3(E[a2], Kg);
            matvec3(K, E[a2], KE);
            for (int b3 = 0; b3 < 2; ++b3) M2[b3][a2] = dot3(E[b3], KE);
        }
        double Mi[2][2];
        if (!inv2(M2, Mi)) return -1;
        double w0[2] = {-(Mi[0][0] * b2[0] + Mi[0][1] * b2[1]), -(Mi[1][0] * b2[0] + Mi[1][1] * b2[1])};
        double f0 = dot3(g, Kg) + b2[0] * w0[0] + b2[1] * w0[1];
        if (!(f0 > 0.0)) return -1;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) o->S[i][j] = -M2[i][j] / f0;
        o->gc[0] = w0[0];
        o->gc[1] = w0[1];
    }
    if (!inv2(o->S, o->Sinv)) return -1;
    return 0;
}

double or_fan_halfwidth(const or_object* o, double fan_phi)
{
    double e0 = cos(fan_phi), e1 = sin(fan_phi);
    double q = e0 * (o->S[0][0] * e0 + o->S[0][1] * e1) + e1 * (o->S[1][0] * e0 + o->S[1][1] * e1);
    return 1.0 / sqrt(q);
}

void or_square_grid(const or_object* o, int64_t n_target, double h_in, double* h, int64_t* nx,
                    int64_t* ny, double* x0, double* y0)
{
    /* spacing so that about n_target grid points fall inside the projected ellipse, whose
     * area is pi / sqrt(det S) */
    double hh = h_in > 0.0 ? h_in : sqrt(PI / (sqrt(det2(o->S)) * (double)n_target));
    double X = sqrt(o->Sinv[0][0]), Y = sqrt(o->Sinv[1][1]);
    int64_t kx = (int64_t)ceil(X / hh), ky = (int64_t)ceil(Y / hh);
    *h = hh;
    *nx = 2 * kx + 2;
    *ny = 2 * ky + 2;
    /* x_i = cx + (i + 1/2 - nx/2) h */
    *x0 = o->gc[0];
    *y0 = o->gc[1];
}

static double grid_coord(double c, int64_t i, int64_t n, double h)
{
    return c + ((double)i + 0.5 - (double)(n / 2)) * h;
}

double or_caustic_cap(const or_object* o)
{
    /* GO is off by O(1) within about one Airy width (lambda/L)^(2/3) of a fold, where dA/dOmega
     * grows like L^2 (L/lambda)^(1/3); rays beyond that cap are treated as caustic */
    return o->Lmax * o->Lmax * cbrt(o->Lmax / o->lambda);
}

/* ------------------------------------------------------------------------------------- */
/* O1: one ray                                                                           */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    double k[3];    /* unit propagation direction */
    double n;       /* refractive index of the medium */
    double u[2][3]; /* wavefront basis, orthonormal, perpendicular to k */
    double Q[2][2]; /* wavefront curvature matrix in (u1, u2) */
    cplx E[2];      /* field components along u1, u2 */
    double T[2][2]; /* transverse offset of this wave per unit incident offset (x, y) */
} wave_t;

typedef struct {
    wave_t refl, trans;
    int trans_ok;
    double cos_in, cos_trans; /* |k.n| of the incident and the transmitted wave */
} split_t;

/* builds one outgoing wave (reflected or transmitted) of an interaction */
static void outgoing(const or_object* o, const double s[2][3], const double nh[3],
                     const double C[2][2], const double kvi[3], double ki,
                     const double PQP[2][2], const double PiinvT[2][2], const wave_t* in,
                     const double kv[3], double kmag, double n_med, const double ep[3],
                     cplx c_perp, cplx c_par, cplx Eperp, cplx Epar, wave_t* out)
{
    (void)o;
    for (int c = 0; c < 3; ++c) out->k[c] = kv[c] / kmag;
    out->n = n_med;
    /* outgoing wavefront basis: (e_perp, e_perp x k') */
    for (int c = 0; c < 3; ++c) out->u[0][c] = ep[c];
    cross3(ep, out->k, out->u[1]);
    /* P' (Eq. Theta-r): P'_ab = s_a . v_b */
    double Pp[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) Pp[a][b] = dot3(s[a], out->u[b]);
    /* right-hand side of the wavefront equation: k_i P_i Q_i P_i^T + C n.(k' - k_i) */
    double dk[3] = {kv[0] - kvi[0], kv[1] - kvi[1], kv[2] - kvi[2]};
    double cn = dot3(nh, dk);
    double M[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) M[a][b] = ki * PQP[a][b] + C[a][b] * cn;
    /* Q' = P'^{-1} M P'^{-T} / k' */
    double Ppinv[2][2], PpinvT[2][2], tmp[2][2];
    inv2(Pp, Ppinv);
    transpose2(Ppinv, PpinvT);
    mul2(Ppinv, M, tmp);
    mul2(tmp, PpinvT, out->Q);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) out->Q[a][b] /= kmag;
    /* transverse offsets: t_c = P_i^{-T} t_i, t' = P'^T t_c */
    double PpT[2][2];
    transpose2(Pp, PpT);
    mul2(PpT, PiinvT, tmp);
    mul2(tmp, in->T, out->T);
    out->E[0] = c_perp * Eperp;
    out->E[1] = c_par * Epar;
}

/* ------------------------------------------------------------------------------------- */
/* the surface: ellipsoid (e = 1) or superellipsoid F(x) = sum_i |u_i|^(2e) = 1,            */
/* u = diag(1/a) R^T (x - c); F is convex for e >= 1, so a line meets the surface twice      */
/* at most and the Introduction's principle (iii) (one curvature matrix per point) holds     */
/* wherever F is twice differentiable, which e >= 1 ensures                                  */
/* ------------------------------------------------------------------------------------- */

/* body coordinates u of point x and the body-frame rate kappa of direction k (u(t) = u + t kappa) */
static void body_line(const or_object* o, const double x[3], const double k[3], double u[3], double kap[3])
{
    for (int i = 0; i < 3; ++i) {
        double su = 0.0, sk = 0.0;
        for (int j = 0; j < 3; ++j) {
            su += o->R[j][i] * (x[j] - o->center[j]);
            sk += o->R[j][i] * k[j];
        }
        u[i] = su / o->semi[i];
        kap[i] = sk / o->semi[i];
    }
}

/* phi(t) = F(x + t k) - 1 and its derivative along the line */
static double line_phi(const or_object* o, const double u[3], const double kap[3], double t, double* dphi)
{
    const double e = o->shape_e;
    double f = -1.0, df = 0.0;
    for (int i = 0; i < 3; ++i) {
        double v = u[i] + t * kap[i], av = fabs(v);
        f += pow(av, 2.0 * e);
        df += 2.0 * e * copysign(pow(av, 2.0 * e - 1.0), v) * kap[i];
    }
    if (dphi) *dphi = df;
    return f;
}

/* g = grad F / 2 and H = (Hessian of F) / 2 at surface point x; for e = 1 these are W (x - c) and W.
 * The surface's second fundamental form for the outward normal g / |g| is s^T H s / |g|. */
static void shape_gH(const or_object* o, const double x[3], double g[3], double H[3][3])
{
    double d[3] = {x[0] - o->center[0], x[1] - o->center[1], x[2] - o->center[2]};
    if (o->shape_e == 1.0) {
        matvec3(o->W, d, g);
        memcpy(H, o->W, sizeof(o->W));
        return;
    }
    const double e = o->shape_e;
    double gb[3], hb[3];
    for (int i = 0; i < 3; ++i) {
        double ui = (o->R[0][i] * d[0] + o->R[1][i] * d[1] + o->R[2][i] * d[2]) / o->semi[i];
        double au = fabs(ui);
        /* d/dx_b of |u_i|^(2e) / 2 = e |u_i|^(2e-1) sgn(u_i) / a_i, second derivative
         * e (2e - 1) |u_i|^(2e-2) / a_i^2, both along body axis i */
        gb[i] = e * copysign(pow(au, 2.0 * e - 1.0), ui) / o->semi[i];
        hb[i] = e * (2.0 * e - 1.0) * pow(au, 2.0 * e - 2.0) / (o->semi[i] * o->semi[i]);
    }
    for (int i = 0; i < 3; ++i) {
        g[i] = o->R[i][0] * gb[0] + o->R[i][1] * gb[1] + o->R[i][2] * gb[2];
        for (int j = 0; j < 3; ++j)
            H[i][j] = o->R[i][0] * o->R[j][0] * hb[0] + o->R[i][1] * o->R[j][1] * hb[1] + o->R[i][2] * o->R[j][2] * hb[2];
    }
}

/* parameter t at which the line u + t kappa leaves the body box |u_i| <= 1 (u inside it) */
static double box_exit(const double u[3], const double kap[3])
{
    double t = INFINITY;
    for (int i = 0; i < 3; ++i)
        if (kap[i] != 0.0) t = fmin(t, (copysign(1.0, kap[i]) - u[i]) / kap[i]);
    return t;
}

/* superellipsoid chord from surface point r along the inward direction k: the positive root of the
 * convex phi with phi(0) = 0.  The box exit lies at or beyond it (phi >= 0 there, F >= 1 on the box
 * faces), and Newton from the right of a root of a convex increasing function decreases
 * monotonically to it. */
static double chord_super(const or_object* o, const double r[3], const double k[3])
{
    double u[3], kap[3];
    body_line(o, r, k, u, kap);
    double t = box_exit(u, kap);
    if (!(t > 0.0) || !isfinite(t)) return 0.0;
    const double t0 = t;
    for (int it = 0; it < 400; ++it) {
        double df, f = line_phi(o, u, kap, t, &df);
        if (!(f > 0.0) || !(df > 0.0)) break;
        double step = f / df;
        t -= step;
        if (step <= 1e-16 * t0) break;
    }
    return t;
}

/* entry of a line into the superellipsoid: the smaller root of phi.  The line crosses the body box on
 * [t_in, t_out]; bisection on the increasing phi' there finds the minimum of phi (no hit unless
 * it is negative); Newton from t_in (phi >= 0, decreasing) increases monotonically to the root. */
static int entry_super(const or_object* o, const double r0[3], const double k[3], double* t_hit)
{
    double u[3], kap[3];
    body_line(o, r0, k, u, kap);
    double tin = -INFINITY, tout = INFINITY;
    for (int i = 0; i < 3; ++i) {
        if (kap[i] == 0.0) {
            if (!(fabs(u[i]) < 1.0)) return 0;
            continue;
        }
        double ta = (-1.0 - u[i]) / kap[i], tb = (1.0 - u[i]) / kap[i];
        tin = fmax(tin, fmin(ta, tb));
        tout = fmin(tout, fmax(ta, tb));
    }
    if (!(tin < tout)) return 0;
    double a = tin, b = tout;
    for (int it = 0; it < 200 && b - a > 1e-16 * (fabs(a) + fabs(b)); ++it) {
        double mid = 0.5 * (a + b), dm;
        line_phi(o, u, kap, mid, &dm);
        if (dm > 0.0) b = mid;
        else a = mid;
    }
    double tm = 0.5 * (a + b);
    if (!(line_phi(o, u, kap, tm, NULL) < 0.0)) return 0;
    double t = tin;
    for (int it = 0; it < 400; ++it) {
        double df, f = line_phi(o, u, kap, t, &df);
        if (!(f > 0.0) || !(df < 0.0)) break;
        double step = -f / df;
        t += step;
        if (step <= 1e-16 * fabs(tm)) break;
    }
    *t_hit = t;
    return 1;
}

/* one reflection / refraction at surface point r, wave `in` arriving from the medium in->n into
 * the medium n_other.  Returns 0 for a grazing ray. */
static int interact(const or_object* o, const double r[3], const wave_t* in, double n_other,
                    split_t* sp)
{
    double g[3], H[3][3];
    shape_gH(o, r, g, H);
    double gn = norm3(g);
    double nh[3] = {g[0] / gn, g[1] / gn, g[2] / gn}; /* outward normal */
    double cos_i = dot3(in->k, nh);
    if (fabs(cos_i) < GRAZE) return 0;
    /* e_perp normal to the incident plane (Fig. 2) */
    double ep[3];
    cross3(in->k, nh, ep);
    double len = norm3(ep);
    if (len < 1e-12) {
        for (int c = 0; c < 3; ++c) ep[c] = in->u[0][c];
    } else {
        for (int c = 0; c < 3; ++c) ep[c] /= len;
    }
    /* surface basis (s1, s2) = (e_perp, n x e_perp) and the curvature matrix C in it:
     * second fundamental form of the surface with respect to the outward normal */
    double s[2][3];
    for (int c = 0; c < 3; ++c) s[0][c] = ep[c];
    cross3(nh, ep, s[1]);
    double C[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double Ws[3];
            matvec3(H, s[b], Ws);
            C[a][b] = dot3(s[a], Ws) / gn;
        }
    /* Eq. (SnellVec): the tangential component of the wave vector is kept */
    double ki = o->k0 * in->n, kt = o->k0 * n_other;
    double kin = ki * cos_i; /* signed normal component of the incident wave vector */
    double kvi[3], ktau[3], kvl[3], kvt[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
        kvi[c] = ki * in->k[c];
        ktau[c] = kvi[c] - kin * nh[c];
        kvl[c] = ktau[c] - kin * nh[c];
    }
    double ktau2 = dot3(ktau, ktau);
    double ktn2 = kt * kt - ktau2;
    cplx ktn;
    if (ktn2 > 0.0) {
        double kr = copysign(sqrt(ktn2), kin);
        ktn = kr;
        for (int c = 0; c < 3; ++c) kvt[c] = ktau[c] + kr * nh[c];
        sp->trans_ok = 1;
    } else {
        /* total internal reflection: evanescent normal component, decaying on the far side */
        ktn = I * copysign(sqrt(-ktn2), kin);
        sp->trans_ok = 0;
    }
    /* Eq. (Fres), with m the index of the far medium relative to the near one */
    double mr = n_other / in->n;
    cplx rperp = (kin - ktn) / (kin + ktn);
    cplx rpar = (mr * mr * kin - ktn) / (mr * mr * kin + ktn);
    cplx tperp = 2.0 * kin / (kin + ktn);
    cplx tpar = 2.0 * mr * kin / (mr * mr * kin + ktn);
    /* incident field projected on (e_perp, e_par_i), e_par_i = e_perp x k_i */
    double epi[3];
    cross3(ep, in->k, epi);
    cplx Eperp = in->E[0] * dot3(in->u[0], ep) + in->E[1] * dot3(in->u[1], ep);
    cplx Epar = in->E[0] * dot3(in->u[0], epi) + in->E[1] * dot3(in->u[1], epi);
    /* incident term of Eq. (WavefrontEqVec): P_i Q_i P_i^T with P_i,ab = s_a . u_b */
    double Pi[2][2], PiT[2][2], tmp[2][2], PQP[2][2], Piinv[2][2], PiinvT[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) Pi[a][b] = dot3(s[a], in->u[b]);
    transpose2(Pi, PiT);
    mul2(Pi, in->Q, tmp);
    mul2(tmp, PiT, PQP);
    inv2(Pi, Piinv);
    transpose2(Piinv, PiinvT);
    outgoing(o, s, nh, C, kvi, ki, PQP, PiinvT, in, kvl, ki, in->n, ep, rperp, rpar, Eperp, Epar,
             &sp->refl);
    if (sp->trans_ok)
        outgoing(o, s, nh, C, kvi, ki, PQP, PiinvT, in, kvt, kt, n_other, ep, tperp, tpar, Eperp,
                 Epar, &sp->trans);
    sp->cos_in = fabs(cos_i);
    sp->cos_trans = sp->trans_ok ? fabs(dot3(sp->trans.k, nh)) : 0.0;
    return 1;
}

/* length of the chord from surface point r along the inward direction k */
static double chord(const or_object* o, const double r[3], const double k[3])
{
    if (o->shape_e != 1.0) return chord_super(o, r, k);
    double u[3] = {r[0] - o->center[0], r[1] - o->center[1], r[2] - o->center[2]};
    double Wk[3], Wu[3];
    matvec3(o->W, k, Wk);
    matvec3(o->W, u, Wu);
    double A = dot3(k, Wk), B = dot3(k, Wu), Cq = dot3(u, Wu) - 1.0;
    double disc = B * B - A * Cq;
    if (disc < 0.0) disc = 0.0;
    return (-B + sqrt(disc)) / A;
}

/* free propagation of the wavefront over distance d: Q(d) = Q (I + d Q)^{-1}; the leg's
 * Gaussian-curvature ratio kappa_G(q+1)/kappa'_Gq = 1/det(I + d Q) enters D_p (Eq. DivFactVCRM)
 * and every negative eigenvalue of I + d Q is a focal line crossed */
static int propagate(wave_t* w, double d, double* dlegs, int* nf)
{
    double A[2][2] = {{1.0 + d * w->Q[0][0], d * w->Q[0][1]}, {d * w->Q[1][0], 1.0 + d * w->Q[1][1]}};
    double detA = det2(A), Ainv[2][2];
    if (detA == 0.0 || !inv2(A, Ainv)) return 0;
    mul2(w->Q, Ainv, w->Q);
    *dlegs /= fabs(detA);
    *nf += neg_eigs(A);
    mul2(A, w->T, w->T);
    return 1;
}

/* far-field record of an outgoing wave leaving the object at rexit */
static void far_field(const or_object* o, const wave_t* w, const double rexit[3], double path,
                      double dlegs, int nf_legs, double cosprod, int nrefl, double* rec)
{
    double detQ = det2(w->Q);
    if (!isfinite(detQ)) return;
    /* an exit wave flat in a principal direction (det Q' = 0, where a stretch of surface has no
     * curvature) sends its energy into a single direction: a caustic at infinity, kept as a valid
     * ray with the caustic flag and no amplitude (its cells mask the directions they cover) */
    const int flat = !(fabs(detQ) > 0.0);
    /* last leg to infinity: kappa_GM / kappa'_G(p+1) -> 1/(r^2 det Q'); r^2 is removed */
    int nf = nf_legs + neg_eigs(w->Q);
    double D = flat ? INFINITY : dlegs / fabs(detQ);
    cplx ph = flat ? 0.0 : minus_i_pow(nf) * sqrt(D);
    for (int c = 0; c < 3; ++c) {
        cplx Fc = ph * (w->E[0] * w->u[0][c] + w->E[1] * w->u[1][c]);
        rec[OR_F + 2 * c] = creal(Fc);
        rec[OR_F + 2 * c + 1] = cimag(Fc);
    }
    /* Eq. (PhasePath) read for the far field: optical path to the exit point minus s.r_exit */
    rec[OR_PSI] = o->k0 * (path - dot3(w->k, rexit));
    double J[2][2];
    mul2(w->Q, w->T, J);
    double detJ = det2(J);
    double vx[3];
    cross3(w->u[0], w->u[1], vx);
    double hand = dot3(w->k, vx) > 0.0 ? 1.0 : -1.0;
    rec[OR_VALID] = 1.0;
    rec[OR_NF] = (double)nf;
    rec[OR_ORIENT] = (detJ > 0.0 ? 1.0 : -1.0) * hand;
    rec[OR_NREFL] = (double)nrefl;
    for (int c = 0; c < 3; ++c) {
        rec[OR_S + c] = w->k[c];
        rec[OR_V1 + c] = w->u[0][c];
        rec[OR_V2 + c] = w->u[1][c];
        rec[OR_REXIT + c] = rexit[c];
    }
    rec[OR_D] = D;
    rec[OR_DGEO] = 1.0 / fabs(detJ);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            rec[OR_J + 2 * a + b] = J[a][b];
            rec[OR_Q + 2 * a + b] = w->Q[a][b];
        }
    rec[OR_E + 0] = creal(w->E[0]);
    rec[OR_E + 1] = cimag(w->E[0]);
    rec[OR_E + 2] = creal(w->E[1]);
    rec[OR_E + 3] = cimag(w->E[1]);
    rec[OR_DLEGS] = dlegs;
    rec[OR_NFLEGS] = (double)nf_legs;
    rec[OR_PATH] = path;
    double e2 = creal(w->E[0] * conj(w->E[0]) + w->E[1] * conj(w->E[1]));
    rec[OR_POWER] = e2 * cosprod;
    rec[OR_COSPROD] = cosprod;
    rec[OR_CAUSTIC] = (flat || rec[OR_DGEO] > or_caustic_cap(o)) ? 1.0 : 0.0;
}

/* Record of the same ray at the point M where it crosses the sphere |M| = R (Eqs. IntVCRM,
 * DivFactVCRM and PhasePath at a finite point): the last leg of length t from the exit point ends
 * the product of Gaussian-curvature ratios with kappa_GM / kappa'_G(p+1) = 1 / det(I + t Q'), its
 * negative eigenvalues are focal lines crossed, and the optical path runs to M.  The record's
 * direction is the unit vector of M, its amplitude the field at M for a unit incident wave
 * (dimensionless), its phase k0 (path + t).  The orientation is that of (x, y) -> M on the sphere
 * (the far-field one times sign det(I + t Q') sign det Q'), the caustic measure
 * t^2 / |det(I + t Q') det T|, the far-field dA/dOmega in the limit t -> infinity. */
int or_near_record(const or_object* o, const double* far, double R, double* rec)
{
    memcpy(rec, far, sizeof(double) * OR_NFIELD);
    if (far[OR_VALID] == 0.0) return 0;
    const double* r = far + OR_REXIT;
    const double* sv = far + OR_S;
    double sr = dot3(sv, r), rr = dot3(r, r), disc = sr * sr - rr + R * R;
    if (!(R * R > rr) || disc < 0.0) {
        rec[OR_VALID] = 0.0;
        return 0;
    }
    double t = -sr + sqrt(disc);
    double Q[2][2] = {{far[OR_Q + 0], far[OR_Q + 1]}, {far[OR_Q + 2], far[OR_Q + 3]}};
    double A[2][2] = {{1.0 + t * Q[0][0], t * Q[0][1]}, {t * Q[1][0], 1.0 + t * Q[1][1]}};
    double detA = det2(A), detQ = det2(Q);
    double J[2][2] = {{far[OR_J + 0], far[OR_J + 1]}, {far[OR_J + 2], far[OR_J + 3]}};
    double detJ = det2(J);
    if (!(fabs(detA) > 0.0) || !(fabs(detQ) > 0.0) || !(fabs(detJ) > 0.0)) {
        rec[OR_VALID] = 0.0;
        return 0;
    }
    int nf = (int)far[OR_NFLEGS] + neg_eigs(A);
    double D = far[OR_DLEGS] / fabs(detA);
    cplx E0 = far[OR_E + 0] + I * far[OR_E + 1], E1 = far[OR_E + 2] + I * far[OR_E + 3];
    cplx ph = minus_i_pow(nf) * sqrt(D);
    for (int c = 0; c < 3; ++c) {
        cplx Fc = ph * (E0 * far[OR_V1 + c] + E1 * far[OR_V2 + c]);
        rec[OR_F + 2 * c] = creal(Fc);
        rec[OR_F + 2 * c + 1] = cimag(Fc);
        rec[OR_S + c] = (r[c] + t * sv[c]) / R;
    }
    rec[OR_PSI] = o->k0 * (far[OR_PATH] + t);
    rec[OR_NF] = (double)nf;
    rec[OR_ORIENT] = far[OR_ORIENT] * (detA > 0.0 ? 1.0 : -1.0) * (detQ > 0.0 ? 1.0 : -1.0);
    rec[OR_D] = D;
    rec[OR_DGEO] = t * t * fabs(detQ) / (fabs(detA) * fabs(detJ));
    rec[OR_CAUSTIC] = rec[OR_DGEO] > or_caustic_cap(o) ? 1.0 : 0.0;
    return 1;
}

int or_trace_ray(const or_object* o, double x, double y, int pmax, double* out, double* p_inside)
{
    memset(out, 0, sizeof(double) * (size_t)(pmax + 1) * OR_NFIELD);
    if (p_inside) *p_inside = 0.0;
    wave_t w;
    memset(&w, 0, sizeof(w));
    double r[3], path;
    if (!o->src) {
        /* incident ray of the plane wave, started below the object */
        double r0[3] = {x, y, o->zstart};
        double t;
        if (o->shape_e != 1.0) {
            const double kz[3] = {0.0, 0.0, 1.0};
            if (!entry_super(o, r0, kz, &t)) return 0;
        } else {
            double u[3] = {r0[0] - o->center[0], r0[1] - o->center[1], r0[2] - o->center[2]};
            double Wu[3];
            matvec3(o->W, u, Wu);
            double A = o->W[2][2], B = Wu[2], Cq = dot3(u, Wu) - 1.0;
            double disc = B * B - A * Cq;
            if (!(disc > 0.0)) return 0;
            t = (-B - sqrt(disc)) / A;
        }
        r[0] = r0[0];
        r[1] = r0[1];
        r[2] = r0[2] + t;
        w.k[2] = 1.0;
        w.n = 1.0;
        w.u[0][0] = 1.0;
        w.u[1][1] = 1.0;
        w.E[0] = o->jones[0];
        w.E[1] = o->jones[1];
        w.T[0][0] = 1.0;
        w.T[1][1] = 1.0;
        /* phase of the incident plane wave at the first point, zero at the origin (Phi_i) */
        path = r[2];
    } else {
        /* point source: the ray toward X = c + x e1 + y e2 reaches the surface at distance rho
         * with the spherical wave's curvature I / rho (diverging), amplitude 1 / rho (A_0 of
         * Eq. IntVCRM) and phase k rho (Phi_i of Eq. PhaseTotal) */
        double v[3], g[3];
        for (int i = 0; i < 3; ++i) {
            v[i] = o->center[i] + x * o->e1[i] + y * o->e2[i] - o->src_pos[i];
            g[i] = o->src_pos[i] - o->center[i];
        }
        double dP = sqrt(dot3(v, v));
        for (int i = 0; i < 3; ++i) w.k[i] = v[i] / dP;
        double rho;
        if (o->shape_e != 1.0) {
            /* superellipsoid: the smaller root of the line function from the source */
            if (!entry_super(o, o->src_pos, w.k, &rho)) return 0;
            for (int i = 0; i < 3; ++i) r[i] = o->src_pos[i] + rho * w.k[i];
        } else {
            /* the quadratic is solved from the ray's point of closest approach to the centre, so that
             * a distant source does not cancel the discriminant: rho = t0 + u */
            double t0 = -dot3(w.k, g), f[3], Wk[3], Wf[3];
            for (int i = 0; i < 3; ++i) f[i] = g[i] + t0 * w.k[i]; /* foot point minus centre */
            matvec3(o->W, w.k, Wk);
            matvec3(o->W, f, Wf);
            double A = dot3(w.k, Wk), B = dot3(w.k, Wf), Cq = dot3(f, Wf) - 1.0;
            double disc = B * B - A * Cq;
            if (!(disc > 0.0)) return 0;
            rho = t0 + (-B - sqrt(disc)) / A;
            if (!(rho > 0.0)) return 0;
            for (int i = 0; i < 3; ++i) r[i] = o->center[i] + f[i] + (rho - t0) * w.k[i];
        }
        w.n = 1.0;
        /* basis u1 = e1 made perpendicular to k, u2 = k x u1 */
        double ek = dot3(o->e1, w.k);
        for (int i = 0; i < 3; ++i) w.u[0][i] = o->e1[i] - ek * w.k[i];
        double nu = sqrt(dot3(w.u[0], w.u[0]));
        for (int i = 0; i < 3; ++i) w.u[0][i] /= nu;
        cross3(w.k, w.u[0], w.u[1]);
        w.Q[0][0] = w.Q[1][1] = 1.0 / rho;
        cplx pv[3], pk = 0.0;
        for (int i = 0; i < 3; ++i) {
            pv[i] = o->jones[0] * o->e1[i] + o->jones[1] * o->e2[i];
            pk += pv[i] * w.k[i];
        }
        for (int i = 0; i < 3; ++i) pv[i] -= pk * w.k[i];
        for (int a = 0; a < 2; ++a) {
            cplx e = 0.0;
            for (int i = 0; i < 3; ++i) e += pv[i] * w.u[a][i];
            w.E[a] = e / rho;
        }
        /* transverse offset at the surface per unit (x, y): (rho / |X - s|) times the plane's
         * axes projected on the basis */
        const double* ax[2] = {o->e1, o->e2};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) w.T[a][b] = rho / dP * dot3(w.u[a], ax[b]);
        path = rho;
    }
    double dlegs = 1.0, cosprod = 1.0;
    int nf = 0, nrefl = 0;
    for (int q = 1; q <= pmax + 1; ++q) {
        double n_other = (q == 1) ? o->m : 1.0;
        split_t sp;
        if (!interact(o, r, &w, n_other, &sp)) return 1;
        if (q == 1) {
            /* p = 0: external reflection, Eq. (epsilon_VCRM) first line */
            far_field(o, &sp.refl, r, path, 1.0, 0, 1.0, 1, out);
            if (!sp.trans_ok) return 1;
            w = sp.trans;
            cosprod *= sp.cos_trans / sp.cos_in;
        } else {
            /* p = q - 1 leaves by refraction; the reflected wave continues inside */
            if (sp.trans_ok)
                far_field(o, &sp.trans, r, path, dlegs, nf, cosprod * sp.cos_trans / sp.cos_in,
                          nrefl, out + (size_t)(q - 1) * OR_NFIELD);
            w = sp.refl;
            nrefl++;
        }
        if (q == pmax + 1) break;
        double d = chord(o, r, w.k);
        if (!(d > 0.0)) return 1;
        if (!propagate(&w, d, &dlegs, &nf)) return 1;
        path += w.n * d;
        for (int c = 0; c < 3; ++c) r[c] += d * w.k[c];
    }
    if (p_inside) {
        double e2 = creal(w.E[0] * conj(w.E[0]) + w.E[1] * conj(w.E[1]));
        *p_inside = e2 * w.n * cosprod;
    }
    return 1;
}

void or_trace_rays(const or_object* o, const double* xy, int64_t n, int pmax, double* out,
                   int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t i = 0; i < n; ++i)
        or_trace_ray(o, xy[2 * i], xy[2 * i + 1], pmax, out + (size_t)i * (pmax + 1) * OR_NFIELD, NULL);
    (void)nthreads;
}

/* ------------------------------------------------------------------------------------- */
/* O3: Newton on the exact trace                                                          */
/* ------------------------------------------------------------------------------------- */

/* Residual |target - s_p(x, y)| of the exact trace at xy; the record of order p goes to buf.
 * Returns 0 when order p does not leave the object from this impact point. */
static int newton_eval(const or_object* o, int p, const double target[3], const double* xy, double* buf,
                       double* res)
{
    or_trace_ray(o, xy[0], xy[1], p, buf, NULL);
    const double* r = buf + (size_t)p * OR_NFIELD;
    if (r[OR_VALID] == 0.0) return 0;
    double d[3] = {target[0] - r[OR_S], target[1] - r[OR_S + 1], target[2] - r[OR_S + 2]};
    *res = norm3(d);
    return 1;
}

/* Newton steps xy <- xy + J^{-1} [v1.d, v2.d] with d = target - s and J = ds/d(x, y) of the
 * record, each step shortened by halving (at most max_halvings times; or_newton: 12) until the trace of the new point
 * leaves in order p with a smaller residual.  Converged when |d| < tol at one of the first
 * max_checks evaluations (or_newton: 1e-11 within 30) and the root lies within rmax of the seed
 * (rmax <= 0: anywhere), so that the ray found is the one the seed stands for and not a
 * neighbouring branch of the same order.  xy ends at the last point reached. */
int or_newton(const or_object* o, int p, const double target[3], double* xy, double rmax, double* rec)
{
    return or_newton_ex(o, p, target, xy, rmax, 30, 1e-11, 12, rec);
}

int or_newton_ex(const or_object* o, int p, const double target[3], double* xy, double rmax, int max_checks,
                 double tol, int max_halvings, double* rec)
{
    const size_t nb = (size_t)(p + 1) * OR_NFIELD;
    double* buf = (double*)malloc(sizeof(double) * 2 * nb);
    double* cur = buf;
    double* trial = buf + nb;
    const double x0 = xy[0], y0 = xy[1];
    int ret = -1;
    double res;
    if (newton_eval(o, p, target, xy, cur, &res)) {
        for (int it = 0; it < max_checks; ++it) {
            const double* r = cur + (size_t)p * OR_NFIELD;
            if (res < tol) {
                if (rmax <= 0.0 || hypot(xy[0] - x0, xy[1] - y0) <= rmax) {
                    memcpy(rec, r, sizeof(double) * OR_NFIELD);
                    ret = it;
                }
                break;
            }
            if (it == max_checks - 1) break;
            double d[3] = {target[0] - r[OR_S], target[1] - r[OR_S + 1], target[2] - r[OR_S + 2]};
            double rhs0 = dot3(r + OR_V1, d), rhs1 = dot3(r + OR_V2, d);
            double J[2][2] = {{r[OR_J], r[OR_J + 1]}, {r[OR_J + 2], r[OR_J + 3]}}, Ji[2][2];
            if (!inv2(J, Ji)) break;
            const double dx = Ji[0][0] * rhs0 + Ji[0][1] * rhs1, dy = Ji[1][0] * rhs0 + Ji[1][1] * rhs1;
            double lam = 1.0;
            int accepted = 0;
            for (int h = 0; h <= max_halvings; ++h, lam *= 0.5) {
                double cand[2] = {xy[0] + lam * dx, xy[1] + lam * dy}, rc;
                if (newton_eval(o, p, target, cand, trial, &rc) && rc < res) {
                    xy[0] = cand[0];
                    xy[1] = cand[1];
                    res = rc;
                    double* t = cur;
                    cur = trial;
                    trial = t;
                    accepted = 1;
                    break;
                }
            }
            if (!accepted) break;
        }
    }
    free(buf);
    return ret;
}

/* Newton in the impact parameter b of a fan: in-plane exit angle alpha(b) = alpha_t */
static int newton_fan(const or_object* o, int p, double fan_phi, double alpha_t, double* b,
                      double* rec)
{
    double ef[3] = {cos(fan_phi), sin(fan_phi), 0.0};
    double* buf = (double*)malloc(sizeof(double) * (size_t)(p + 1) * OR_NFIELD);
    int ret = -1;
    for (int it = 0; it < 40; ++it) {
        or_trace_ray(o, o->center[0] + *b * ef[0], o->center[1] + *b * ef[1], p, buf, NULL);
        const double* r = buf + (size_t)p * OR_NFIELD;
        if (r[OR_VALID] == 0.0) break;
        double al = atan2(dot3(r + OR_S, ef), r[OR_S + 2]);
        double da = wrap_angle(alpha_t - al);
        if (fabs(da) < 1e-13) {
            memcpy(rec, r, sizeof(double) * OR_NFIELD);
            ret = it;
            break;
        }
        /* d s / d b = J (ef_x, ef_y) in the exit basis; d alpha = (d s) . e_alpha */
        double j0 = r[OR_J] * ef[0] + r[OR_J + 1] * ef[1];
        double j1 = r[OR_J + 2] * ef[0] + r[OR_J + 3] * ef[1];
        double ds[3];
        for (int c = 0; c < 3; ++c) ds[c] = j0 * r[OR_V1 + c] + j1 * r[OR_V2 + c];
        double ea[3] = {cos(al) * ef[0], cos(al) * ef[1], -sin(al)};
        double dadb = dot3(ds, ea);
        if (dadb == 0.0) break;
        *b += da / dadb;
    }
    free(buf);
    return ret;
}

/* ------------------------------------------------------------------------------------- */
/* O2 / O3 / O4 on a 1-D fan                                                              */
/* ------------------------------------------------------------------------------------- */

/* contribution F e^{i Psi} of one record projected on (e_theta, e_phi) */
void or_project_add(const double F[6], double psi, const double eth[3], const double eph[3], double weight,
                    double* acc)
{
    cplx ph = cexp(I * psi);
    cplx ft = 0.0, fp = 0.0;
    for (int c = 0; c < 3; ++c) {
        cplx Fc = (F[2 * c] + I * F[2 * c + 1]) * ph;
        ft += Fc * eth[c];
        fp += Fc * eph[c];
    }
    acc[0] += weight * creal(ft);
    acc[1] += weight * cimag(ft);
    acc[2] += weight * creal(fp);
    acc[3] += weight * cimag(fp);
}

/* as or_project_add, onto (e_r, e_theta, e_phi): the field at a finite point M has a radial part
 * because the ray through M need not be radial (acc: 6 doubles) */
static void project_add3(const double F[6], double psi, const double* er, const double* eth, const double* eph,
                         double* acc)
{
    cplx ph = cexp(I * psi);
    cplx fr = 0.0, ft = 0.0, fp = 0.0;
    for (int c = 0; c < 3; ++c) {
        cplx Fc = (F[2 * c] + I * F[2 * c + 1]) * ph;
        fr += Fc * er[c];
        ft += Fc * eth[c];
        fp += Fc * eph[c];
    }
    acc[0] += creal(fr);
    acc[1] += cimag(fr);
    acc[2] += creal(ft);
    acc[3] += cimag(ft);
    acc[4] += creal(fp);
    acc[5] += cimag(fp);
}

/* 1 for |x| <= x0, cos^2 ramp to 0 at x1 */
static double ramp(double x, double x0, double x1)
{
    if (x <= x0) return 1.0;
    if (x >= x1) return 0.0;
    double c = cos(0.5 * PI * (x - x0) / (x1 - x0));
    return c * c;
}

typedef struct {
    int p;
    int64_t jc, jlo, jhi; /* fold ray and window rays [jlo, jhi] */
    double alpha_c;
    int ok;
    double* xap;   /* aperture crossing points, 3 per ray */
    cplx* U;       /* aperture field, 3 per ray, times taper, dxi and the sagittal factor */
} po_window;

int or_field_fan(const or_object* o, int64_t nrays, double fan_phi, int pmax, const double* alpha,
                 int64_t ndir, int flags, double* out, uint8_t* mask)
{
    const int np = pmax + 1;
    if (o->src || o->shape_e != 1.0) return -1; /* fans: plane wave on an ellipsoid only */
    double wdt = or_fan_halfwidth(o, fan_phi);
    double ef[3] = {cos(fan_phi), sin(fan_phi), 0.0};
    double* rec = (double*)malloc(sizeof(double) * (size_t)nrays * np * OR_NFIELD);
    double* al = (double*)malloc(sizeof(double) * (size_t)nrays * np);
    double* bj = (double*)malloc(sizeof(double) * (size_t)nrays);
    if (!rec || !al || !bj) return -1;
    for (int64_t j = 0; j < nrays; ++j) {
        double b = -wdt + ((double)j + 0.5) * (2.0 * wdt / (double)nrays);
        bj[j] = b;
        or_trace_ray(o, o->center[0] + b * ef[0], o->center[1] + b * ef[1], pmax,
                     rec + (size_t)j * np * OR_NFIELD, NULL);
        for (int p = 0; p < np; ++p) {
            const double* r = rec + ((size_t)j * np + p) * OR_NFIELD;
            al[j * np + p] = atan2(dot3(r + OR_S, ef), r[OR_S + 2]);
        }
    }
    memset(out, 0, sizeof(double) * (size_t)ndir * np * 4);
    memset(mask, 0, (size_t)ndir);
    /* target directions and their (e_theta, e_phi) */
    double* eth = (double*)malloc(sizeof(double) * 3 * (size_t)ndir);
    double* eph = (double*)malloc(sizeof(double) * 3 * (size_t)ndir);
    double* dirv = (double*)malloc(sizeof(double) * 3 * (size_t)ndir);
    double axial = 2.0 * o->lambda / o->Lmin;
    for (int64_t k = 0; k < ndir; ++k) {
        double a = alpha[k];
        double th = fabs(a), ph = a >= 0.0 ? fan_phi : fan_phi + PI;
        eth[3 * k] = cos(th) * cos(ph);
        eth[3 * k + 1] = cos(th) * sin(ph);
        eth[3 * k + 2] = -sin(th);
        eph[3 * k] = -sin(ph);
        eph[3 * k + 1] = cos(ph);
        eph[3 * k + 2] = 0.0;
        dirv[3 * k] = sin(th) * cos(ph);
        dirv[3 * k + 1] = sin(th) * sin(ph);
        dirv[3 * k + 2] = cos(th);
        if (th < axial || th > PI - axial) mask[k] |= OR_MASK_AXIAL;
    }
    /* angular scales of a fold of an object of size L: the Airy width (lambda/L)^(2/3) and the
     * Fresnel width 1/sqrt(k0 L) of the aperture plane through the object centre.  The PO value
     * is used alone within 1.5 Airy widths of the fold direction and blended into the ray sum by
     * 3; the aperture keeps every ray of the fold within 3 Airy + 3 Fresnel widths and tapers
     * the next 3 Fresnel widths to zero. */
    const double Aw = pow(o->lambda / o->Lmax, 2.0 / 3.0), Fw = 1.0 / sqrt(o->k0 * o->Lmax);
    const double po_full = 1.5 * Aw, po_end = 3.0 * Aw;
    const double ap_full = 3.0 * Aw + 3.0 * Fw, ap_end = 3.0 * Aw + 6.0 * Fw;

    for (int p = 0; p < np; ++p) {
        /* ---- O4: in-plane folds of this order and their aperture fields ---- */
        int nwin = 0;
        po_window win[8];
        if ((flags & OR_FIELD_PO) && p >= 1) {
            for (int64_t j = 1; j + 1 < nrays && nwin < 8; ++j) {
                const double* r0 = rec + ((size_t)(j - 1) * np + p) * OR_NFIELD;
                const double* r1 = rec + ((size_t)j * np + p) * OR_NFIELD;
                const double* r2 = rec + ((size_t)(j + 1) * np + p) * OR_NFIELD;
                if (r0[OR_VALID] == 0.0 || r1[OR_VALID] == 0.0 || r2[OR_VALID] == 0.0) continue;
                double d0 = wrap_angle(al[j * np + p] - al[(j - 1) * np + p]);
                double d1 = wrap_angle(al[(j + 1) * np + p] - al[j * np + p]);
                if (!(d0 * d1 < 0.0)) continue;
                po_window* wv = &win[nwin];
                wv->p = p;
                wv->jc = j;
                wv->alpha_c = al[j * np + p];
                /* the window walks along the fan while the rays stay valid, within ap_end of the
                 * fold direction, on the same side of the +-pi seam and without another fold */
                int64_t lo = j, hi = j;
                while (lo - 1 >= 0 && rec[((size_t)(lo - 1) * np + p) * OR_NFIELD + OR_VALID] != 0.0 &&
                       fabs(wrap_angle(al[(lo - 1) * np + p] - wv->alpha_c)) < ap_end &&
                       fabs(al[(lo - 1) * np + p] - al[lo * np + p]) < PI &&
                       (al[(lo - 1) * np + p] - al[lo * np + p]) * d0 < 0.0)
                    --lo;
                while (hi + 1 < nrays && rec[((size_t)(hi + 1) * np + p) * OR_NFIELD + OR_VALID] != 0.0 &&
                       fabs(wrap_angle(al[(hi + 1) * np + p] - wv->alpha_c)) < ap_end &&
                       fabs(al[(hi + 1) * np + p] - al[hi * np + p]) < PI &&
                       (al[(hi + 1) * np + p] - al[hi * np + p]) * d1 > 0.0)
                    ++hi;
                wv->jlo = lo;
                wv->jhi = hi;
                int64_t nw = hi - lo + 1;
                wv->xap = (double*)malloc(sizeof(double) * 3 * (size_t)nw);
                wv->U = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)nw);
                double* xi = (double*)malloc(sizeof(double) * (size_t)nw);
                /* aperture: the line of the fan plane through the object centre, perpendicular to
                 * the fold ray (the plane of the virtual exit wavefront) */
                const double* rc = o->center;
                const double* sc = r1 + OR_S;
                double exi[3] = {cos(wv->alpha_c) * ef[0], cos(wv->alpha_c) * ef[1], -sin(wv->alpha_c)};
                double npl[3];
                double zz[3] = {0, 0, 1};
                cross3(ef, zz, npl); /* normal of the plane of the fan (sagittal direction) */
                wv->ok = nw >= 3;
                for (int64_t i = lo; i <= hi && wv->ok; ++i) {
                    const double* ri = rec + ((size_t)i * np + p) * OR_NFIELD;
                    double dd[3] = {rc[0] - ri[OR_REXIT], rc[1] - ri[OR_REXIT + 1], rc[2] - ri[OR_REXIT + 2]};
                    double tau = dot3(sc, dd) / dot3(sc, ri + OR_S);
                    double* xa = wv->xap + 3 * (i - lo);
                    for (int c = 0; c < 3; ++c) xa[c] = ri[OR_REXIT + c] + tau * ri[OR_S + c];
                    double rel[3] = {xa[0] - rc[0], xa[1] - rc[1], xa[2] - rc[2]};
                    xi[i - lo] = dot3(exi, rel);
                    /* carry the exit wave along its ray to the aperture line (forward for
                     * tau > 0, backward for tau < 0); each focal line passed on the way adds
                     * e^{-i pi/2} going forward and e^{+i pi/2} going backward */
                    double Q[2][2] = {{ri[OR_Q], ri[OR_Q + 1]}, {ri[OR_Q + 2], ri[OR_Q + 3]}};
                    double Am[2][2] = {{1.0 + tau * Q[0][0], tau * Q[0][1]}, {tau * Q[1][0], 1.0 + tau * Q[1][1]}};
                    double dA = det2(Am), Ai[2][2], Qa[2][2];
                    if (dA == 0.0 || !inv2(Am, Ai)) {
                        wv->ok = 0;
                        break;
                    }
                    int nfl = neg_eigs(Am);
                    int nf_ap = (int)ri[OR_NFLEGS] + (tau > 0.0 ? nfl : -nfl);
                    mul2(Q, Ai, Qa);
                    double c1 = dot3(npl, ri + OR_V1), c2 = dot3(npl, ri + OR_V2);
                    double Qs = c1 * (Qa[0][0] * c1 + Qa[0][1] * c2) + c2 * (Qa[1][0] * c1 + Qa[1][1] * c2);
                    if (Qs == 0.0) {
                        wv->ok = 0;
                        break;
                    }
                    double Rs = 1.0 / Qs;
                    double Dap = ri[OR_DLEGS] / fabs(dA);
                    cplx E0 = ri[OR_E] + I * ri[OR_E + 1], E1 = ri[OR_E + 2] + I * ri[OR_E + 3];
                    cplx amp = sqrt(Dap) * minus_i_pow(nf_ap) *
                               cexp(I * o->k0 * (ri[OR_PATH] + tau));
                    /* sagittal Fresnel integral: sqrt(|R_s|) e^{i pi/4 sgn R_s} */
                    cplx sag = sqrt(fabs(Rs)) * cexp(I * 0.25 * PI * (Rs > 0.0 ? 1.0 : -1.0));
                    double tap = ramp(fabs(wrap_angle(al[i * np + p] - wv->alpha_c)), ap_full, ap_end);
                    for (int c = 0; c < 3; ++c)
                        wv->U[3 * (i - lo) + c] = tap * sag * amp * (E0 * ri[OR_V1 + c] + E1 * ri[OR_V2 + c]);
                }
                /* trapezoid weights |d xi| along the ray parameter: where rays cross before the
                 * line, each branch through a point of the aperture is counted */
                if (wv->ok) {
                    for (int64_t i = 0; i < nw; ++i) {
                        double dxi;
                        if (i == 0) dxi = 0.5 * (xi[1] - xi[0]);
                        else if (i == nw - 1) dxi = 0.5 * (xi[nw - 1] - xi[nw - 2]);
                        else dxi = 0.5 * (xi[i + 1] - xi[i - 1]);
                        for (int c = 0; c < 3; ++c) wv->U[3 * i + c] *= fabs(dxi);
                    }
                }
                free(xi);
                ++nwin;
            }
        }

        /* in-plane folds of this order (sign changes of d alpha / d b), for the exact-near-folds
         * mode: hits within 2 deg of a fold direction are evaluated by Newton */
        double folds[64];
        int nfold = 0;
        if (flags & OR_FIELD_EXACT_FOLDS) {
            for (int64_t j = 1; j + 1 < nrays && nfold < 64; ++j) {
                if (rec[((size_t)(j - 1) * np + p) * OR_NFIELD + OR_VALID] == 0.0 ||
                    rec[((size_t)j * np + p) * OR_NFIELD + OR_VALID] == 0.0 ||
                    rec[((size_t)(j + 1) * np + p) * OR_NFIELD + OR_VALID] == 0.0)
                    continue;
                double d0 = wrap_angle(al[j * np + p] - al[(j - 1) * np + p]);
                double d1 = wrap_angle(al[(j + 1) * np + p] - al[j * np + p]);
                if (d0 * d1 < 0.0) folds[nfold++] = al[j * np + p];
            }
        }
        const double fold_window = 2.0 * PI / 180.0;

        /* ---- O2 (or O3): segment (j, j+1) owns alpha with lambda in [0, 1) ---- */
        for (int64_t j = 0; j + 1 < nrays; ++j) {
            const double* ra = rec + ((size_t)j * np + p) * OR_NFIELD;
            const double* rb = rec + ((size_t)(j + 1) * np + p) * OR_NFIELD;
            if (ra[OR_VALID] == 0.0 || rb[OR_VALID] == 0.0) continue;
            int consistent = ra[OR_NF] == rb[OR_NF] && ra[OR_ORIENT] == rb[OR_ORIENT] &&
                             ra[OR_CAUSTIC] == 0.0 && rb[OR_CAUSTIC] == 0.0;
            double a0 = al[j * np + p];
            double da = wrap_angle(al[(j + 1) * np + p] - a0);
            if (da == 0.0) continue;
            int wi = -1;
            for (int w = 0; w < nwin; ++w)
                if (win[w].ok && j >= win[w].jlo && j + 1 <= win[w].jhi) wi = w;
            for (int64_t k = 0; k < ndir; ++k) {
                double lam = wrap_angle(alpha[k] - a0) / da;
                if (!(lam >= 0.0 && lam < 1.0)) continue;
                if (!consistent) {
                    if (wi < 0) mask[k] |= OR_MASK_CAUSTIC;
                    continue;
                }
                double wgo = 1.0;
                if (wi >= 0) wgo = 1.0 - ramp(fabs(wrap_angle(alpha[k] - win[wi].alpha_c)), po_full, po_end);
                if (wgo == 0.0) continue;
                double* acc = out + ((size_t)k * np + p) * 4;
                int exact = (flags & OR_FIELD_EXACT) != 0;
                for (int f = 0; f < nfold && !exact; ++f)
                    if (fabs(wrap_angle(alpha[k] - folds[f])) < fold_window) exact = 1;
                if (exact) {
                    double b = bj[j] + lam * (bj[j + 1] - bj[j]);
                    double* r = (double*)malloc(sizeof(double) * OR_NFIELD);
                    if (newton_fan(o, p, fan_phi, alpha[k], &b, r) >= 0) {
                        or_project_add(r + OR_F, r[OR_PSI], eth + 3 * k, eph + 3 * k, wgo, acc);
                        free(r);
                        continue;
                    }
                    free(r);
                }
                double F[6], psi = (1.0 - lam) * ra[OR_PSI] + lam * rb[OR_PSI];
                for (int c = 0; c < 6; ++c) F[c] = (1.0 - lam) * ra[OR_F + c] + lam * rb[OR_F + c];
                or_project_add(F, psi, eth + 3 * k, eph + 3 * k, wgo, acc);
            }
        }

        /* ---- O4: the PO integral over the window, blended in around the fold ---- */
        for (int w = 0; w < nwin; ++w) {
            po_window* wv = &win[w];
            if (!wv->ok) continue;
            cplx pre = sqrt(o->k0 / (2.0 * PI)) * (-I);
            for (int64_t k = 0; k < ndir; ++k) {
                double s = ramp(fabs(wrap_angle(alpha[k] - wv->alpha_c)), po_full, po_end);
                if (s == 0.0) continue;
                cplx ft = 0.0, fp = 0.0;
                for (int64_t i = 0; i <= wv->jhi - wv->jlo; ++i) {
                    cplx e = cexp(-I * o->k0 * dot3(dirv + 3 * k, wv->xap + 3 * i));
                    for (int c = 0; c < 3; ++c) {
                        ft += wv->U[3 * i + c] * e * eth[3 * k + c];
                        fp += wv->U[3 * i + c] * e * eph[3 * k + c];
                    }
                }
                ft *= pre * s;
                fp *= pre * s;
                double* acc = out + ((size_t)k * np + p) * 4;
                acc[0] += creal(ft);
                acc[1] += cimag(ft);
                acc[2] += creal(fp);
                acc[3] += cimag(fp);
                mask[k] |= OR_MASK_PO;
            }
        }
        for (int w = 0; w < nwin; ++w) {
            free(win[w].xap);
            free(win[w].U);
        }
    }
    free(rec);
    free(al);
    free(bj);
    free(eth);
    free(eph);
    free(dirv);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* O2 / O3 on a 2-D square ray grid and the (theta, phi) direction grid                    */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    double s[3];
    double F[6];
    double psi;
    double x, y; /* impact point */
    int valid, nf, orient, caustic;
} crec;

/* edge function (s_lo x s_hi) . x with the endpoints in canonical order (lower ray id first),
 * returned for the traversal a -> b; both triangles sharing the edge evaluate the same product */
static double edge_fn(int64_t ia, const double* sa, int64_t ib, const double* sb, const double* x)
{
    double c[3];
    if (ia < ib) {
        cross3(sa, sb, c);
        return dot3(c, x);
    }
    cross3(sb, sa, c);
    return -dot3(c, x);
}

/* half-open inside rule for one edge of a triangle of orientation sigma */
static int edge_in(double e, int64_t ia, int64_t ib, int sigma)
{
    double se = sigma > 0 ? e : -e;
    if (se > 0.0) return 1;
    if (se < 0.0) return 0;
    return (ia < ib) == (sigma > 0);
}

/* The square-grid field on either the cell-centred (theta, phi) grid (list == NULL) or the
 * directions of a list (n_list x (theta, phi)); one loop body tests a direction against a cell
 * triangle for both. */
/* corders (may be NULL): per direction, bit p set where a cell triangle of order p that is not
 * consistent covers it (the directions the caustic mask bit comes from, by order) */
static int64_t field_square(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi,
                            const double* list, int64_t n_list, const int64_t* window, int flags, double* out,
                            uint8_t* mask, int nthreads, int64_t* newton_fail, double near_R, uint8_t* counts,
                            uint32_t* corders)
{
    const int np = pmax + 1;
    double h, xc, yc;
    int64_t nx, ny;
    or_square_grid(o, n_target, h_in, &h, &nx, &ny, &xc, &yc);
    int64_t ix0 = 0, ix1 = nx - 1, iy0 = 0, iy1 = ny - 1; /* cells [ix0, ix1) x [iy0, iy1) */
    if (window) {
        ix0 = window[0] < 0 ? 0 : window[0];
        ix1 = window[1] > nx - 1 ? nx - 1 : window[1];
        iy0 = window[2] < 0 ? 0 : window[2];
        iy1 = window[3] > ny - 1 ? ny - 1 : window[3];
    }
    if (ix1 <= ix0 || iy1 <= iy0) return 0;
    int64_t wx = ix1 - ix0 + 1, wy = iy1 - iy0 + 1;
    crec* cr = (crec*)malloc(sizeof(crec) * (size_t)wx * wy * np);
    if (!cr) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double* buf = (double*)malloc(sizeof(double) * (size_t)np * OR_NFIELD);
        double near[OR_NFIELD];
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t jy = 0; jy < wy; ++jy)
            for (int64_t jx = 0; jx < wx; ++jx) {
                double x = grid_coord(xc, ix0 + jx, nx, h), y = grid_coord(yc, iy0 + jy, ny, h);
                /* only points strictly inside the projected cross-section are rays */
                double dx = x - xc, dy = y - yc;
                double qf = dx * (o->S[0][0] * dx + o->S[0][1] * dy) + dy * (o->S[1][0] * dx + o->S[1][1] * dy);
                if (qf < 1.0) or_trace_ray(o, x, y, pmax, buf, NULL);
                else memset(buf, 0, sizeof(double) * (size_t)np * OR_NFIELD);
                for (int p = 0; p < np; ++p) {
                    const double* r = buf + (size_t)p * OR_NFIELD;
                    if (near_R > 0.0) {
                        or_near_record(o, r, near_R, near);
                        r = near;
                    }
                    crec* c = cr + ((size_t)(jy * wx + jx) * np + p);
                    memcpy(c->s, r + OR_S, sizeof(c->s));
                    memcpy(c->F, r + OR_F, sizeof(c->F));
                    c->psi = r[OR_PSI];
                    c->x = x;
                    c->y = y;
                    c->valid = r[OR_VALID] != 0.0;
                    c->nf = (int)r[OR_NF];
                    c->orient = (int)r[OR_ORIENT];
                    c->caustic = r[OR_CAUSTIC] != 0.0;
                }
            }
        free(buf);
    }
    const int64_t ndir = list ? n_list : (int64_t)ntheta * nphi;
    const int nout = near_R > 0.0 ? 6 : 4; /* (E_r,) E_theta, E_phi: re, im */
    memset(out, 0, sizeof(double) * (size_t)ndir * np * nout);
    memset(mask, 0, (size_t)ndir);
    if (counts) memset(counts, 0, (size_t)ndir * np);
    if (corders) memset(corders, 0, sizeof(uint32_t) * (size_t)ndir);
    const double dth = list ? 1.0 : PI / ntheta, dph = list ? 1.0 : 2.0 * PI / nphi;
    double axial = 2.0 * o->lambda / o->Lmin;
    /* unit vector, e_theta, e_phi of every direction */
    double* dv = (double*)malloc(sizeof(double) * 9 * (size_t)(ndir > 0 ? ndir : 1));
    for (int64_t dk = 0; dk < ndir; ++dk) {
        double th, ph;
        if (list) {
            th = list[2 * dk];
            ph = list[2 * dk + 1];
        } else {
            th = (dk / nphi + 0.5) * dth;
            ph = -PI + (dk % nphi + 0.5) * dph;
        }
        double* d = dv + 9 * dk;
        d[0] = sin(th) * cos(ph);
        d[1] = sin(th) * sin(ph);
        d[2] = cos(th);
        d[3] = cos(th) * cos(ph);
        d[4] = cos(th) * sin(ph);
        d[5] = -sin(th);
        d[6] = -sin(ph);
        d[7] = cos(ph);
        d[8] = 0.0;
        if (th < axial || th > PI - axial) mask[dk] |= OR_MASK_AXIAL;
    }
    int64_t hits = 0, nfail = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : hits, nfail)
#endif
    for (int64_t row = 0; row < (int64_t)np * (iy1 - iy0); ++row) {
        int p = (int)(row / (iy1 - iy0));
        int64_t cy = iy0 + row % (iy1 - iy0);
        double* nbuf = (double*)malloc(sizeof(double) * OR_NFIELD);
        for (int64_t cx = ix0; cx < ix1; ++cx) {
            /* the cell (cx, cy) is split along its diagonal into two counter-clockwise triangles */
            int64_t c00 = cy * nx + cx, c10 = c00 + 1, c01 = c00 + nx, c11 = c01 + 1;
            int64_t tri[2][3] = {{c00, c10, c11}, {c00, c11, c01}};
            for (int t = 0; t < 2; ++t) {
                const crec* R[3];
                int64_t id[3];
                for (int v = 0; v < 3; ++v) {
                    id[v] = tri[t][v];
                    int64_t gx = id[v] % nx, gy = id[v] / nx;
                    R[v] = cr + ((size_t)((gy - iy0) * wx + (gx - ix0)) * np + p);
                }
                if (!R[0]->valid || !R[1]->valid || !R[2]->valid) continue;
                int consistent = R[0]->nf == R[1]->nf && R[1]->nf == R[2]->nf &&
                                 R[0]->orient == R[1]->orient && R[1]->orient == R[2]->orient &&
                                 !R[0]->caustic && !R[1]->caustic && !R[2]->caustic;
                double c12[3];
                cross3(R[1]->s, R[2]->s, c12);
                double vol = dot3(R[0]->s, c12);
                int sigma = vol > 0.0 ? 1 : (vol < 0.0 ? -1 : 0);
                if (sigma == 0) continue;
                if (sigma != R[0]->orient) consistent = 0; /* folded inside the cell */
                /* candidate directions: the cap around the normalised corner mean */
                double cm[3] = {R[0]->s[0] + R[1]->s[0] + R[2]->s[0], R[0]->s[1] + R[1]->s[1] + R[2]->s[1],
                                R[0]->s[2] + R[1]->s[2] + R[2]->s[2]};
                double cn = norm3(cm);
                if (!(cn > 0.0)) continue;
                for (int c = 0; c < 3; ++c) cm[c] /= cn;
                double mind = 1.0;
                for (int v = 0; v < 3; ++v) mind = fmin(mind, dot3(cm, R[v]->s));
                /* corners more than 90 deg from their mean do not lie in one hemisphere: the edge
                   planes then bound no proper spherical triangle, and the cell is skipped */
                if (!(mind > 0.0)) continue;
                double rho = acos(fmax(-1.0, fmin(1.0, mind))) + 1e-9;
                double thc = atan2(sqrt(cm[0] * cm[0] + cm[1] * cm[1]), cm[2]);
                double phc = atan2(cm[1], cm[0]);
                /* candidate directions: the list (all within the cap), or the grid rows and
                   columns whose centres fall in the cap */
                int64_t ncand = 0, jp0 = 0, jcount = 0;
                int it0 = 0, it1 = -1;
                if (list) {
                    ncand = ndir;
                } else {
                    it0 = (int)ceil((thc - rho) / dth - 0.5);
                    it1 = (int)floor((thc + rho) / dth - 0.5);
                    if (it0 < 0) it0 = 0;
                    if (it1 > ntheta - 1) it1 = ntheta - 1;
                    int allphi = (thc - rho <= 0.0) || (thc + rho >= PI);
                    double dphi = 0.0;
                    if (!allphi) {
                        double sr = sin(rho) / sin(thc);
                        if (sr >= 1.0) allphi = 1;
                        else dphi = asin(sr);
                    }
                    jp0 = 0;
                    jcount = nphi;
                    if (!allphi) {
                        jp0 = (int64_t)ceil((phc - dphi + PI) / dph - 0.5);
                        int64_t jp1 = (int64_t)floor((phc + dphi + PI) / dph - 0.5);
                        jcount = jp1 - jp0 + 1;
                        if (jcount > nphi) {
                            jp0 = 0;
                            jcount = nphi;
                        }
                    }
                    ncand = it1 >= it0 && jcount > 0 ? (int64_t)(it1 - it0 + 1) * jcount : 0;
                }
                const double cosr = cos(rho);
                for (int64_t q = 0; q < ncand; ++q) {
                    int64_t dk;
                    if (list) {
                        dk = q;
                        if (dot3(cm, dv + 9 * dk) < cosr - 1e-12) continue;
                    } else {
                        int it = it0 + (int)(q / jcount);
                        int64_t jp = ((jp0 + q % jcount) % nphi + nphi) % nphi;
                        dk = (int64_t)it * nphi + jp;
                    }
                    {
                        const double* x = dv + 9 * dk;
                        double e01 = edge_fn(id[0], R[0]->s, id[1], R[1]->s, x);
                        double e12 = edge_fn(id[1], R[1]->s, id[2], R[2]->s, x);
                        double e20 = edge_fn(id[2], R[2]->s, id[0], R[0]->s, x);
                        if (!edge_in(e01, id[0], id[1], sigma) || !edge_in(e12, id[1], id[2], sigma) ||
                            !edge_in(e20, id[2], id[0], sigma))
                            continue;
                        if (!consistent) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                            mask[dk] |= OR_MASK_CAUSTIC;
                            if (corders) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                                corders[dk] |= 1u << p;
                            }
                            continue;
                        }
                        /* barycentric weights of the central projection onto the corner plane */
                        double ssum = e01 + e12 + e20;
                        double l0 = e12 / ssum, l1 = e20 / ssum, l2 = e01 / ssum;
                        double F[6], psi;
                        int done = 0;
                        if (flags & OR_FIELD_EXACT) {
                            double xy[2] = {l0 * R[0]->x + l1 * R[1]->x + l2 * R[2]->x,
                                            l0 * R[0]->y + l1 * R[1]->y + l2 * R[2]->y};
                            if (or_newton(o, p, x, xy, 8.0 * h, nbuf) >= 0) {
                                memcpy(F, nbuf + OR_F, sizeof(F));
                                psi = nbuf[OR_PSI];
                                done = 1;
                            } else {
                                nfail++;
                                if (counts) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                                    counts[(size_t)dk * np + p] |= 0x80;
                                }
                            }
                        }
                        if (!done) {
                            for (int c = 0; c < 6; ++c) F[c] = l0 * R[0]->F[c] + l1 * R[1]->F[c] + l2 * R[2]->F[c];
                            psi = l0 * R[0]->psi + l1 * R[1]->psi + l2 * R[2]->psi;
                        }
                        const double* eth = x + 3;
                        const double* eph = x + 6;
                        double acc[6] = {0, 0, 0, 0, 0, 0};
                        if (nout == 6) project_add3(F, psi, x, eth, eph, acc);
                        else or_project_add(F, psi, eth, eph, 1.0, acc);
                        double* dst = out + ((size_t)dk * np + p) * nout;
                        for (int c = 0; c < nout; ++c) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                            dst[c] += acc[c];
                        }
                        if (counts) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                            counts[(size_t)dk * np + p] += 1;
                        }
                        hits++;
                    }
                }
            }
        }
        free(nbuf);
    }
    free(cr);
    free(dv);
    if (newton_fail) *newton_fail = nfail;
    return hits;
}

int64_t or_field_grid(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi,
                      const int64_t* window, int flags, double* out, uint8_t* mask, int nthreads,
                      int64_t* newton_fail)
{
    return field_square(o, n_target, h_in, pmax, ntheta, nphi, NULL, 0, window, flags, out, mask, nthreads,
                        newton_fail, 0.0, NULL, NULL);
}

int64_t or_field_grid_counts(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi,
                             int flags, double* out, uint8_t* mask, uint8_t* counts, int nthreads, int64_t* newton_fail)
{
    return field_square(o, n_target, h_in, pmax, ntheta, nphi, NULL, 0, NULL, flags, out, mask, nthreads,
                        newton_fail, 0.0, counts, NULL);
}

int64_t or_field_sphere(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi, double R,
                        double* out, uint8_t* mask, int nthreads)
{
    double rc = sqrt(dot3(o->center, o->center));
    if (!(R > rc + o->Rbound)) return -1;
    return field_square(o, n_target, h_in, pmax, ntheta, nphi, NULL, 0, NULL, 0, out, mask, nthreads, NULL, R, NULL, NULL);
}

int64_t or_field_dirs(const or_object* o, int64_t n_target, double h_in, int pmax, const double* dirs,
                      int64_t ndir, int flags, double* out, uint8_t* mask, int nthreads, int64_t* newton_fail)
{
    return field_square(o, n_target, h_in, pmax, 0, 0, dirs, ndir, NULL, flags, out, mask, nthreads,
                        newton_fail, 0.0, NULL, NULL);
}

/* ------------------------------------------------------------------------------------- */
/* 2-D physical optics over an aperture of rays ("Diffraction effect correction based on   */
/* VCRM": near singularities the ray sum is replaced by a diffraction integral of the      */
/* complex amplitudes the rays carry)                                                       */
/* ------------------------------------------------------------------------------------- */

int64_t or_field_po2d(const or_object* o, int64_t n_target, double h_in, int p, const int64_t* window,
                      double ap_theta, double ap_phi, double cone_full, double cone_end, const double* dirs,
                      int64_t ndir, double* out)
{
    double h, xc, yc;
    int64_t nx, ny;
    or_square_grid(o, n_target, h_in, &h, &nx, &ny, &xc, &yc);
    const int64_t ix0 = window[0], ix1 = window[1], iy0 = window[2], iy1 = window[3];
    if (ix0 < 0 || iy0 < 0 || ix1 >= nx || iy1 >= ny || ix1 - ix0 < 2 || iy1 - iy0 < 2 || p < 0) return -1;
    if (!(cone_full >= 0.0 && cone_end > cone_full && cone_end <= 0.5 * PI)) return -1;
    const int64_t wx = ix1 - ix0 + 1, wy = iy1 - iy0 + 1, n = wx * wy;
    /* aperture: the plane through the object centre with normal a */
    const double a[3] = {sin(ap_theta) * cos(ap_phi), sin(ap_theta) * sin(ap_phi), cos(ap_theta)};
    double* xa = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    cplx* U = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)n);
    uint8_t* ok = (uint8_t*)malloc((size_t)n);
    double* buf = (double*)malloc(sizeof(double) * (size_t)(p + 1) * OR_NFIELD);
    if (!xa || !U || !ok || !buf) {
        free(xa); free(U); free(ok); free(buf);
        return -1;
    }
    /* each ray's exit wave carried along its ray to the plane: the point x, and the field
     * U = E' sqrt(D_legs / |det(I + tau Q')|) (-i)^{N_f} e^{i k0 (L + tau)} (Eqs. IntVCRM,
     * DivFactVCRM, PhasePath), focal lines counted forward (tau > 0) or undone backward */
    double* wgt = (double*)malloc(sizeof(double) * (size_t)n);
    if (!wgt) {
        free(xa); free(U); free(ok); free(buf);
        return -1;
    }
    free(buf);
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
    double* rb = (double*)malloc(sizeof(double) * (size_t)(p + 1) * OR_NFIELD);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int64_t jy = 0; jy < wy; ++jy)
        for (int64_t jx = 0; jx < wx; ++jx) {
            const int64_t q = jy * wx + jx;
            ok[q] = 0;
            wgt[q] = 0.0;
            double x = grid_coord(xc, ix0 + jx, nx, h), y = grid_coord(yc, iy0 + jy, ny, h);
            if (!or_trace_ray(o, x, y, p, rb, NULL)) continue;
            const double* r = rb + (size_t)p * OR_NFIELD;
            if (r[OR_VALID] == 0.0) continue;
            const double* sj = r + OR_S;
            double dd[3] = {o->center[0] - r[OR_REXIT], o->center[1] - r[OR_REXIT + 1], o->center[2] - r[OR_REXIT + 2]};
            double sa = dot3(a, sj);
            if (!(fabs(sa) > 1e-6)) continue;
            double tau = dot3(a, dd) / sa;
            for (int c = 0; c < 3; ++c) xa[3 * q + c] = r[OR_REXIT + c] + tau * sj[c];
            double Am[2][2] = {{1.0 + tau * r[OR_Q], tau * r[OR_Q + 1]}, {tau * r[OR_Q + 2], 1.0 + tau * r[OR_Q + 3]}};
            double dA = det2(Am);
            if (dA == 0.0) continue;
            int nfl = neg_eigs(Am);
            int nf_ap = (int)r[OR_NFLEGS] + (tau > 0.0 ? nfl : -nfl);
            cplx amp = sqrt(r[OR_DLEGS] / fabs(dA)) * minus_i_pow(nf_ap) * cexp(I * o->k0 * (r[OR_PATH] + tau));
            cplx E0 = r[OR_E] + I * r[OR_E + 1], E1 = r[OR_E + 2] + I * r[OR_E + 3];
            for (int c = 0; c < 3; ++c) U[3 * q + c] = amp * (E0 * r[OR_V1 + c] + E1 * r[OR_V2 + c]);
            /* the aperture keeps the rays whose exit directions lie within cone_full of the axis and
             * tapers them to zero at cone_end (the role of the 1-D window's angular taper) */
            double ca = dot3(a, sj);
            wgt[q] = ramp(acos(ca > 1.0 ? 1.0 : (ca < -1.0 ? -1.0 : ca)), cone_full, cone_end);
            ok[q] = 1;
        }
    free(rb);
    }
    /* area of the plane per grid cell at each ray, from central differences of the aperture
     * points over the grid (one-sided at the window edge and next to rays that do not leave),
     * times the angular taper: each branch through a point of the plane is counted */
    int64_t used = 0;
    for (int64_t jy = 0; jy < wy; ++jy)
        for (int64_t jx = 0; jx < wx; ++jx) {
            const int64_t q = jy * wx + jx;
            if (!ok[q]) continue;
            const int64_t qxm = jx > 0 && ok[q - 1] ? q - 1 : q, qxp = jx + 1 < wx && ok[q + 1] ? q + 1 : q;
            const int64_t qym = jy > 0 && ok[q - wx] ? q - wx : q, qyp = jy + 1 < wy && ok[q + wx] ? q + wx : q;
            double w = wgt[q];
            if (qxm == qxp || qym == qyp || w == 0.0) {
                wgt[q] = 0.0; /* out of the sum; it stays a neighbour of the others */
                continue;
            }
            double ex[3], ey[3], cr[3];
            for (int c = 0; c < 3; ++c) {
                ex[c] = (xa[3 * qxp + c] - xa[3 * qxm + c]) / (double)(qxp - qxm);
                ey[c] = (xa[3 * qyp + c] - xa[3 * qym + c]) / (double)((qyp - qym) / wx);
            }
            cross3(ex, ey, cr);
            double area = fabs(dot3(cr, a));
            for (int c = 0; c < 3; ++c) U[3 * q + c] *= w * area;
            ++used;
        }
    for (int64_t q = 0; q < n; ++q)
        if (wgt[q] == 0.0) ok[q] = 0;
    /* Kirchhoff far field of the plane aperture: F(s) = k0 / (2 pi i) sum U dA e^{-i k0 s.x} */
    const cplx pre = -I * o->k0 / (2.0 * PI);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < ndir; ++k) {
        double th = dirs[2 * k], ph = dirs[2 * k + 1];
        double sv[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
        double et[3] = {cos(th) * cos(ph), cos(th) * sin(ph), -sin(th)};
        double ep[3] = {-sin(ph), cos(ph), 0.0};
        cplx ft = 0.0, fp = 0.0;
        for (int64_t q = 0; q < n; ++q) {
            if (!ok[q]) continue;
            cplx e = cexp(-I * o->k0 * dot3(sv, xa + 3 * q));
            for (int c = 0; c < 3; ++c) {
                ft += U[3 * q + c] * e * et[c];
                fp += U[3 * q + c] * e * ep[c];
            }
        }
        ft *= pre;
        fp *= pre;
        out[4 * k] = creal(ft);
        out[4 * k + 1] = cimag(ft);
        out[4 * k + 2] = creal(fp);
        out[4 * k + 3] = cimag(fp);
    }
    free(xa);
    free(U);
    free(ok);
    free(wgt);
    return used;
}

/* ------------------------------------------------------------------------------------- */
/* 2-D physical optics at the caustics of a square-grid field                              */
/* ------------------------------------------------------------------------------------- */

/* what the aperture integral needs of one (ray, order) record */
typedef struct {
    int valid;
    double s[3], r[3], Q[4], E[4], v1[3], v2[3], dlegs, nflegs, path;
} aprec;

/* Reading of "Diffraction effect correction based on VCRM" and the "Strategy of Ray Theory of
 * Waves" for 3-D caustics, which the paper leaves "under study": near the directions a fold covers,
 * the field of that order is the Kirchhoff integral of the exit waves over a plane (the 2-D form of
 * the fan's physical optics), blended into the ray sum with the fan's angular taper.
 *
 *   C_p    the directions covered by a cell triangle of order p that is not consistent (the
 *          directions whose caustic mask bit comes from order p);
 *   d_p(u) the angle from u to the nearest direction of C_p;
 *   s_p(u) = ramp(d_p(u), po_full, po_end): 1 within po_full, cos^2 down to 0 at po_end;
 *   F_p(u) = (1 - s_p(u)) F_rays,p(u) + s_p(u) F_PO,p(u).
 *
 * F_PO of a direction u of the (theta, phi) grid tile it falls in (tile_theta x tile_phi
 * directions) is taken over the plane through the object centre whose normal a is the tile's centre
 * direction: every ray of order p carries its exit wave to the plane (x, U as or_field_po2d), each
 * weighted by ramp(g, rho + cone_full, rho + cone_end) of the angle g between its exit direction
 * and a (rho: the largest angle from a to a direction of the tile), the plane's area per grid cell
 * from central differences of the neighbours' crossing points, and
 *   F_PO(u) = k0 / (2 pi i) (u . a) sum_j w_j U_j dA_j e^{-i k0 u . x_j}
 * projected on (e_theta, e_phi), the far field of the plane's field (Rayleigh-Sommerfeld; the factor
 * u . a makes the result independent of the plane to the order of the ray fields themselves).
 * Orders p >= p_min are corrected; the caustic bit stays on a direction of C_p only where s_p < 1
 * (so none, for po_full > 0: s_p = 1 on C_p), and every corrected direction has OR_MASK_PO. */
int64_t or_field_grid_caustic(const or_object* o, int64_t n_target, double h_in, int pmax, int ntheta, int nphi,
                              const double* cp, double* out, uint8_t* mask, double* weights, uint32_t* corders_out,
                              double* l1, int nthreads)
{
    const int np = pmax + 1;
    const int tt = (int)cp[0], tp = (int)cp[1];
    const double po_full = cp[2], po_end = cp[3], cone_full = cp[4], cone_end = cp[5];
    const int p_min = (int)cp[6];
    if (o->src || o->shape_e != 1.0) return -1; /* plane wave on an ellipsoid */
    if (ntheta < 1 || nphi < 1 || tt < 1 || tp < 1 || p_min < 0 || p_min > pmax || pmax > 31) return -1;
    if (!(po_full >= 0.0 && po_end > po_full && cone_full >= 0.0 && cone_end > cone_full)) return -1;
    const int64_t ndir = (int64_t)ntheta * nphi;
    const double dth = PI / ntheta, dph = 2.0 * PI / nphi;
    double h, xc, yc;
    int64_t nx, ny;
    or_square_grid(o, n_target, h_in, &h, &nx, &ny, &xc, &yc);
    const int nc = np - p_min;
    const int64_t nv = nx * ny;
    uint32_t* corders = (uint32_t*)calloc((size_t)ndir, sizeof(uint32_t));
    double* sw = (double*)malloc(sizeof(double) * (size_t)ndir);
    aprec* ar = (aprec*)calloc((size_t)nv * nc, sizeof(aprec));
    double* dv = (double*)malloc(sizeof(double) * 9 * (size_t)ndir);
    double* xq = (double*)malloc(sizeof(double) * 3 * (size_t)nv);
    double* wq = (double*)malloc(sizeof(double) * (size_t)nv);
    uint8_t* okq = (uint8_t*)malloc((size_t)nv);
    cplx* Tq = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)nv);
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)nv);
    int64_t* cdir = (int64_t*)malloc(sizeof(int64_t) * (size_t)ndir);
    /* the ray sum of every order, and the orders of the caustic directions */
    int64_t rc = -1;
    if (corders && sw && ar && dv && xq && wq && okq && Tq && list && cdir)
        rc = field_square(o, n_target, h_in, pmax, ntheta, nphi, NULL, 0, NULL, 0, out, mask, nthreads, NULL, 0.0,
                          NULL, corders);
    if (rc < 0) {
        free(corders); free(sw); free(ar); free(dv); free(xq); free(wq); free(okq); free(Tq); free(list); free(cdir);
        return rc;
    }
    if (weights) memset(weights, 0, sizeof(double) * (size_t)ndir * np);
    if (l1) memset(l1, 0, sizeof(double) * (size_t)ndir * np);
    /* the exit records of every grid vertex for the corrected orders */
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double* buf = (double*)malloc(sizeof(double) * (size_t)np * OR_NFIELD);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ix = 0; ix < nx; ++ix) {
                double x = grid_coord(xc, ix, nx, h), y = grid_coord(yc, iy, ny, h);
                double dx = x - xc, dy = y - yc;
                double qf = dx * (o->S[0][0] * dx + o->S[0][1] * dy) + dy * (o->S[1][0] * dx + o->S[1][1] * dy);
                if (!(qf < 1.0)) continue;
                or_trace_ray(o, x, y, pmax, buf, NULL);
                for (int p = p_min; p < np; ++p) {
                    const double* r = buf + (size_t)p * OR_NFIELD;
                    aprec* a = ar + (size_t)(p - p_min) * nv + iy * nx + ix;
                    a->valid = r[OR_VALID] != 0.0;
                    if (!a->valid) continue;
                    memcpy(a->s, r + OR_S, sizeof(a->s));
                    memcpy(a->r, r + OR_REXIT, sizeof(a->r));
                    memcpy(a->Q, r + OR_Q, sizeof(a->Q));
                    memcpy(a->E, r + OR_E, sizeof(a->E));
                    memcpy(a->v1, r + OR_V1, sizeof(a->v1));
                    memcpy(a->v2, r + OR_V2, sizeof(a->v2));
                    a->dlegs = r[OR_DLEGS];
                    a->nflegs = r[OR_NFLEGS];
                    a->path = r[OR_PATH];
                }
            }
        free(buf);
    }
    /* unit vector, e_theta, e_phi of every direction */
    for (int64_t k = 0; k < ndir; ++k) {
        double th = (k / nphi + 0.5) * dth, ph = -PI + (k % nphi + 0.5) * dph;
        double* d = dv + 9 * k;
        d[0] = sin(th) * cos(ph);
        d[1] = sin(th) * sin(ph);
        d[2] = cos(th);
        d[3] = cos(th) * cos(ph);
        d[4] = cos(th) * sin(ph);
        d[5] = -sin(th);
        d[6] = -sin(ph);
        d[7] = cos(ph);
        d[8] = 0.0;
    }
    const int ntt = (ntheta + tt - 1) / tt, ntp = (nphi + tp - 1) / tp;
    const cplx pre = -I * o->k0 / (2.0 * PI);
    /* the caustic orders of each direction that the correction leaves uncovered (s_p < 1) */
    uint32_t* left = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)ndir);
    if (!left) rc = -1;
    else memcpy(left, corders, sizeof(uint32_t) * (size_t)ndir);
    for (int p = p_min; p < np && rc >= 0; ++p) {
        const aprec* arp = ar + (size_t)(p - p_min) * nv;
        /* s_p: the taper of the angle to the nearest caustic direction of order p; the caustic
         * directions are listed in row order, and only rows within po_end can be that close */
        int64_t ncd = 0;
        for (int64_t k = 0; k < ndir; ++k)
            if (corders[k] & (1u << p)) cdir[ncd++] = k;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
        for (int64_t k = 0; k < ndir; ++k) {
            const double thk = (k / nphi + 0.5) * dth;
            double best = -2.0;
            for (int64_t c = 0; c < ncd; ++c) {
                const double thc = (cdir[c] / nphi + 0.5) * dth;
                if (fabs(thc - thk) > po_end) continue;
                best = fmax(best, dot3(dv + 9 * k, dv + 9 * cdir[c]));
            }
            const double d = best < -1.5 ? 2.0 * PI : acos(fmin(1.0, fmax(-1.0, best)));
            sw[k] = d < po_end ? ramp(d, po_full, po_end) : 0.0;
        }
        for (int bt = 0; bt < ntt && rc >= 0; ++bt)
            for (int bp = 0; bp < ntp && rc >= 0; ++bp) {
                const int r0 = bt * tt, r1 = r0 + tt < ntheta ? r0 + tt : ntheta;
                const int c0 = bp * tp, c1 = c0 + tp < nphi ? c0 + tp : nphi;
                int active = 0;
                for (int i = r0; i < r1; ++i)
                    for (int j = c0; j < c1; ++j) active |= sw[(int64_t)i * nphi + j] > 0.0;
                if (!active) continue;
                /* the aperture of the tile: the plane through the centre normal to the tile's
                 * centre direction; rho, the largest angle from there to a direction of the tile */
                const double tha = 0.5 * (r0 + r1) * dth, pha = -PI + 0.5 * (c0 + c1) * dph;
                const double a[3] = {sin(tha) * cos(pha), sin(tha) * sin(pha), cos(tha)};
                double rho = 0.0;
                for (int i = r0; i < r1; ++i)
                    for (int j = c0; j < c1; ++j)
                        rho = fmax(rho, acos(fmin(1.0, fmax(-1.0, dot3(a, dv + 9 * ((int64_t)i * nphi + j))))));
                const double cf = rho + cone_full, ce = rho + cone_end;
                if (!(ce < 0.5 * PI)) {
                    rc = -2; /* the cone reaches the plane */
                    break;
                }
                /* every ray's crossing point; the field and weight of those in the cone */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256)
#endif
                for (int64_t q = 0; q < nv; ++q) {
                    const aprec* r = arp + q;
                    okq[q] = 0;
                    wq[q] = 0.0;
                    if (!r->valid) continue;
                    const double sa = dot3(a, r->s);
                    if (!(fabs(sa) > 1e-6)) continue;
                    const double dd[3] = {o->center[0] - r->r[0], o->center[1] - r->r[1], o->center[2] - r->r[2]};
                    const double tau = dot3(a, dd) / sa;
                    for (int c = 0; c < 3; ++c) xq[3 * q + c] = r->r[c] + tau * r->s[c];
                    okq[q] = 1;
                    const double w = ramp(acos(fmin(1.0, fmax(-1.0, sa))), cf, ce);
                    if (w == 0.0) continue;
                    double Am[2][2] = {{1.0 + tau * r->Q[0], tau * r->Q[1]}, {tau * r->Q[2], 1.0 + tau * r->Q[3]}};
                    const double det = det2(Am);
                    if (det == 0.0) continue;
                    const int nfl = neg_eigs(Am);
                    const int nf_ap = (int)r->nflegs + (tau > 0.0 ? nfl : -nfl);
                    const cplx amp = sqrt(r->dlegs / fabs(det)) * minus_i_pow(nf_ap) * cexp(I * o->k0 * (r->path + tau));
                    const cplx E0 = r->E[0] + I * r->E[1], E1 = r->E[2] + I * r->E[3];
                    for (int c = 0; c < 3; ++c) Tq[3 * q + c] = amp * (E0 * r->v1[c] + E1 * r->v2[c]);
                    wq[q] = w;
                }
                /* the plane's area per grid cell (central differences, one-sided next to a
                 * vertex without a crossing, none where an axis has no neighbour at all) */
                int64_t nl = 0;
                for (int64_t q = 0; q < nv; ++q) {
                    if (wq[q] == 0.0) continue;
                    const int64_t ix = q % nx, iy = q / nx;
                    const int64_t qxm = ix > 0 && okq[q - 1] ? q - 1 : q, qxp = ix + 1 < nx && okq[q + 1] ? q + 1 : q;
                    const int64_t qym = iy > 0 && okq[q - nx] ? q - nx : q, qyp = iy + 1 < ny && okq[q + nx] ? q + nx : q;
                    if (qxm == qxp || qym == qyp) continue;
                    double ex[3], ey[3], cr[3];
                    for (int c = 0; c < 3; ++c) {
                        ex[c] = (xq[3 * qxp + c] - xq[3 * qxm + c]) / (double)(qxp - qxm);
                        ey[c] = (xq[3 * qyp + c] - xq[3 * qym + c]) / (double)((qyp - qym) / nx);
                    }
                    cross3(ex, ey, cr);
                    const double f = wq[q] * fabs(dot3(cr, a));
                    for (int c = 0; c < 3; ++c) Tq[3 * q + c] *= f;
                    list[nl++] = q;
                }
                /* the far field of the plane at the tile's directions in the correction zone */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
                for (int i = r0; i < r1; ++i)
                    for (int j = c0; j < c1; ++j) {
                        const int64_t k = (int64_t)i * nphi + j;
                        if (!(sw[k] > 0.0)) continue;
                        const double* u = dv + 9 * k;
                        cplx v[3] = {0.0, 0.0, 0.0};
                        double norm1 = 0.0;
                        for (int64_t m = 0; m < nl; ++m) {
                            const int64_t q = list[m];
                            const cplx e = cexp(-I * o->k0 * dot3(u, xq + 3 * q));
                            double t2 = 0.0;
                            for (int c = 0; c < 3; ++c) {
                                v[c] += Tq[3 * q + c] * e;
                                t2 += creal(Tq[3 * q + c]) * creal(Tq[3 * q + c]) + cimag(Tq[3 * q + c]) * cimag(Tq[3 * q + c]);
                            }
                            norm1 += sqrt(t2);
                        }
                        const double ua = dot3(u, a);
                        cplx ft = 0.0, fp = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            ft += v[c] * u[3 + c];
                            fp += v[c] * u[6 + c];
                        }
                        ft *= pre * ua;
                        fp *= pre * ua;
                        const double s = sw[k];
                        double* acc = out + ((size_t)k * np + p) * 4;
                        acc[0] = (1.0 - s) * acc[0] + s * creal(ft);
                        acc[1] = (1.0 - s) * acc[1] + s * cimag(ft);
                        acc[2] = (1.0 - s) * acc[2] + s * creal(fp);
                        acc[3] = (1.0 - s) * acc[3] + s * cimag(fp);
                        if (l1) l1[(size_t)k * np + p] = s * o->k0 / (2.0 * PI) * fabs(ua) * norm1;
                        mask[k] |= OR_MASK_PO;
                    }
            }
        for (int64_t k = 0; k < ndir && rc >= 0; ++k) {
            if (weights) weights[(size_t)k * np + p] = sw[k];
            if (sw[k] == 1.0) left[k] &= ~(1u << p); /* the order's ray sum is wholly replaced */
        }
    }
    /* the caustic bit stays where an order's caustic direction is not wholly corrected */
    if (rc >= 0)
        for (int64_t k = 0; k < ndir; ++k)
            mask[k] = (uint8_t)((mask[k] & ~OR_MASK_CAUSTIC) | (left[k] ? OR_MASK_CAUSTIC : 0u));
    if (corders_out) memcpy(corders_out, corders, sizeof(uint32_t) * (size_t)ndir);
    free(left);
    free(corders);
    free(sw);
    free(ar);
    free(dv);
    free(xq);
    free(wq);
    free(okq);
    free(Tq);
    free(list);
    free(cdir);
    return rc;
}

/* ------------------------------------------------------------------------------------- */
/* Learned proposal: network seeds, Newton on the exact trace, deduplicated roots          */
/* ------------------------------------------------------------------------------------- */

#include "mlp_oracle.h"

/* the learned field on the cell-centred (theta, phi) grid (list == NULL) or on the directions of a
 * list (n_list x (theta, phi)) */
static int64_t field_learned(const or_object* o, const double* theta, int pmax, int ntheta, int nphi,
                             const double* list, int64_t n_list, double p_min, int max_steps, double tol,
                             int max_halvings, double* out, uint8_t* mask, uint8_t* roots)
{
    const int np = pmax + 1;
    const int64_t ndir = list ? n_list : (int64_t)ntheta * nphi;
    const double dth = list ? 1.0 : PI / ntheta, dph = list ? 1.0 : 2.0 * PI / nphi;
    const double axial = 2.0 * o->lambda / o->Lmin;
    const double dedup = 1e-6 * o->Lmax;
    /* tol <= 0: per object, a phase error k0 L |s - t| below 1e-4 rad */
    if (!(tol > 0.0)) tol = fmin(1e-6, 1e-4 / (o->k0 * o->Lmax));
    memset(out, 0, sizeof(double) * 4 * (size_t)np * (size_t)ndir);
    memset(mask, 0, (size_t)ndir);
    if (roots) memset(roots, 0, (size_t)ndir * (size_t)np);
    int64_t total = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
#endif
    for (int64_t dk = 0; dk < ndir; ++dk) {
        double th, ph;
        if (list) {
            th = list[2 * dk];
            ph = list[2 * dk + 1];
        } else {
            th = ((int)(dk / nphi) + 0.5) * dth;
            ph = -PI + ((int)(dk % nphi) + 0.5) * dph;
        }
        const double s[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
        const double eth[3] = {cos(th) * cos(ph), cos(th) * sin(ph), -sin(th)};
        const double eph[3] = {-sin(ph), cos(ph), 0.0};
        uint8_t mk = (th < axial || th > PI - axial) ? OR_MASK_AXIAL : 0;
        double x[OM_IN], y[OM_OUT];
        om_features(o, s, x);
        double* rec = (double*)malloc(sizeof(double) * (size_t)np * OR_NFIELD);
        for (int p = 0; p < np; ++p) {
            om_forward(theta + (size_t)p * OM_NPARAM, x, 1, 1, y);
            /* softmax weights of the heads */
            double zmax = y[8], w[OM_HEADS], se = 0.0;
            for (int k = 1; k < OM_HEADS; ++k) zmax = fmax(zmax, y[8 + k]);
            for (int k = 0; k < OM_HEADS; ++k) {
                w[k] = exp(y[8 + k] - zmax);
                se += w[k];
            }
            double found[OM_HEADS][2];
            int nfound = 0, uncertain = 0;
            for (int k = 0; k < OM_HEADS; ++k) {
                if (w[k] / se < p_min) continue;
                double xy[2];
                double uv[2] = {y[2 * k], y[2 * k + 1]};
                /* an entry point lies inside the section: seeds beyond radius 0.999 move onto it */
                const double ru = hypot(uv[0], uv[1]);
                if (ru > 0.999) {
                    uv[0] *= 0.999 / ru;
                    uv[1] *= 0.999 / ru;
                }
                om_uv_to_xy(o, uv, &xy[0], &xy[1]);
                if (or_newton_ex(o, p, s, xy, 0.0, max_steps + 1, tol, max_halvings, rec) < 0) {
                    uncertain = 1; /* a confident head that did not converge */
                    continue;
                }
                int dup = 0;
                for (int q = 0; q < nfound; ++q)
                    if (hypot(xy[0] - found[q][0], xy[1] - found[q][1]) <= dedup) dup = 1;
                if (dup) continue;
                found[nfound][0] = xy[0];
                found[nfound][1] = xy[1];
                nfound++;
                if (rec[OR_CAUSTIC] != 0.0) {
                    mk |= OR_MASK_CAUSTIC;
                    continue;
                }
                or_project_add(rec + OR_F, rec[OR_PSI], eth, eph, 1.0, out + ((size_t)dk * np + p) * 4);
            }
            if (roots) roots[(size_t)dk * np + p] = (uint8_t)(nfound | (uncertain ? 0x80 : 0));
            total += nfound;
        }
        free(rec);
        mask[dk] = mk;
    }
    return total;
}

int64_t or_field_learned(const or_object* o, const double* theta, int pmax, int ntheta, int nphi, double p_min,
                         int max_steps, double tol, int max_halvings, double* out, uint8_t* mask, uint8_t* roots)
{
    return field_learned(o, theta, pmax, ntheta, nphi, NULL, 0, p_min, max_steps, tol, max_halvings, out, mask,
                         roots);
}

int64_t or_field_learned_dirs(const or_object* o, const double* theta, int pmax, const double* dirs, int64_t ndir,
                              double p_min, int max_steps, double tol, int max_halvings, double* out, uint8_t* mask,
                              uint8_t* roots)
{
    return field_learned(o, theta, pmax, 0, 0, dirs, ndir, p_min, max_steps, tol, max_halvings, out, mask, roots);
}
