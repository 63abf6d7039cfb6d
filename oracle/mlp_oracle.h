/*
 * mlp_oracle.h -- plain FP64 CPU oracle of the learned inverse-map proposal (MLP) that seeds
 * Newton steps on the exact trace.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite and the CPU-baseline leg of
 * bench.py may load this code.  It shares nothing with the CUDA library.
 *
 * The paper has no learned component; this follows the network stated for the learned proposal
 * (per scattering order: 3 hidden layers of width 128, GELU, K = 4 candidate entry points with
 * confidences).  Definitions fixed here (and restated, independently, by the CUDA side):
 *
 *   features x (16): exit direction s (3, lab frame), the rotation matrix R body -> lab
 *                    (9, row-major), semi-axes over the largest one (3), m - 1 (1);
 *   entry point uv:  d = (x - cx, y - cy) on the incidence plane, S = L L^T the Cholesky
 *                    factor of the projected ellipse (d^T S d <= 1 inside), uv = L^T d,
 *                    so that the projected section is the unit disk;
 *   network:         h1 = g(W1 x + b1), h2 = g(W2 h1 + b2), h3 = g(W3 h2 + b3),
 *                    y = W4 h3 + b4; W_l row-major (out x in); g the tanh form of GELU,
 *                    g(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
 *   outputs y (16):  y[2k], y[2k+1] the uv of head k (k < 4), y[8 + k] the logit of head k,
 *                    y[12..15] unused;
 *   labels:          a row's label is 0 (no ray: ignored) or 1 + (N_f mod 4), N_f the focal
 *                    lines of its ray: the branches of one direction and order differ in N_f
 *                    (their orientation follows its parity), so head N_f mod 4 learns one branch;
 *   loss of a row:   j = label - 1, loss = |uv_j - uv*|^2 + beta CE(softmax(y[8..11]), j);
 *                    mean over the labelled rows;
 *   Adam:            m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *                    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * bf16 = 1 rounds the weights, the inputs and every hidden activation to bfloat16 (round to
 * nearest even) before it enters a product, as the tensor-core kernels do; arithmetic stays FP64.
 */
#ifndef MLP_ORACLE_H
#define MLP_ORACLE_H

#include <stdint.h>

#include "rtw_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

#define OM_IN 16
#define OM_H 128
#define OM_OUT 16
#define OM_HEADS 4
/* parameter offsets (doubles) */
#define OM_W1 0
#define OM_B1 (OM_W1 + OM_H * OM_IN)
#define OM_W2 (OM_B1 + OM_H)
#define OM_B2 (OM_W2 + OM_H * OM_H)
#define OM_W3 (OM_B2 + OM_H)
#define OM_B3 (OM_W3 + OM_H * OM_H)
#define OM_W4 (OM_B3 + OM_H)
#define OM_B4 (OM_W4 + OM_OUT * OM_H)
#define OM_NPARAM (OM_B4 + OM_OUT)

double om_gelu(double z);
double om_gelu_grad(double z);
double om_round_bf16(double v);

/* features of exit direction s for object o (16 doubles) */
void om_features(const or_object* o, const double s[3], double* x);
/* entry point (x, y) <-> unit-disk coordinates uv */
void om_xy_to_uv(const or_object* o, double x, double y, double uv[2]);
void om_uv_to_xy(const or_object* o, const double uv[2], double* x, double* y);

/* y (n x 16) of rows x (n x 16) */
void om_forward(const double* theta, const double* x, int64_t n, int bf16, double* y);
/* mean loss over the labelled rows (label 1..4: head label - 1 carries the target; 0: ignored)
 * and its gradient (OM_NPARAM doubles, overwritten) */
double om_loss_grad(const double* theta, const double* x, const double* target, const uint8_t* label, int64_t n,
                    double beta, int bf16, double* grad);
/* one Adam step t (1-based) on n parameters */
void om_adam(double* theta, double* m, double* v, const double* grad, int64_t n, int t, double lr, double b1,
             double b2, double eps);

#ifdef __cplusplus
}
#endif
#endif
