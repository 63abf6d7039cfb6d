/*
 * mlp_oracle.c -- plain FP64 CPU oracle of the learned inverse-map proposal (see mlp_oracle.h).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Written for reading, not speed: one row at a time,
 * every layer a plain double loop, backpropagation by hand in the order of the forward pass
 * reversed.
 */
#include "mlp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double kPiO = 3.14159265358979323846;

/* tanh form of GELU and its derivative */
double om_gelu(double z)
{
    const double c = sqrt(2.0 / kPiO);
    return 0.5 * z * (1.0 + tanh(c * (z + 0.044715 * z * z * z)));
}

double om_gelu_grad(double z)
{
    const double c = sqrt(2.0 / kPiO);
    const double u = c * (z + 0.044715 * z * z * z);
    const double t = tanh(u);
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * c * (1.0 + 3.0 * 0.044715 * z * z);
}

/* bfloat16: the upper 16 bits of the IEEE single, rounded to nearest even */
double om_round_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan unchanged */
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

void om_features(const or_object* o, const double s[3], double* x)
{
    double R[9], semi[3], m;
    or_object_frame(o, R, semi, NULL, NULL, &m);
    const double L = fmax(semi[0], fmax(semi[1], semi[2]));
    for (int i = 0; i < 3; ++i) x[i] = s[i];
    for (int i = 0; i < 9; ++i) x[3 + i] = R[i];
    for (int i = 0; i < 3; ++i) x[12 + i] = semi[i] / L;
    x[15] = m - 1.0;
}

/* Cholesky factor of S: S = L L^T, L lower triangular */
static void chol2(const double S[4], double* l00, double* l10, double* l11)
{
    *l00 = sqrt(S[0]);
    *l10 = S[2] / *l00;
    *l11 = sqrt(S[3] - *l10 * *l10);
}

void om_xy_to_uv(const or_object* o, double x, double y, double uv[2])
{
    double c[3], S[4], l00, l10, l11;
    or_object_frame(o, NULL, NULL, c, S, NULL);
    chol2(S, &l00, &l10, &l11);
    const double d0 = x - c[0], d1 = y - c[1];
    uv[0] = l00 * d0 + l10 * d1;
    uv[1] = l11 * d1;
}

void om_uv_to_xy(const or_object* o, const double uv[2], double* x, double* y)
{
    double c[3], S[4], l00, l10, l11;
    or_object_frame(o, NULL, NULL, c, S, NULL);
    chol2(S, &l00, &l10, &l11);
    const double d1 = uv[1] / l11;
    const double d0 = (uv[0] - l10 * d1) / l00;
    *x = c[0] + d0;
    *y = c[1] + d1;
}

static double rb(double v, int bf16) { return bf16 ? om_round_bf16(v) : v; }

/* one dense layer: out[o] = sum_i W[o][i] in[i] + b[o] */
static void dense(const double* W, const double* b, const double* in, int nin, int nout, int bf16, double* out)
{
    for (int o = 0; o < nout; ++o) {
        double acc = 0.0;
        for (int i = 0; i < nin; ++i) acc += rb(W[o * nin + i], bf16) * in[i];
        out[o] = acc + b[o];
    }
}

/* forward pass of one row; keeps the pre-activations z1..z3 and the layer inputs a0..a3 */
typedef struct {
    double a0[OM_IN];
    double z1[OM_H], a1[OM_H];
    double z2[OM_H], a2[OM_H];
    double z3[OM_H], a3[OM_H];
    double y[OM_OUT];
} om_row;

static void forward_row(const double* th, const double* x, int bf16, om_row* r)
{
    for (int i = 0; i < OM_IN; ++i) r->a0[i] = rb(x[i], bf16);
    dense(th + OM_W1, th + OM_B1, r->a0, OM_IN, OM_H, bf16, r->z1);
    for (int i = 0; i < OM_H; ++i) r->a1[i] = rb(om_gelu(r->z1[i]), bf16);
    dense(th + OM_W2, th + OM_B2, r->a1, OM_H, OM_H, bf16, r->z2);
    for (int i = 0; i < OM_H; ++i) r->a2[i] = rb(om_gelu(r->z2[i]), bf16);
    dense(th + OM_W3, th + OM_B3, r->a2, OM_H, OM_H, bf16, r->z3);
    for (int i = 0; i < OM_H; ++i) r->a3[i] = rb(om_gelu(r->z3[i]), bf16);
    dense(th + OM_W4, th + OM_B4, r->a3, OM_H, OM_OUT, bf16, r->y);
}

void om_forward(const double* theta, const double* x, int64_t n, int bf16, double* y)
{
    om_row* r = (om_row*)malloc(sizeof(om_row));
    for (int64_t i = 0; i < n; ++i) {
        forward_row(theta, x + i * OM_IN, bf16, r);
        memcpy(y + i * OM_OUT, r->y, sizeof(r->y));
    }
    free(r);
}

/* gradient of one layer given dz (nout): dW += dz a^T, db += dz, din = W^T dz */
static void dense_back(const double* W, const double* a, const double* dz, int nin, int nout, int bf16, double* dW,
                       double* db, double* din)
{
    for (int o = 0; o < nout; ++o) {
        db[o] += dz[o];
        for (int i = 0; i < nin; ++i) dW[o * nin + i] += dz[o] * a[i];
    }
    if (din)
        for (int i = 0; i < nin; ++i) {
            double acc = 0.0;
            for (int o = 0; o < nout; ++o) acc += rb(W[o * nin + i], bf16) * dz[o];
            din[i] = acc;
        }
}

double om_loss_grad(const double* theta, const double* x, const double* target, const uint8_t* label, int64_t n,
                    double beta, int bf16, double* grad)
{
    memset(grad, 0, sizeof(double) * OM_NPARAM);
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) nv += label[i] != 0;
    if (nv == 0) return 0.0;
    const double inv = 1.0 / (double)nv;
    om_row* r = (om_row*)malloc(sizeof(om_row));
    double loss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!label[i]) continue;
        forward_row(theta, x + i * OM_IN, bf16, r);
        const double* t = target + 2 * i;
        /* the head of the ray's branch carries the regression term */
        const int j = (label[i] - 1) % OM_HEADS;
        const double e0 = r->y[2 * j] - t[0], e1 = r->y[2 * j + 1] - t[1];
        const double best = e0 * e0 + e1 * e1;
        /* softmax cross-entropy of the logits against head j */
        double zmax = r->y[8];
        for (int k = 1; k < OM_HEADS; ++k) zmax = fmax(zmax, r->y[8 + k]);
        double se = 0.0, pk[OM_HEADS];
        for (int k = 0; k < OM_HEADS; ++k) {
            pk[k] = exp(r->y[8 + k] - zmax);
            se += pk[k];
        }
        for (int k = 0; k < OM_HEADS; ++k) pk[k] /= se;
        loss += (best - beta * log(pk[j])) * inv;
        double dy[OM_OUT] = {0};
        dy[2 * j] = 2.0 * (r->y[2 * j] - t[0]) * inv;
        dy[2 * j + 1] = 2.0 * (r->y[2 * j + 1] - t[1]) * inv;
        for (int k = 0; k < OM_HEADS; ++k) dy[8 + k] = beta * (pk[k] - (k == j ? 1.0 : 0.0)) * inv;
        double d3[OM_H], d2[OM_H], d1[OM_H];
        dense_back(theta + OM_W4, r->a3, dy, OM_H, OM_OUT, bf16, grad + OM_W4, grad + OM_B4, d3);
        for (int k = 0; k < OM_H; ++k) d3[k] *= om_gelu_grad(r->z3[k]);
        dense_back(theta + OM_W3, r->a2, d3, OM_H, OM_H, bf16, grad + OM_W3, grad + OM_B3, d2);
        for (int k = 0; k < OM_H; ++k) d2[k] *= om_gelu_grad(r->z2[k]);
        dense_back(theta + OM_W2, r->a1, d2, OM_H, OM_H, bf16, grad + OM_W2, grad + OM_B2, d1);
        for (int k = 0; k < OM_H; ++k) d1[k] *= om_gelu_grad(r->z1[k]);
        dense_back(theta + OM_W1, r->a0, d1, OM_IN, OM_H, bf16, grad + OM_W1, grad + OM_B1, NULL);
    }
    free(r);
    return loss;
}

void om_adam(double* theta, double* m, double* v, const double* grad, int64_t n, int t, double lr, double b1,
             double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
