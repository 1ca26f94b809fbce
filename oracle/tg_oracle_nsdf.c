/*
 * tg_oracle_nsdf.c -- FP64 oracle of the learned signed-distance surrogate of
 * an object: a multiresolution hash encoding (Mueller, Evans, Schied, Keller,
 * "Instant Neural Graphics Primitives with a Multiresolution Hash Encoding",
 * 2022) of the object-frame point, feeding a ReLU MLP whose single output is
 * the signed distance in millimetres.
 *
 * TEST INFRASTRUCTURE ONLY (see tg_oracle.h): shares nothing with the CUDA
 * path.
 *
 * The paper fixes only the sizes (16 levels, 2 features per level, 2^16
 * entries per level, two hidden layers of 64, BF16 weights, FP16 table).  The
 * readings taken here:
 *   - level l = 0..15 has N_l = floor(16 * 2^(l/3)) cells per axis, the
 *     geometric series from 16 to 512 (exact powers of two at l = 0, 3, ..15);
 *   - the point u = (q - lo) / (hi - lo) in [0,1]^3 sits in cell
 *     i = min(floor(u N_l), N_l - 1) with fractions f = u N_l - i;
 *   - vertex (i, j, k) of a level is stored at entry i + (N+1) (j + (N+1) k)
 *     while (N+1)^3 <= 2^16, else at (i xor j * 2654435761 xor
 *     k * 805459861) mod 2^16 in 32-bit unsigned arithmetic (the primes of
 *     the hash encoding's paper);
 *   - each entry holds 2 binary16 features; the level's 2 encoding values are
 *     the trilinear interpolation of the cell's 8 corner entries;
 *   - enc (32) -> h1 = ReLU(W1 enc) (64) -> h2 = ReLU(W2 h1) (64) ->
 *     out = W3 h2, millimetres; no biases (6,208 bfloat16 weights);
 *   - with round = 1, enc, h1 and h2 are rounded to bfloat16 (nearest, ties
 *     to even) before the next product, as a tensor-core evaluation does;
 *     round = 0 is the exact real-valued network;
 *   - outside the encoding box phi = phi(clamp(q)) + |q - clamp(q)| with the
 *     gradient taken at the clamped point, as for the SDF grids;
 *   - training loss: mean over the batch of |out - label| (labels in mm);
 *     gradients pass through the bfloat16 roundings unchanged;
 *   - Adam with bias correction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "tg_oracle.h"

/* ---- bfloat16 <-> double, from the format (1 sign, 8 exponent, 7 fraction bits) */
double or_bf16_to_double(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* nearest bfloat16, ties to even; finite inputs */
uint16_t or_double_to_bf16(double x) {
    if (isnan(x)) return 0x7fc0u;
    double a = fabs(x), r;
    if (a == 0.0) {
        r = 0.0;
    } else if (a < 0x1p-126) {        /* subnormal: multiples of 2^-133 */
        r = nearbyint(a * 0x1p133) * 0x1p-133;
    } else {
        int e;
        double m = frexp(a, &e);      /* a = m 2^e, m in [0.5, 1): 8 significant bits kept */
        r = ldexp(nearbyint(ldexp(m, 8)), e - 8);
        if (r >= 0x1p128) r = INFINITY;
    }
    float f = (float)copysign(r, x);
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

static double bf16_round(double x) { return or_bf16_to_double(or_double_to_bf16(x)); }

/* ---- encoding geometry ------------------------------------------------------ */
int32_t or_nsdf_resolution(int32_t level) {
    if (level % 3 == 0) return 16 << (level / 3);
    return (int32_t)floor(16.0 * pow(2.0, (double)level / 3.0));
}

uint32_t or_nsdf_index(int32_t level, int64_t i, int64_t j, int64_t k) {
    const int64_t n1 = (int64_t)or_nsdf_resolution(level) + 1;
    if (n1 * n1 * n1 <= (int64_t)OR_NSDF_TABLE) return (uint32_t)(i + n1 * (j + n1 * k));
    uint32_t h = (uint32_t)i ^ ((uint32_t)j * 2654435761u) ^ ((uint32_t)k * 805459861u);
    return h & (OR_NSDF_TABLE - 1u);
}

static double feat(const or_nsdf* n, int l, uint32_t idx, int f) {
    return or_half_to_double(n->table[((size_t)l * OR_NSDF_TABLE + idx) * OR_NSDF_FEATURES + f]);
}

/* one level: corner entries, weights and d(weight)/d(fraction) */
typedef struct {
    uint32_t idx[8];
    double w[8];
    double dw[8][3];
    int32_t res;
} level_cell;

static void cell_of(int l, const double u[3], level_cell* c) {
    const int32_t N = or_nsdf_resolution(l);
    int64_t i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double p = u[a] * (double)N;
        int64_t i = (int64_t)floor(p);
        if (i > N - 1) i = N - 1;
        if (i < 0) i = 0;
        i0[a] = i;
        f[a] = p - (double)i;
    }
    c->res = N;
    for (int corner = 0; corner < 8; ++corner) {
        const int d[3] = {corner & 1, (corner >> 1) & 1, (corner >> 2) & 1};
        double t[3], dt[3];
        for (int a = 0; a < 3; ++a) {
            t[a] = d[a] ? f[a] : 1.0 - f[a];
            dt[a] = d[a] ? 1.0 : -1.0;
        }
        c->idx[corner] = or_nsdf_index(l, i0[0] + d[0], i0[1] + d[1], i0[2] + d[2]);
        c->w[corner] = t[0] * t[1] * t[2];
        c->dw[corner][0] = dt[0] * t[1] * t[2];
        c->dw[corner][1] = t[0] * dt[1] * t[2];
        c->dw[corner][2] = t[0] * t[1] * dt[2];
    }
}

/* everything a forward pass computes for one point */
typedef struct {
    double c[3];                       /* clamped point */
    double u[3];
    level_cell cell[OR_NSDF_LEVELS];
    double enc[OR_NSDF_IN];            /* after rounding when round = 1 */
    double z1[OR_NSDF_HIDDEN], h1[OR_NSDF_HIDDEN];
    double z2[OR_NSDF_HIDDEN], h2[OR_NSDF_HIDDEN];
    double out;                        /* mm */
} nsdf_trace;

static double W1(const or_nsdf* n, int o, int i) { return or_bf16_to_double(n->w1[o * OR_NSDF_IN + i]); }
static double W2(const or_nsdf* n, int o, int i) { return or_bf16_to_double(n->w2[o * OR_NSDF_HIDDEN + i]); }
static double W3(const or_nsdf* n, int i) { return or_bf16_to_double(n->w3[i]); }

static void forward(const or_nsdf* n, const double q[3], int round, nsdf_trace* t) {
    for (int a = 0; a < 3; ++a) {
        t->c[a] = q[a] < n->lo[a] ? n->lo[a] : (q[a] > n->hi[a] ? n->hi[a] : q[a]);
        t->u[a] = (t->c[a] - n->lo[a]) / (n->hi[a] - n->lo[a]);
    }
    for (int l = 0; l < OR_NSDF_LEVELS; ++l) {
        level_cell* c = &t->cell[l];
        cell_of(l, t->u, c);
        for (int f = 0; f < OR_NSDF_FEATURES; ++f) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += c->w[k] * feat(n, l, c->idx[k], f);
            t->enc[l * OR_NSDF_FEATURES + f] = round ? bf16_round(s) : s;
        }
    }
    for (int o = 0; o < OR_NSDF_HIDDEN; ++o) {
        double s = 0.0;
        for (int i = 0; i < OR_NSDF_IN; ++i) s += W1(n, o, i) * t->enc[i];
        t->z1[o] = s;
        double h = s > 0.0 ? s : 0.0;
        t->h1[o] = round ? bf16_round(h) : h;
    }
    for (int o = 0; o < OR_NSDF_HIDDEN; ++o) {
        double s = 0.0;
        for (int i = 0; i < OR_NSDF_HIDDEN; ++i) s += W2(n, o, i) * t->h1[i];
        t->z2[o] = s;
        double h = s > 0.0 ? s : 0.0;
        t->h2[o] = round ? bf16_round(h) : h;
    }
    double s = 0.0;
    for (int i = 0; i < OR_NSDF_HIDDEN; ++i) s += W3(n, i) * t->h2[i];
    t->out = s;
}

/* d out / d enc by the chain rule through the ReLUs (roundings pass through) */
static void out_grad_enc(const or_nsdf* n, const nsdf_trace* t, double g_enc[OR_NSDF_IN], double g_z1[OR_NSDF_HIDDEN],
                         double g_z2[OR_NSDF_HIDDEN]) {
    for (int o = 0; o < OR_NSDF_HIDDEN; ++o) g_z2[o] = t->z2[o] > 0.0 ? W3(n, o) : 0.0;
    for (int i = 0; i < OR_NSDF_HIDDEN; ++i) {
        double s = 0.0;
        for (int o = 0; o < OR_NSDF_HIDDEN; ++o) s += g_z2[o] * W2(n, o, i);
        g_z1[i] = t->z1[i] > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < OR_NSDF_IN; ++i) {
        double s = 0.0;
        for (int o = 0; o < OR_NSDF_HIDDEN; ++o) s += g_z1[o] * W1(n, o, i);
        g_enc[i] = s;
    }
}

double or_nsdf_eval(const or_nsdf* n, const double q[3], int32_t round, double grad_raw[3]) {
    nsdf_trace* t = (nsdf_trace*)malloc(sizeof(nsdf_trace));
    forward(n, q, round, t);
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = q[a] - t->c[a];
    const double phi = 1e-3 * t->out + sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (grad_raw) {
        double g_enc[OR_NSDF_IN], g_z1[OR_NSDF_HIDDEN], g_z2[OR_NSDF_HIDDEN];
        out_grad_enc(n, t, g_enc, g_z1, g_z2);
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int l = 0; l < OR_NSDF_LEVELS; ++l) {
                const level_cell* c = &t->cell[l];
                for (int f = 0; f < OR_NSDF_FEATURES; ++f) {
                    double de = 0.0;
                    for (int k = 0; k < 8; ++k) de += c->dw[k][a] * feat(n, l, c->idx[k], f);
                    s += g_enc[l * OR_NSDF_FEATURES + f] * de * (double)c->res;
                }
            }
            /* d phi (m) / d q (m): the net is in mm over u = (q - lo) / extent */
            grad_raw[a] = 1e-3 * s / (n->hi[a] - n->lo[a]);
        }
    }
    free(t);
    return phi;
}

/* Contact normal of a learned SDF: the gradient by the four-point
   tetrahedral central difference at h = 0.25 mm (object frame),
   sum_k v_k phi(q + h v_k) / (4 h) with v_k = (1,-1,-1), (-1,-1,1),
   (-1,1,-1), (1,1,1) (sum_k v_k v_k^T = 4 I, so the stencil is exact on
   affine fields).  phi is the full distance, outside extension included.
   The analytic gradient of a hash-encoded network jumps at every cell face
   of its finest levels (cells of ~0.1 mm); the stencil averages over a few
   of them. */
void or_nsdf_normal(const or_nsdf* n, const double q[3], int32_t round, double g[3]) {
    static const double v[4][3] = {{1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}, {1, 1, 1}};
    const double h = 2.5e-4;
    g[0] = g[1] = g[2] = 0.0;
    for (int k = 0; k < 4; ++k) {
        double p[3] = {q[0] + h * v[k][0], q[1] + h * v[k][1], q[2] + h * v[k][2]};
        const double phi = or_nsdf_eval(n, p, round, 0);
        for (int a = 0; a < 3; ++a) g[a] += v[k][a] * phi / (4.0 * h);
    }
}

/* Largest change of `out` (mm) that one bfloat16 rounding decided the other
   way can cause: an activation moved by one bfloat16 spacing at its value,
   propagated through |W| (the ReLU pattern held fixed). */
double or_nsdf_flip_bound(const or_nsdf* n, const double q[3]) {
    nsdf_trace* t = (nsdf_trace*)malloc(sizeof(nsdf_trace));
    forward(n, q, 1, t);
    double a2[OR_NSDF_HIDDEN], a1[OR_NSDF_HIDDEN], best = 0.0;
    for (int o = 0; o < OR_NSDF_HIDDEN; ++o) a2[o] = t->z2[o] > 0.0 ? fabs(W3(n, o)) : 0.0;
    for (int i = 0; i < OR_NSDF_HIDDEN; ++i) {
        double s = 0.0;
        for (int o = 0; o < OR_NSDF_HIDDEN; ++o) s += a2[o] * fabs(W2(n, o, i));
        a1[i] = t->z1[i] > 0.0 ? s : 0.0;
    }
#define ULP(x) ((x) == 0.0 ? 0.0 : ldexp(1.0, ilogb(x) - 7))
    for (int o = 0; o < OR_NSDF_HIDDEN; ++o) {
        double v = (t->z2[o] > 0.0 ? fabs(W3(n, o)) : 0.0) * ULP(t->h2[o]);
        if (v > best) best = v;
        v = a1[o] * ULP(t->h1[o]);
        if (v > best) best = v;
    }
    for (int i = 0; i < OR_NSDF_IN; ++i) {
        double s = 0.0;
        for (int o = 0; o < OR_NSDF_HIDDEN; ++o) s += a1[o] * fabs(W1(n, o, i));
        double v = s * ULP(t->enc[i]);
        if (v > best) best = v;
    }
#undef ULP
    free(t);
    return best;
}

/* Mean L1 loss over a batch and its gradient with respect to every weight
   and every table entry (FP64, dense arrays: g_w1 [64][32], g_w2 [64][64],
   g_w3 [64], g_table [16][2^16][2]).  Returns the loss. */
double or_nsdf_loss_grad(const or_nsdf* n, int64_t B, const double* pts, const double* labels_mm, int32_t round,
                         double* g_w1, double* g_w2, double* g_w3, double* g_table) {
    memset(g_w1, 0, sizeof(double) * OR_NSDF_HIDDEN * OR_NSDF_IN);
    memset(g_w2, 0, sizeof(double) * OR_NSDF_HIDDEN * OR_NSDF_HIDDEN);
    memset(g_w3, 0, sizeof(double) * OR_NSDF_HIDDEN);
    memset(g_table, 0, sizeof(double) * OR_NSDF_LEVELS * OR_NSDF_TABLE * OR_NSDF_FEATURES);
    nsdf_trace* t = (nsdf_trace*)malloc(sizeof(nsdf_trace));
    double loss = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        forward(n, pts + 3 * b, round, t);
        const double r = t->out - labels_mm[b];
        loss += fabs(r);
        const double g_out = (r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0)) / (double)B;
        if (g_out == 0.0) continue;
        double g_z2[OR_NSDF_HIDDEN], g_z1[OR_NSDF_HIDDEN], g_enc[OR_NSDF_IN];
        for (int i = 0; i < OR_NSDF_HIDDEN; ++i) g_w3[i] += g_out * t->h2[i];
        for (int o = 0; o < OR_NSDF_HIDDEN; ++o) g_z2[o] = t->z2[o] > 0.0 ? g_out * W3(n, o) : 0.0;
        for (int o = 0; o < OR_NSDF_HIDDEN; ++o)
            for (int i = 0; i < OR_NSDF_HIDDEN; ++i) g_w2[o * OR_NSDF_HIDDEN + i] += g_z2[o] * t->h1[i];
        for (int i = 0; i < OR_NSDF_HIDDEN; ++i) {
            double s = 0.0;
            for (int o = 0; o < OR_NSDF_HIDDEN; ++o) s += g_z2[o] * W2(n, o, i);
            g_z1[i] = t->z1[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < OR_NSDF_HIDDEN; ++o)
            for (int i = 0; i < OR_NSDF_IN; ++i) g_w1[o * OR_NSDF_IN + i] += g_z1[o] * t->enc[i];
        for (int i = 0; i < OR_NSDF_IN; ++i) {
            double s = 0.0;
            for (int o = 0; o < OR_NSDF_HIDDEN; ++o) s += g_z1[o] * W1(n, o, i);
            g_enc[i] = s;
        }
        for (int l = 0; l < OR_NSDF_LEVELS; ++l)
            for (int k = 0; k < 8; ++k)
                for (int f = 0; f < OR_NSDF_FEATURES; ++f)
                    g_table[((size_t)l * OR_NSDF_TABLE + t->cell[l].idx[k]) * OR_NSDF_FEATURES + f] +=
                        t->cell[l].w[k] * g_enc[l * OR_NSDF_FEATURES + f];
    }
    free(t);
    return loss / (double)B;
}

/* One Adam step (bias-corrected; t counts from 1) over n parameters. */
void or_adam_step(int64_t n, double* theta, double* m, double* v, const double* g, double lr, double beta1,
                  double beta2, double eps, int32_t t) {
    const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* batched evaluation for the tests */
void or_nsdf_eval_batch(const or_nsdf* n, int64_t B, const double* pts, int32_t round, double* phi, double* grad_raw) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t b = 0; b < B; ++b) phi[b] = or_nsdf_eval(n, pts + 3 * b, round, grad_raw ? grad_raw + 3 * b : 0);
}

void or_nsdf_normal_batch(const or_nsdf* n, int64_t B, const double* pts, int32_t round, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t b = 0; b < B; ++b) or_nsdf_normal(n, pts + 3 * b, round, g + 3 * b);
}

void or_nsdf_flip_bound_batch(const or_nsdf* n, int64_t B, const double* pts, double* out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t b = 0; b < B; ++b) out[b] = or_nsdf_flip_bound(n, pts + 3 * b);
}
