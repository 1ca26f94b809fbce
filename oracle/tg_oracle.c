/*
 * tg_oracle.c -- FP64 CPU oracle for the Tactile Genesis contact query and
 * noise model.  TEST INFRASTRUCTURE ONLY (see tg_oracle.h): used by tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs, never
 * by the product path.
 *
 * Each function follows one passage of the paper (arxiv 2606.22332):
 *   Appendix A "Probe geometry and contact-depth query"  Eqs. 1-2
 *   Appendix A "ContactProbe"                          Eq. 3
 *   Appendix A "KinematicTaxel"                        Eqs. 4-9, 11
 *   Appendix A "Sensor Noise Model"                    Eqs. 25-31
 *   Appendix B "Tactile Observation Types"             Eq. 32 (agg_force)
 * plus the published methods the paper relies on without printing them:
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *   Box-Muller (1958),
 *   closest point on a triangle by Voronoi regions (Ericson, RTCD 5.1.5),
 *   generalised winding number (Jacobson et al. 2013) with the
 *   Van Oosterom-Strackee (1983) solid angle.
 * Where the paper is silent, each function states the reading it takes.
 */
#include "tg_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

/* ======================================================================== */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 bit     */
/* multiplications with the published multipliers and Weyl key increments. */
/* ======================================================================== */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0,1): the top 24 bits plus one half, scaled by 2^-24 */
double or_uniform(uint32_t x) { return ((double)(x >> 8) + 0.5) * 0x1p-24; }

/* Box-Muller: two independent standard normals from two uniforms */
void or_box_muller(uint32_t x0, uint32_t x1, double* z0, double* z1) {
    double u0 = or_uniform(x0), u1 = or_uniform(x1);
    double r = sqrt(-2.0 * log(u0));
    *z0 = r * cos(2.0 * PI * u1);
    *z1 = r * sin(2.0 * PI * u1);
}

/* Philox stream tags: which draw a counter belongs to */
enum {
    TAG_EPISODE = 1,  /* w0 dead Bernoulli, w1..w3 gain (depth, ft, prox) */
    TAG_STUCK = 2,    /* w0..w2 stuck readout uniforms (depth, ft, prox) */
    TAG_FT_A = 16,    /* normals: drift fx fy fz tx */
    TAG_FT_B = 17,    /* normals: drift ty tz, white fx fy */
    TAG_FT_C = 18,    /* normals: white fz tx ty tz */
    TAG_SCALAR = 19,  /* normals: drift depth, white depth, drift prox, white prox */
    TAG_RADIUS = 20,  /* w0: probe-radius noise */
    TAG_DR = 32,      /* per-env domain randomisation */
    TAG_JITTER = 33   /* per-env read-delay jitter */
};

static void philox_draw(uint64_t seed, uint64_t gid, uint32_t word1, uint32_t tag, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)gid, word1, tag, (uint32_t)(gid >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* Probe-radius noise offset (Appendix "Sensor Noise Model", probe-level
   imperfections): eps = rho (2u - 1), u the 24-bit uniform of word w.  It is
   formed in binary32 -- u as (float)(w >> 8) + 1/2 rounded, times 2^-24;
   2u - 1 is then exact; one rounding of the product -- so that every
   implementation forms the same value. */
static float radius_eps(double rho, uint32_t w) {
    volatile float u = ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-08f;
    volatile float s = 2.0f * u - 1.0f;
    volatile float e = (float)rho * s;
    return e;
}

static void philox_normals(uint64_t seed, uint64_t gid, uint32_t step, uint32_t tag, double z[4]) {
    uint32_t w[4];
    philox_draw(seed, gid, step, tag, w);
    or_box_muller(w[0], w[1], &z[0], &z[1]);
    or_box_muller(w[2], w[3], &z[2], &z[3]);
}

/* Per-step domain randomisation of one env (config 4 of the evaluation):
   one Philox block at counter (env id, step, DR, 0) gives u0, u1, u2 and
   mu = lo + (hi - lo) u0, k = ... u1, scale = ... u2.  The bounds and the
   drawn values are binary32 numbers, the precision per-env parameters have
   when a caller passes them in: the value is formed in FP64 and rounded. */
void or_dr_draw(const or_params* P, uint32_t env_gid, uint32_t step, double out[3]) {
    uint32_t w[4];
    philox_draw(P->seed, env_gid, step, TAG_DR, w);
    const double* b[3] = {P->dr_mu, P->dr_k, P->dr_scale};
    for (int i = 0; i < 3; ++i) {
        double lo = (double)(float)b[i][0], hi = (double)(float)b[i][1];
        out[i] = (double)(float)(lo + (hi - lo) * or_uniform(w[i]));
    }
}

/* Bernoulli(p) decided on integers: the top 24 bits below round(p 2^24) */
static int bernoulli(uint32_t x, double p) {
    double thr = nearbyint(p * 16777216.0);
    return (double)(x >> 8) < thr;
}

/* ======================================================================== */
/* IEEE 754 binary16 <-> double, written from the format definition.        */
/* ======================================================================== */
uint16_t or_double_to_half(double x) {
    uint16_t sign = signbit(x) ? 0x8000u : 0u;
    double a = fabs(x);
    if (isnan(x)) return 0x7e00u;
    if (a >= 65520.0) return (uint16_t)(sign | 0x7c00u);
    if (a < 0x1p-14) {            /* subnormal: a multiple of 2^-24 */
        double m = nearbyint(a * 0x1p24);
        return (uint16_t)(sign | (uint16_t)m);
    }
    int e;
    double fr = frexp(a, &e);     /* a = fr 2^e, fr in [0.5, 1) */
    int E = e - 1;                /* a = (1 + f) 2^E */
    double m = nearbyint((fr * 2.0 - 1.0) * 1024.0);
    if (m == 1024.0) { m = 0.0; E += 1; }
    if (E > 15) return (uint16_t)(sign | 0x7c00u);
    return (uint16_t)(sign | (uint16_t)((E + 15) << 10) | (uint16_t)m);
}

double or_half_to_double(uint16_t h) {
    int s = h >> 15, E = (h >> 10) & 31, m = h & 1023;
    double v;
    if (E == 0) v = ldexp((double)m, -24);
    else if (E == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(m + 1024), E - 25);
    return s ? -v : v;
}

/* ======================================================================== */
/* small vector helpers                                                      */
/* ======================================================================== */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3]) {
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void sub3(const double a[3], const double b[3], double o[3]) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void matvec(const double R[9], const double v[3], double o[3]) {
    double t0 = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    double t1 = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    double t2 = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static void matTvec(const double R[9], const double v[3], double o[3]) {
    double t0 = R[0] * v[0] + R[3] * v[1] + R[6] * v[2];
    double t1 = R[1] * v[0] + R[4] * v[1] + R[7] * v[2];
    double t2 = R[2] * v[0] + R[5] * v[1] + R[8] * v[2];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static void matmul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

/* ======================================================================== */
/* Poses (Appendix A, Eq. 1 and the constant-velocity advance of the        */
/* synthetic workload): rotation of a quaternion of any norm, Rodrigues.    */
/* ======================================================================== */
void or_quat_to_mat(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double s = 2.0 / (w * w + x * x + y * y + z * z);
    R[0] = 1.0 - s * (y * y + z * z); R[1] = s * (x * y - w * z);       R[2] = s * (x * z + w * y);
    R[3] = s * (x * y + w * z);       R[4] = 1.0 - s * (x * x + z * z); R[5] = s * (y * z - w * x);
    R[6] = s * (x * z - w * y);       R[7] = s * (y * z + w * x);       R[8] = 1.0 - s * (x * x + y * y);
}

/* p = p0 + v tau ;  R = exp([w] tau) R(q0)  with exp by Rodrigues' formula */
void or_advance_pose(const double p0[3], const double q0[4], const double v[3],
                     const double w[3], double tau, double p[3], double R[9]) {
    double R0[9];
    or_quat_to_mat(q0, R0);
    for (int a = 0; a < 3; ++a) p[a] = p0[a] + v[a] * tau;
    double th = norm3(w) * tau;
    if (th == 0.0) { memcpy(R, R0, sizeof(R0)); return; }
    double k[3] = {w[0] / norm3(w), w[1] / norm3(w), w[2] / norm3(w)};
    double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
    double K2[9];
    matmul(K, K, K2);
    double s = sin(th), c1 = 1.0 - cos(th);
    double E[9];
    for (int i = 0; i < 9; ++i) E[i] = (i % 4 == 0 ? 1.0 : 0.0) + s * K[i] + c1 * K2[i];
    matmul(E, R0, R);
}

/* ======================================================================== */
/* Signed distance fields (Appendix A, Eq. 2: depth uses phi_g, normal is   */
/* grad phi).  Every function returns phi and writes the unit gradient g.   */
/* ======================================================================== */
double or_sdf_sphere(double r, const double q[3], double g[3]) {
    double n = norm3(q);
    if (n > 0.0) { g[0] = q[0] / n; g[1] = q[1] / n; g[2] = q[2] / n; }
    else { g[0] = 0.0; g[1] = 0.0; g[2] = 1.0; }
    return n - r;
}

/* axis-aligned box of half extents h centred at the origin */
double or_sdf_box(const double h[3], const double q[3], double g[3]) {
    double d[3], o[3];
    for (int a = 0; a < 3; ++a) { d[a] = fabs(q[a]) - h[a]; o[a] = d[a] > 0.0 ? d[a] : 0.0; }
    double outside = norm3(o);
    int amax = 0;
    if (d[1] > d[amax]) amax = 1;
    if (d[2] > d[amax]) amax = 2;
    if (outside > 0.0) {
        for (int a = 0; a < 3; ++a) g[a] = (q[a] < 0.0 ? -o[a] : o[a]) / outside;
        return outside;
    }
    g[0] = g[1] = g[2] = 0.0;
    g[amax] = q[amax] < 0.0 ? -1.0 : 1.0;
    return d[amax];
}

/* half-space z <= 0 (the surface is the plane z = 0, outward normal +z) */
double or_sdf_plane(const double q[3], double g[3]) {
    g[0] = 0.0; g[1] = 0.0; g[2] = 1.0;
    return q[2];
}

/* Closest point on triangle abc to p by Voronoi-region classification.
   region: 0 face, 1 a, 2 b, 3 c, 4 edge ab, 5 edge ac, 6 edge bc.
   Returns the Euclidean distance |p - cp|. */
double or_closest_point_triangle(const double p[3], const double a[3], const double b[3],
                                 const double c[3], double cp[3], int* region) {
    double ab[3], ac[3], ap[3], bp[3], cpv[3];
    sub3(b, a, ab); sub3(c, a, ac); sub3(p, a, ap);
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) {
        memcpy(cp, a, 3 * sizeof(double)); *region = 1;
        goto done;
    }
    sub3(p, b, bp);
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) {
        memcpy(cp, b, 3 * sizeof(double)); *region = 2;
        goto done;
    }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double v = d1 / (d1 - d3);
        for (int i = 0; i < 3; ++i) cp[i] = a[i] + v * ab[i];
        *region = 4;
        goto done;
    }
    sub3(p, c, cpv);
    double d5 = dot3(ab, cpv), d6 = dot3(ac, cpv);
    if (d6 >= 0.0 && d5 <= d6) {
        memcpy(cp, c, 3 * sizeof(double)); *region = 3;
        goto done;
    }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double w = d2 / (d2 - d6);
        for (int i = 0; i < 3; ++i) cp[i] = a[i] + w * ac[i];
        *region = 5;
        goto done;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int i = 0; i < 3; ++i) cp[i] = b[i] + w * (c[i] - b[i]);
        *region = 6;
        goto done;
    }
    {
        double den = 1.0 / (va + vb + vc);
        double v = vb * den, w = vc * den;
        for (int i = 0; i < 3; ++i) cp[i] = a[i] + ab[i] * v + ac[i] * w;
        *region = 0;
    }
done:;
    double dd[3];
    sub3(p, cp, dd);
    return norm3(dd);
}

static void vert(const float* V, int32_t i, double o[3]) {
    o[0] = (double)V[3 * i]; o[1] = (double)V[3 * i + 1]; o[2] = (double)V[3 * i + 2];
}

/* ray-triangle intersection (Moller and Trumbore 1997): t >= 0 of the hit of
   o + t d with triangle abc, or -1 */
static double ray_triangle(const double o[3], const double d[3], const double a[3], const double b[3],
                           const double c[3]) {
    double e1[3], e2[3], p[3], s[3], qv[3];
    sub3(b, a, e1); sub3(c, a, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (fabs(det) < 1e-300) return -1.0;
    double inv = 1.0 / det;
    sub3(o, a, s);
    double u = dot3(s, p) * inv;
    if (u < 0.0 || u > 1.0) return -1.0;
    cross3(s, e1, qv);
    double v = dot3(d, qv) * inv;
    if (v < 0.0 || u + v > 1.0) return -1.0;
    double t = dot3(e2, qv) * inv;
    return t >= 0.0 ? t : -1.0;
}

double or_raycast_depth(const float* V, const int32_t* F, int32_t nf, double scale, const double q[3],
                        const double u[3], double R, double n_out[3], int32_t* face_out, double* ray_pen) {
    double best = 0.0, rbest = -INFINITY;
    int32_t bface = -1;
    for (int32_t f = 0; f < nf; ++f) {
        double a[3], b[3], c[3], cp[3];
        int reg;
        vert(V, F[3 * f], a); vert(V, F[3 * f + 1], b); vert(V, F[3 * f + 2], c);
        for (int i = 0; i < 3; ++i) { a[i] *= scale; b[i] *= scale; c[i] *= scale; }
        double pen = R - or_closest_point_triangle(q, a, b, c, cp, &reg);
        double t = ray_triangle(q, u, a, b, c);
        if (t >= 0.0) {
            if (R - t > rbest) rbest = R - t;
            if (R - t > pen) pen = R - t;
        }
        if (pen > best) {
            best = pen;
            bface = f;
        }
    }
    n_out[0] = n_out[1] = n_out[2] = 0.0;
    if (bface >= 0) {
        double a[3], b[3], c[3], e1[3], e2[3];
        vert(V, F[3 * bface], a); vert(V, F[3 * bface + 1], b); vert(V, F[3 * bface + 2], c);
        sub3(b, a, e1); sub3(c, a, e2);
        cross3(e1, e2, n_out);
        double l = norm3(n_out);
        for (int i = 0; i < 3; ++i) n_out[i] /= l;
    }
    if (face_out) *face_out = bface;
    if (ray_pen) *ray_pen = rbest;
    return best;
}

/* 1 when a triangle other than `face` whose normal is not parallel to n
   penetrates within 1e-12 m of `pen` (an edge or a vertex shared by
   non-coplanar faces is the deepest feature: either face's normal is the
   backend's answer) */
static int raycast_tie(const float* V, const int32_t* F, int32_t nf, double scale, const double q[3], double R,
                       double pen, int32_t face, const double n[3]) {
    for (int32_t f = 0; f < nf; ++f) {
        if (f == face) continue;
        double a[3], b[3], c[3], cp[3], e1[3], e2[3], m[3];
        int reg;
        vert(V, F[3 * f], a); vert(V, F[3 * f + 1], b); vert(V, F[3 * f + 2], c);
        for (int i = 0; i < 3; ++i) { a[i] *= scale; b[i] *= scale; c[i] *= scale; }
        if (R - or_closest_point_triangle(q, a, b, c, cp, &reg) < pen - 1e-12) continue;
        sub3(b, a, e1); sub3(c, a, e2);
        cross3(e1, e2, m);
        if (fabs(dot3(m, n)) < (1.0 - 1e-9) * norm3(m)) return 1;
    }
    return 0;
}

/* generalised winding number: sum of signed solid angles / (4 pi) */
double or_winding_number(const float* V, const int32_t* F, int32_t nf, const double p[3]) {
    double total = 0.0;
    for (int32_t f = 0; f < nf; ++f) {
        double a[3], b[3], c[3], A[3], B[3], C[3], BxC[3];
        vert(V, F[3 * f], a); vert(V, F[3 * f + 1], b); vert(V, F[3 * f + 2], c);
        sub3(a, p, A); sub3(b, p, B); sub3(c, p, C);
        double la = norm3(A), lb = norm3(B), lc = norm3(C);
        cross3(B, C, BxC);
        double num = dot3(A, BxC);
        double den = la * lb * lc + dot3(A, B) * lc + dot3(B, C) * la + dot3(C, A) * lb;
        total += 2.0 * atan2(num, den);
    }
    return total / (4.0 * PI);
}

/* exact mesh SDF: unsigned distance = min over faces; negative where the
   winding number exceeds 1/2; gradient sign (q - c*)/|q - c*|, or the face
   normal of the nearest face when the point lies on the surface. */
double or_sdf_mesh(const float* V, const int32_t* F, int32_t nf, const double p[3], double g[3]) {
    double best = INFINITY, bcp[3] = {0, 0, 0};
    int32_t bface = 0;
    for (int32_t f = 0; f < nf; ++f) {
        double a[3], b[3], c[3], cp[3];
        int reg;
        vert(V, F[3 * f], a); vert(V, F[3 * f + 1], b); vert(V, F[3 * f + 2], c);
        double d = or_closest_point_triangle(p, a, b, c, cp, &reg);
        if (d < best) { best = d; bface = f; memcpy(bcp, cp, sizeof(bcp)); }
    }
    double w = or_winding_number(V, F, nf, p);
    double sign = w > 0.5 ? -1.0 : 1.0;
    if (best >= 1e-12) {
        for (int i = 0; i < 3; ++i) g[i] = sign * (p[i] - bcp[i]) / best;
    } else {
        double a[3], b[3], c[3], ab[3], ac[3], n[3];
        vert(V, F[3 * bface], a); vert(V, F[3 * bface + 1], b); vert(V, F[3 * bface + 2], c);
        sub3(b, a, ab); sub3(c, a, ac); cross3(ab, ac, n);
        double nn = norm3(n);
        for (int i = 0; i < 3; ++i) g[i] = n[i] / nn;
    }
    return sign * best;
}

/* Sampled grid: node (i,j,k) at lo + (i,j,k) h, h = (hi - lo)/(dims - 1);
   trilinear interpolation of the stored values at the point clamped into the
   box, plus the distance from the point to the box; the gradient is the
   analytic gradient of the trilinear interpolant at the clamped point. */
static double grid_node(const or_object* o, int i, int j, int k) {
    size_t idx = ((size_t)k * (size_t)o->dims[1] + (size_t)j) * (size_t)o->dims[0] + (size_t)i;
    if (o->fp16) return or_half_to_double(((const uint16_t*)o->values)[idx]);
    return (double)((const float*)o->values)[idx];
}

double or_sdf_grid(const or_object* o, const double q[3], double g[3]) {
    double c[3], f[3], h[3];
    int i0[3];
    for (int a = 0; a < 3; ++a) {
        c[a] = q[a] < o->lo[a] ? o->lo[a] : (q[a] > o->hi[a] ? o->hi[a] : q[a]);
        h[a] = (o->hi[a] - o->lo[a]) / (double)(o->dims[a] - 1);
        double u = (c[a] - o->lo[a]) / h[a];
        int i = (int)floor(u);
        if (i > o->dims[a] - 2) i = o->dims[a] - 2;
        if (i < 0) i = 0;
        i0[a] = i;
        f[a] = u - (double)i;
    }
    double v[2][2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) v[dz][dy][dx] = grid_node(o, i0[0] + dx, i0[1] + dy, i0[2] + dz);
    double fx = f[0], fy = f[1], fz = f[2];
    double phi = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                phi += v[dz][dy][dx] * (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy) gx += (v[dz][dy][1] - v[dz][dy][0]) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
    for (int dz = 0; dz < 2; ++dz)
        for (int dx = 0; dx < 2; ++dx) gy += (v[dz][1][dx] - v[dz][0][dx]) * (dx ? fx : 1.0 - fx) * (dz ? fz : 1.0 - fz);
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) gz += (v[1][dy][dx] - v[0][dy][dx]) * (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
    double gr[3] = {gx / h[0], gy / h[1], gz / h[2]};
    double gn = norm3(gr);
    if (gn > 0.0) { g[0] = gr[0] / gn; g[1] = gr[1] / gn; g[2] = gr[2] / gn; }
    else {
        double qn = norm3(q);
        if (qn > 0.0) { g[0] = q[0] / qn; g[1] = q[1] / qn; g[2] = q[2] / qn; }
        else { g[0] = 0.0; g[1] = 0.0; g[2] = 1.0; }
    }
    double out[3];
    sub3(q, c, out);
    return phi + norm3(out);
}

double or_sdf_object(const or_object* o, const double q[3], double g[3]) {
    switch (o->kind) {
    case OR_SPHERE: return or_sdf_sphere(o->radius, q, g);
    case OR_BOX: return or_sdf_box(o->half, q, g);
    case OR_PLANE: return or_sdf_plane(q, g);
    case OR_MESH: return or_sdf_mesh(o->verts, o->faces, o->n_faces, q, g);
    case OR_GRID: return or_sdf_grid(o, q, g);
    case OR_NEURAL: {
        double gr[3];
        double phi = or_nsdf_eval(o->nsdf, q, 1, 0);
        or_nsdf_normal(o->nsdf, q, 1, gr);
        double gn = norm3(gr);
        if (gn > 0.0) { g[0] = gr[0] / gn; g[1] = gr[1] / gn; g[2] = gr[2] / gn; }
        else {
            double qn = norm3(q);
            if (qn > 0.0) { g[0] = q[0] / qn; g[1] = q[1] / qn; g[2] = q[2] / qn; }
            else { g[0] = 0.0; g[1] = 0.0; g[2] = 1.0; }
        }
        return phi;
    }
    default: g[0] = g[1] = g[2] = NAN; return NAN;
    }
}

void or_sdf_object_batch(const or_object* o, const double* q, int64_t n, double* phi, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) phi[i] = or_sdf_object(o, q + 3 * i, g + 3 * i);
}

/* exact mesh SDF sampled at the grid nodes, rounded to float or binary16 */
void or_bake_grid(const float* V, const int32_t* F, int32_t nf, const int32_t dims[3],
                  const double lo[3], const double hi[3], int32_t fp16, void* out, int32_t threads) {
    int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = 0; idx < n; ++idx) {
        int i = (int)(idx % dims[0]);
        int j = (int)((idx / dims[0]) % dims[1]);
        int k = (int)(idx / ((int64_t)dims[0] * dims[1]));
        double p[3], g[3];
        p[0] = lo[0] + i * ((hi[0] - lo[0]) / (double)(dims[0] - 1));
        p[1] = lo[1] + j * ((hi[1] - lo[1]) / (double)(dims[1] - 1));
        p[2] = lo[2] + k * ((hi[2] - lo[2]) / (double)(dims[2] - 1));
        double phi = or_sdf_mesh(V, F, nf, p, g);
        if (fp16) ((uint16_t*)out)[idx] = or_double_to_half(phi);
        else ((float*)out)[idx] = (float)phi;
    }
}

/* ======================================================================== */
/* Proximity by rays: the first root of the signed distance along a ray.    */
/* The object frame may be scaled: phi_world(t) = s phi(q0 + t d) with d    */
/* the world-unit ray direction mapped into the object frame (|d| = 1/s).   */
/* grazing is set when the root is ill-posed: a crossing at a shallow      */
/* angle (|d phi_world / dt| < 0.05), a near miss (min phi_world < 2e-5),  */
/* or a skim (the ray leaves again before it is 2e-5 deep).                */
/* ======================================================================== */
#define OR_GRAZE_SLOPE 0.05
#define OR_GRAZE_GAP 2e-5

static double poly_eval(const double c[4], double t) { return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]; }
static double poly_deriv(const double c[4], double t) { return (3.0 * c[3] * t + 2.0 * c[2]) * t + c[1]; }

/* first root of the cubic on [a, b] (NAN if none); tracks the minimum value */
static double cubic_first_root(const double c[4], double a, double b, double* vmin) {
    double pts[4];
    int np = 0;
    pts[np++] = a;
    /* critical points inside (a, b) */
    double A = 3.0 * c[3], B = 2.0 * c[2], Cc = c[1];
    double crit[2];
    int nc = 0;
    if (A != 0.0) {
        double disc = B * B - 4.0 * A * Cc;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            double r1 = (-B - sq) / (2.0 * A), r2 = (-B + sq) / (2.0 * A);
            if (r1 > r2) { double t = r1; r1 = r2; r2 = t; }
            crit[nc++] = r1;
            crit[nc++] = r2;
        }
    } else if (B != 0.0) {
        crit[nc++] = -Cc / B;
    }
    for (int i = 0; i < nc; ++i)
        if (crit[i] > a && crit[i] < b) pts[np++] = crit[i];
    pts[np++] = b;
    for (int i = 0; i < np; ++i) {
        double v = poly_eval(c, pts[i]);
        if (v < *vmin) *vmin = v;
    }
    for (int i = 0; i + 1 < np; ++i) {
        double lo = pts[i], hi = pts[i + 1];
        double flo = poly_eval(c, lo), fhi = poly_eval(c, hi);
        if (flo == 0.0) return lo;
        if (flo > 0.0 && fhi <= 0.0) {
            if (fhi == 0.0 && hi == b) return hi;
            for (int it = 0; it < 200 && hi - lo > 1e-18; ++it) {
                double m = 0.5 * (lo + hi);
                double fm = poly_eval(c, m);
                if (fm > 0.0) lo = m; else hi = m;
            }
            return hi;
        }
        if (flo < 0.0) return lo; /* already inside (only at the first point) */
    }
    return NAN;
}

static void poly_mul_lin(const double p[4], double a0, double a1, double out[4]) {
    /* (p0 + p1 t + p2 t^2 + p3 t^3) (a0 + a1 t), truncated at degree 3 */
    double o[4];
    o[0] = p[0] * a0;
    o[1] = p[1] * a0 + p[0] * a1;
    o[2] = p[2] * a0 + p[1] * a1;
    o[3] = p[3] * a0 + p[2] * a1;
    memcpy(out, o, sizeof(o));
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* grid: trilinear field along the ray, cell by cell, as exact cubics */
static double grid_first_root(const or_object* o, double scale, const double q0[3], const double d[3], double tmax,
                              int* grazing) {
    double h[3], ta = 0.0, tb = tmax;
    for (int a = 0; a < 3; ++a) {
        h[a] = (o->hi[a] - o->lo[a]) / (double)(o->dims[a] - 1);
        if (d[a] == 0.0) {
            if (q0[a] < o->lo[a] || q0[a] > o->hi[a]) return NAN;
        } else {
            double t1 = (o->lo[a] - q0[a]) / d[a], t2 = (o->hi[a] - q0[a]) / d[a];
            if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
            if (t1 > ta) ta = t1;
            if (t2 < tb) tb = t2;
        }
    }
    if (!(ta < tb)) return NAN;
    /* parameters where the ray crosses a cell plane, plus the ends */
    int cap = 2;
    for (int a = 0; a < 3; ++a) cap += o->dims[a];
    double* ts = (double*)malloc(sizeof(double) * (size_t)cap);
    int nt = 0;
    ts[nt++] = ta;
    ts[nt++] = tb;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        for (int m = 0; m < o->dims[a]; ++m) {
            double t = (o->lo[a] + m * h[a] - q0[a]) / d[a];
            if (t > ta && t < tb) ts[nt++] = t;
        }
    }
    qsort(ts, (size_t)nt, sizeof(double), cmp_double);
    double vmin = INFINITY, root = NAN;
    for (int k = 0; k + 1 < nt && isnan(root); ++k) {
        double t0 = ts[k], t1 = ts[k + 1];
        if (!(t1 > t0)) continue;
        double tm = 0.5 * (t0 + t1);
        int ci[3];
        double x0[3], dx[3];
        for (int a = 0; a < 3; ++a) {
            double u = (q0[a] + tm * d[a] - o->lo[a]) / h[a];
            int i = (int)floor(u);
            if (i > o->dims[a] - 2) i = o->dims[a] - 2;
            if (i < 0) i = 0;
            ci[a] = i;
            x0[a] = (q0[a] - (o->lo[a] + i * h[a])) / h[a];
            dx[a] = d[a] / h[a];
        }
        double v[2][2][2];
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dxx = 0; dxx < 2; ++dxx) v[dz][dy][dxx] = grid_node(o, ci[0] + dxx, ci[1] + dy, ci[2] + dz);
        double a0 = v[0][0][0];
        double ax = v[0][0][1] - v[0][0][0], ay = v[0][1][0] - v[0][0][0], az = v[1][0][0] - v[0][0][0];
        double axy = v[0][1][1] - v[0][0][1] - v[0][1][0] + v[0][0][0];
        double axz = v[1][0][1] - v[0][0][1] - v[1][0][0] + v[0][0][0];
        double ayz = v[1][1][0] - v[0][1][0] - v[1][0][0] + v[0][0][0];
        double axyz = v[1][1][1] - v[0][1][1] - v[1][0][1] - v[1][1][0] + v[0][0][1] + v[0][1][0] + v[1][0][0] - v[0][0][0];
        double X[4] = {x0[0], dx[0], 0, 0}, Y[4] = {x0[1], dx[1], 0, 0}, Z[4] = {x0[2], dx[2], 0, 0};
        double XY[4], XZ[4], YZ[4], XYZ[4];
        poly_mul_lin(X, x0[1], dx[1], XY);
        poly_mul_lin(X, x0[2], dx[2], XZ);
        poly_mul_lin(Y, x0[2], dx[2], YZ);
        poly_mul_lin(XY, x0[2], dx[2], XYZ);
        double c[4];
        for (int i = 0; i < 4; ++i)
            c[i] = (i == 0 ? a0 : 0.0) + ax * X[i] + ay * Y[i] + az * Z[i] + axy * XY[i] + axz * XZ[i] + ayz * YZ[i] + axyz * XYZ[i];
        root = cubic_first_root(c, t0, t1, &vmin);
        if (!isnan(root)) {
            double slope = scale * poly_deriv(c, root);
            if (fabs(slope) < OR_GRAZE_SLOPE) *grazing = 1;
        }
    }
    free(ts);
    if (isnan(root) && scale * vmin < OR_GRAZE_GAP) *grazing = 1;
    return root;
}

static double sphere_first_root(double r, double scale, const double q0[3], const double d[3], double tmax, int* grazing) {
    double A = dot3(d, d), B = 2.0 * dot3(q0, d), Cc = dot3(q0, q0) - r * r;
    double disc = B * B - 4.0 * A * Cc;
    if (disc < 0.0) {
        /* closest approach of the line */
        double tc = -B / (2.0 * A);
        if (tc > 0.0 && tc < tmax) {
            double p[3] = {q0[0] + tc * d[0], q0[1] + tc * d[1], q0[2] + tc * d[2]};
            if (scale * (norm3(p) - r) < OR_GRAZE_GAP) *grazing = 1;
        }
        return NAN;
    }
    double t = (-B - sqrt(disc)) / (2.0 * A);
    if (t < 0.0 || t > tmax) return NAN;
    double p[3] = {q0[0] + t * d[0], q0[1] + t * d[1], q0[2] + t * d[2]};
    double slope = scale * dot3(p, d) / norm3(p);
    if (fabs(slope) < OR_GRAZE_SLOPE) *grazing = 1;
    return t;
}

static double box_first_root(const double hh[3], double scale, const double q0[3], const double d[3], double tmax,
                             int* grazing) {
    double ta = 0.0, tb = tmax;
    int enter_axis = -1;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (q0[a] < -hh[a] || q0[a] > hh[a]) return NAN;
        } else {
            double t1 = (-hh[a] - q0[a]) / d[a], t2 = (hh[a] - q0[a]) / d[a];
            if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
            if (t1 > ta) { ta = t1; enter_axis = a; }
            if (t2 < tb) tb = t2;
        }
    }
    if (!(ta <= tb)) return NAN;
    if (enter_axis >= 0 && fabs(scale * d[enter_axis]) < OR_GRAZE_SLOPE) *grazing = 1;
    return ta;
}

static double mesh_first_root(const or_object* o, double scale, const double q0[3], const double d[3], double tmax,
                              int* grazing) {
    double best = NAN, best_slope = 0.0;
    for (int32_t f = 0; f < o->n_faces; ++f) {
        double a[3], b[3], c[3], e1[3], e2[3], pv[3], tv[3], qv[3];
        vert(o->verts, o->faces[3 * f], a); vert(o->verts, o->faces[3 * f + 1], b); vert(o->verts, o->faces[3 * f + 2], c);
        sub3(b, a, e1); sub3(c, a, e2);
        cross3(d, e2, pv);
        double det = dot3(e1, pv);
        if (det == 0.0) continue;
        double inv = 1.0 / det;
        sub3(q0, a, tv);
        double u = dot3(tv, pv) * inv;
        if (u < 0.0 || u > 1.0) continue;
        cross3(tv, e1, qv);
        double v = dot3(d, qv) * inv;
        if (v < 0.0 || u + v > 1.0) continue;
        double t = dot3(e2, qv) * inv;
        if (t < 0.0 || t > tmax) continue;
        if (isnan(best) || t < best) {
            double n[3];
            cross3(e1, e2, n);
            best = t;
            best_slope = scale * dot3(d, n) / norm3(n);
        }
    }
    if (!isnan(best) && fabs(best_slope) < OR_GRAZE_SLOPE) *grazing = 1;
    return best;
}

/* the field a ray is traced through: the object's SDF (a learned SDF's
   fallback grid), world units */
static double ray_phi(const or_object* o, double scale, const double q0[3], const double d[3], double t) {
    double p[3] = {q0[0] + t * d[0], q0[1] + t * d[1], q0[2] + t * d[2]}, g[3];
    return scale * (o->kind == OR_NEURAL ? or_sdf_grid(o, p, g) : or_sdf_object(o, p, g));
}

/* A crossing after which the ray leaves the object again before it is
   OR_GRAZE_GAP deep (it skims the surface) is as ill-posed for a marching
   scheme as a near miss within OR_GRAZE_GAP: flag it.  Walks inside from the
   root in steps of max(1 um, |phi| / 2), which cannot pass the exit. */
static void flag_skim(const or_object* o, double scale, const double q0[3], const double d[3], double t,
                      double tmax, int* grazing) {
    double tt = t;
    for (int m = 0; m < 2000; ++m) {
        const double phi = ray_phi(o, scale, q0, d, tt);
        if (m > 0 && phi > 0.0) break;           /* out again */
        if (-phi >= OR_GRAZE_GAP) return;        /* a hit that goes deep */
        tt += fmax(1e-6, 0.5 * fabs(phi));
        if (tt > tmax) break;
    }
    *grazing = 1;
}

double or_ray_first_root(const or_object* o, double scale, const double q0[3], const double d[3], double tmax,
                         int* grazing) {
    double g[3];
    if (or_sdf_object(o, q0, g) <= 0.0) return 0.0;  /* the origin is inside: hit at once */
    double t;
    switch (o->kind) {
    case OR_SPHERE: t = sphere_first_root(o->radius, scale, q0, d, tmax, grazing); break;
    case OR_BOX: t = box_first_root(o->half, scale, q0, d, tmax, grazing); break;
    case OR_PLANE: {
        if (d[2] >= 0.0) return NAN;
        t = -q0[2] / d[2];
        if (fabs(scale * d[2]) < OR_GRAZE_SLOPE) *grazing = 1;
        return t <= tmax ? t : NAN;
    }
    case OR_MESH: t = mesh_first_root(o, scale, q0, d, tmax, grazing); break;
    case OR_GRID:
    case OR_NEURAL: t = grid_first_root(o, scale, q0, d, tmax, grazing); break;  /* neural: its fallback grid */
    default: return NAN;
    }
    if (!isnan(t) && !*grazing) flag_skim(o, scale, q0, d, t, tmax, grazing);
    return t;
}

/* ray directions of one probe in the link frame: ray 0 along the normal n,
   rays 1..n_rays-1 on a cone of half-angle `cone` around n at azimuths
   2 pi (k-1)/(n_rays-1) from the tangent u = n x z (n x x if n is along z) */
void or_prox_ray_dirs(const double n[3], int n_rays, double cone, double dirs[][3]) {
    double ez[3] = {0, 0, 1}, ex[3] = {1, 0, 0}, u[3], v[3];
    cross3(n, ez, u);
    if (norm3(u) < 1e-6) cross3(n, ex, u);
    double un = norm3(u);
    for (int a = 0; a < 3; ++a) u[a] /= un;
    cross3(n, u, v);
    for (int a = 0; a < 3; ++a) dirs[0][a] = n[a];
    for (int k = 1; k < n_rays; ++k) {
        double az = 2.0 * PI * (double)(k - 1) / (double)(n_rays - 1);
        for (int a = 0; a < 3; ++a)
            dirs[k][a] = cos(cone) * n[a] + sin(cone) * (cos(az) * u[a] + sin(az) * v[a]);
    }
}

/* Gaussian dilation kernel g(r) = exp(-lambda |r|^2) (Eq. 20) */
double or_marker_kernel_g(double lambda_d, double r2) { return exp(-lambda_d * r2); }

/* ======================================================================== */
/* Sensor formulas                                                           */
/* ======================================================================== */

/* ContactProbe, Eq. 3: on above eta_on, stays on above eta_off */
int or_schmitt(int prev, double d, double eta_on, double eta_off) {
    return (d > eta_on) || (prev && d > eta_off);
}

/* KinematicTaxel, Eqs. 7-9 in the sensor-link frame, with the Coulomb clamp
   on the tangential term: f_t = -k_t v_t min(1, mu |f_n| / (k_t |v_t|)).
   dw_dot_m is (omega_C - omega_L) . m.  d > 0 is required. */
void or_taxel_force(const or_params* P, double k, double mu, double d, const double x[3],
                    const double mbar[3], const double vrel[3], const double dw_dot_m,
                    double f[3], double tau[3]) {
    double s = pow(d, P->alpha);
    double vn_s = dot3(vrel, mbar);
    double vn[3], vt[3], fn[3], ft[3];
    for (int a = 0; a < 3; ++a) { vn[a] = vn_s * mbar[a]; vt[a] = vrel[a] - vn[a]; }
    for (int a = 0; a < 3; ++a) fn[a] = k * s * mbar[a] + P->c * s * vn[a];
    double vt_n = norm3(vt);
    double scale = 1.0;
    if (mu >= 0.0 && P->k_t * vt_n > 0.0) {
        double lim = mu * norm3(fn) / (P->k_t * vt_n);
        if (lim < 1.0) scale = lim;
    }
    for (int a = 0; a < 3; ++a) { ft[a] = -P->k_t * vt[a] * scale; f[a] = fn[a] + ft[a]; }
    double xf[3];
    cross3(x, f, xf);
    for (int a = 0; a < 3; ++a) tau[a] = xf[a] - P->k_omega * dw_dot_m * mbar[a];
}

/* L1-normalised 3x3 Gaussian of standard deviation sigma (lattice steps),
   w[(di+1)*3 + (dj+1)] for row offset di and column offset dj */
void or_crosstalk_weights(double sigma, double w[9]) {
    double s = 0.0;
    for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
            double e = exp(-(double)(di * di + dj * dj) / (2.0 * sigma * sigma));
            w[(di + 1) * 3 + (dj + 1)] = e;
            s += e;
        }
    for (int i = 0; i < 9; ++i) w[i] /= s;
}

static int group_gain_on(const or_noise_group* g) { return !(g->gain_lo == 1.0 && g->gain_hi == 1.0); }

/* ======================================================================== */
/* Reset: dead mask from the episode draw; state cleared (x_{-1}=0, xi=0,   */
/* drift 0, Schmitt off).                                                    */
/* ======================================================================== */
void or_reset(const or_scene* S, const uint8_t* env_mask, uint32_t episode, or_state* st) {
    int64_t T = S->taxel_offsets[S->n_envs];
    for (int32_t e = 0; e < S->n_envs; ++e) {
        if (env_mask && !env_mask[e]) continue;
        st->episode[e] = episode;
        for (int64_t i = S->taxel_offsets[e]; i < S->taxel_offsets[e + 1]; ++i) {
            uint64_t gid = (uint64_t)(S->taxel_gid0[e] + (i - S->taxel_offsets[e]));
            uint32_t w[4];
            philox_draw(S->params.seed, gid, episode, TAG_EPISODE, w);
            int dead = S->R[i] > 0.0f && bernoulli(w[0], S->params.p_dead);
            st->flags[i] = (uint8_t)(dead ? 2 : 0);
            for (int ch = 0; ch < OR_NCH; ++ch) {
                st->hyst_prev[(size_t)ch * T + i] = 0.0;
                st->hyst_xi[(size_t)ch * T + i] = 0.0;
                st->drift[(size_t)ch * T + i] = 0.0;
            }
            if (st->ring) {
                const int32_t K = S->params.delay + S->params.jitter + 1;
                for (int32_t k = 0; k < K * OR_RING_CH; ++k) st->ring[(size_t)k * T + i] = 0.0;
            }
        }
    }
}

/* The read delay of env e at this step: delay + j, j uniform on {0..jitter}
   from the top 24 bits of Philox word 0 at (env id, step, TAG_JITTER), as an
   integer product (exact on every side). */
int32_t or_read_delay(const or_params* P, uint32_t env_gid, uint32_t step) {
    if (P->jitter <= 0) return P->delay;
    uint32_t w[4];
    philox_draw(P->seed, env_gid, step, TAG_JITTER, w);
    return P->delay + (int32_t)(((uint64_t)(w[0] >> 8) * (uint64_t)(P->jitter + 1)) >> 24);
}

/* one noise group applied to one channel value after the clean reading:
   gain and hysteresis (Eqs. 27, 29-30).  Updates the hysteresis state. */
static double gain_hysteresis(const or_noise_group* g, double dt, double gain, double clean,
                              double* prev, double* xi) {
    double x = gain * clean;
    if (g->beta == 0.0) return x;
    double a = exp(-dt / g->tau);
    double xi_t = a * (*xi) + (x - *prev);
    *xi = xi_t;
    *prev = x;
    return x + g->beta * xi_t;
}

/* base noise (Eq. 25) then dead override (Eq. 28): + b + n_t + d_t,
   quantise, stuck value when dead */
static double base_noise(const or_noise_group* g, double z, double white_n, double drift_n,
                         double* drift, int dead, double stuck_u) {
    if (g->sigma_rw != 0.0) *drift += g->sigma_rw * drift_n;
    double y = z + g->bias + g->sigma_white * white_n + (g->sigma_rw != 0.0 ? *drift : 0.0);
    if (g->quant > 0.0) y = g->quant * nearbyint(y / g->quant);
    if (dead) y = g->stuck_lo + (g->stuck_hi - g->stuck_lo) * stuck_u;
    return y;
}

/* A learned-SDF object's network answers where its fallback grid puts the
   probe within this distance (m) of contact (phi_grid <= R + band). */
#define OR_NEURAL_BAND 1e-3

/* ======================================================================== */
/* One step of the whole sensor pipeline for every env of the (sub)scene.   */
/* ======================================================================== */
static void env_step(const or_scene* S, const or_inputs* in, or_state* st, or_outputs* out, int32_t e) {
    const or_params* P = &S->params;
    const int32_t L = S->max_links;
    const int64_t T = S->taxel_offsets[S->n_envs];
    const int64_t t0 = S->taxel_offsets[e], t1 = S->taxel_offsets[e + 1];
    const int64_t n = t1 - t0;

    double k = P->k, mu = P->mu, scale = 1.0;
    if (P->dr_on) {
        double v[3];
        or_dr_draw(P, (uint32_t)S->env_gid[e], in->step, v);
        mu = v[0]; k = v[1]; scale = v[2];
    } else if (in->env_params) {
        mu = in->env_params[3 * e]; k = in->env_params[3 * e + 1]; scale = in->env_params[3 * e + 2];
    }
    const or_object* obj = &S->objects[in->obj_id[e]];

    /* object pose and velocity */
    double pC0[3], qC0[4], vC[3], wC[3], pC[3], RC[9];
    for (int a = 0; a < 3; ++a) pC0[a] = in->obj_pose[7 * e + a];
    for (int a = 0; a < 4; ++a) qC0[a] = in->obj_pose[7 * e + 3 + a];
    for (int a = 0; a < 3; ++a) { vC[a] = in->obj_vel[6 * e + a]; wC[a] = in->obj_vel[6 * e + 3 + a]; }
    or_advance_pose(pC0, qC0, vC, wC, in->pose_dt, pC, RC);

    /* per-taxel scratch in clean order */
    double* hx = (double*)calloc((size_t)n * 6, sizeof(double)); /* x~ of force/torque after hysteresis */
    double* fclean = (double*)calloc((size_t)n * 6, sizeof(double));  /* force entering the noise chain */
    int* active = (int*)calloc((size_t)n, sizeof(int));

    uint32_t episode = st->episode[e];
    int64_t j = t0;
    for (int32_t l = 0; l < L; ++l) {
        int32_t nl = S->link_rows[e * L + l] * S->link_cols[e * L + l];
        if (nl == 0) continue;
        const float* lp = in->link_pose + ((size_t)e * L + l) * 7;
        const float* lv = in->link_vel + ((size_t)e * L + l) * 6;
        double pL0[3], qL0[4], vL[3], wL[3], pL[3], RL[9];
        for (int a = 0; a < 3; ++a) pL0[a] = lp[a];
        for (int a = 0; a < 4; ++a) qL0[a] = lp[3 + a];
        for (int a = 0; a < 3; ++a) { vL[a] = lv[a]; wL[a] = lv[3 + a]; }
        or_advance_pose(pL0, qL0, vL, wL, in->pose_dt, pL, RL);

        for (int32_t m_ = 0; m_ < nl; ++m_, ++j) {
            int64_t jl = j - t0;
            double R = S->R[j];
            if (!(R > 0.0)) continue; /* inactive filler: every output is zero */
            active[jl] = 1;
            uint64_t gid = (uint64_t)(S->taxel_gid0[e] + jl);
            double x[3] = {S->x[j], S->y[j], S->z[j]};
            /* Eq. 1: world position of the probe */
            double q[3];
            matvec(RL, x, q);
            for (int a = 0; a < 3; ++a) q[a] += pL[a];
            /* object frame, scaled: q^ = R_C^T (q - p_C) / s */
            double dq[3], qh[3], go[3], m[3], mbar[3];
            sub3(q, pC, dq);
            matTvec(RC, dq, qh);
            for (int a = 0; a < 3; ++a) qh[a] /= scale;
            double phi;
            if (obj->kind == OR_NEURAL) {
                /* a learned SDF answers within 1 mm of contact as its
                   fallback grid sees it; farther out the grid answers */
                phi = scale * or_sdf_grid(obj, qh, go);
                if (!(phi > R + OR_NEURAL_BAND)) phi = scale * or_sdf_object(obj, qh, go);
            } else if (obj->kind == OR_MESH && P->depth_backend == 1) {
                /* raycast backend: the deepest penetration over the
                   triangles within R (object frame, world units), with that
                   triangle's normal; phi = R - depth (R when none is near) */
                double qo[3], nl_[3] = {S->nx[j], S->ny[j], S->nz[j]}, uw[3], uo[3], rpen;
                int32_t face;
                for (int a = 0; a < 3; ++a) qo[a] = qh[a] * scale;
                matvec(RL, nl_, uw);
                matTvec(RC, uw, uo);
                const double pen = or_raycast_depth(obj->verts, obj->faces, obj->n_faces, scale, qo, uo, R, go, &face,
                                                    &rpen);
                phi = R - pen;
                if (out->depth_tie)
                    out->depth_tie[j] = (uint8_t)(face >= 0 && raycast_tie(obj->verts, obj->faces, obj->n_faces, scale,
                                                                           qo, R, pen, face, go));
            } else {
                phi = scale * or_sdf_object(obj, qh, go);
            }
            matvec(RC, go, m);          /* world normal */
            matTvec(RL, m, mbar);       /* link-frame normal */
            /* Eq. 2 */
            double d = R - phi;
            if (d < 0.0) d = 0.0;
            out->dist[j] = phi - R;
            /* Eq. 3 */
            int prev = st->flags[j] & 1;
            int y = or_schmitt(prev, d, P->eta_on, P->eta_off);
            int dead = (st->flags[j] >> 1) & 1;
            /* the noisy readout's depth: with probe-radius noise, from the
               perturbed radius, with its own Schmitt state (flag bit 2, the
               last noisy contact bit); without it, the clean depth */
            double dn = d;
            int yn = y && !dead;
            if (P->rho > 0.0) {
                uint32_t wr[4];
                philox_draw(P->seed, gid, in->step, TAG_RADIUS, wr);
                double Rn = R + (double)radius_eps(P->rho, wr[0]);
                if (Rn < 0.0) Rn = 0.0;
                dn = Rn - phi;
                if (dn < 0.0) dn = 0.0;
                int ys = or_schmitt((st->flags[j] >> 2) & 1, dn, P->eta_on, P->eta_off);
                yn = ys && !dead;
            }
            st->flags[j] = (uint8_t)((st->flags[j] & 2u) | (unsigned)y | ((unsigned)yn << 2));
            out->contact_clean[j] = (uint8_t)y;
            out->contact_noisy[j] = (uint8_t)yn;
            out->depth_clean[j] = d;

            double f[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
            double fn[3] = {0, 0, 0}, taun[3] = {0, 0, 0};  /* the force the noise chain starts from */
            if (d > 0.0 || dn > 0.0) {
                /* Eqs. 4-6: point velocities and link-frame relative velocity */
                double rC[3], rL[3], vCq[3], vLq[3], tmp[3], vrel[3];
                sub3(q, pC, rC); sub3(q, pL, rL);
                cross3(wC, rC, tmp);
                for (int a = 0; a < 3; ++a) vCq[a] = vC[a] + tmp[a];
                cross3(wL, rL, tmp);
                for (int a = 0; a < 3; ++a) vLq[a] = vL[a] + tmp[a];
                sub3(vCq, vLq, tmp);
                matTvec(RL, tmp, vrel);
                double dw[3];
                sub3(wC, wL, dw);
                if (d > 0.0) or_taxel_force(P, k, mu, d, x, mbar, vrel, dot3(dw, m), f, tau);
                if (P->rho > 0.0) {
                    if (dn > 0.0) or_taxel_force(P, k, mu, dn, x, mbar, vrel, dot3(dw, m), fn, taun);
                } else {
                    for (int a = 0; a < 3; ++a) { fn[a] = f[a]; taun[a] = tau[a]; }
                }
            }
            for (int a = 0; a < 3; ++a) { fclean[jl * 6 + a] = fn[a]; fclean[jl * 6 + 3 + a] = taun[a]; }
            for (int a = 0; a < 3; ++a) { out->ft_clean[(size_t)a * T + j] = f[a]; out->ft_clean[(size_t)(3 + a) * T + j] = tau[a]; }
            if (st->ring) {
                /* read delay: this step's noisy-chain input goes into the
                   ring, the chain reads the one from rd steps earlier (the
                   reset state, 0, before the episode's first steps) */
                const uint32_t K = (uint32_t)(P->delay + P->jitter + 1);
                const uint32_t rd = (uint32_t)or_read_delay(P, (uint32_t)S->env_gid[e], in->step);
                double* w_ = st->ring + (size_t)(in->step % K) * OR_RING_CH * T;
                const double* r_ = st->ring + (size_t)((in->step % K + K - rd) % K) * OR_RING_CH * T;
                w_[j] = dn;
                for (int c = 0; c < 6; ++c) w_[(size_t)(1 + c) * T + j] = fclean[jl * 6 + c];
                w_[(size_t)7 * T + j] = (double)(P->rho > 0.0 ? ((st->flags[j] >> 2) & 1) : y);
                dn = r_[j];
                for (int c = 0; c < 6; ++c) fclean[jl * 6 + c] = r_[(size_t)(1 + c) * T + j];
                out->contact_noisy[j] = (uint8_t)(r_[(size_t)7 * T + j] != 0.0 && !dead);
            }

            /* noise: per-probe gains for this episode */
            uint32_t we[4];
            philox_draw(P->seed, gid, episode, TAG_EPISODE, we);
            double gain_d = group_gain_on(&P->depth) ? P->depth.gain_lo + (P->depth.gain_hi - P->depth.gain_lo) * or_uniform(we[1]) : 1.0;
            double gain_f = group_gain_on(&P->ft) ? P->ft.gain_lo + (P->ft.gain_hi - P->ft.gain_lo) * or_uniform(we[2]) : 1.0;
            /* depth: gain, hysteresis, base noise, dead */
            double hd = gain_hysteresis(&P->depth, P->dt, gain_d, dn, &st->hyst_prev[j], &st->hyst_xi[j]);
            double zs[4];
            philox_normals(P->seed, gid, in->step, TAG_SCALAR, zs);
            uint32_t wst[4];
            philox_draw(P->seed, gid, episode, TAG_STUCK, wst);
            out->depth_noisy[j] = base_noise(&P->depth, hd, zs[1], zs[0], &st->drift[j], dead, or_uniform(wst[0]));
            /* force/torque: gain and hysteresis now, crosstalk after the link */
            for (int c = 0; c < 6; ++c) {
                size_t si = (size_t)(1 + c) * T + j;
                hx[jl * 6 + c] = gain_hysteresis(&P->ft, P->dt, gain_f, fclean[jl * 6 + c], &st->hyst_prev[si], &st->hyst_xi[si]);
            }
            /* proximity (rays from the probe centre, object frame, scaled) */
            if (P->prox_rays > 0) {
                double nl_[3] = {S->nx[j], S->ny[j], S->nz[j]};
                double dirs[64][3];
                or_prox_ray_dirs(nl_, P->prox_rays, P->prox_cone, dirs);
                double reading = 0.0;
                int grazing = 0;
                for (int k = 0; k < P->prox_rays; ++k) {
                    double dw[3], dobj[3];
                    matvec(RL, dirs[k], dw);
                    matTvec(RC, dw, dobj);
                    for (int a = 0; a < 3; ++a) dobj[a] /= scale;
                    double t = or_ray_first_root(obj, scale, qh, dobj, P->prox_range, &grazing);
                    if (!isnan(t)) reading += 1.0 - t / P->prox_range;
                }
                reading /= (double)P->prox_rays;
                out->prox_clean[j] = reading;
                out->prox_grazing[j] = (uint8_t)grazing;
                double gain_p = group_gain_on(&P->prox) ? P->prox.gain_lo + (P->prox.gain_hi - P->prox.gain_lo) * or_uniform(we[3]) : 1.0;
                size_t sp = (size_t)7 * T + j;
                double hp = gain_hysteresis(&P->prox, P->dt, gain_p, reading, &st->hyst_prev[sp], &st->hyst_xi[sp]);
                out->prox_noisy[j] = base_noise(&P->prox, hp, zs[3], zs[2], &st->drift[sp], dead, or_uniform(wst[2]));
            }
        }
    }

    /* Eq. 31: 3x3 crosstalk on each link lattice, then base noise and dead */
    double W[9];
    or_crosstalk_weights(P->xt_sigma, W);
    int64_t lbase = 0;
    for (int32_t l = 0; l < L; ++l) {
        int32_t rows = S->link_rows[e * L + l], cols = S->link_cols[e * L + l];
        int wrap = S->link_wrap[e * L + l];
        int32_t nl = rows * cols;
        if (nl == 0) continue;
        double Fc[3] = {0, 0, 0}, Tc[3] = {0, 0, 0}, Fn[3] = {0, 0, 0}, Tn[3] = {0, 0, 0};
        double Ac[3] = {0, 0, 0}, An[3] = {0, 0, 0};
        int32_t cnt_c = 0, cnt_n = 0;
        for (int32_t r = 0; r < rows; ++r) {
            for (int32_t cc = 0; cc < cols; ++cc) {
                int64_t jl = lbase + (int64_t)r * cols + cc;
                int64_t jg = t0 + jl;
                if (!active[jl]) {
                    if (P->prox_rays > 0) { out->prox_clean[jg] = 0.0; out->prox_noisy[jg] = 0.0; out->prox_grazing[jg] = 0; }
                    out->depth_noisy[jg] = 0.0; out->dist[jg] = 0.0;
                    out->depth_clean[jg] = 0.0;
                    out->contact_clean[jg] = 0; out->contact_noisy[jg] = 0;
                    for (int c = 0; c < 6; ++c) { out->ft_clean[(size_t)c * T + jg] = 0.0; out->ft_noisy[(size_t)c * T + jg] = 0.0; }
                    continue;
                }
                uint64_t gid = (uint64_t)(S->taxel_gid0[e] + jl);
                double z[6];
                for (int c = 0; c < 6; ++c) {
                    double v = hx[jl * 6 + c];
                    if (P->chi != 0.0) {
                        double conv = 0.0;
                        for (int di = -1; di <= 1; ++di) {
                            int32_t rr = r + di;
                            if (rr < 0 || rr >= rows) continue;
                            for (int dj = -1; dj <= 1; ++dj) {
                                int32_t c2 = cc + dj;
                                if (wrap) c2 = (c2 + cols) % cols;
                                else if (c2 < 0 || c2 >= cols) continue;
                                conv += W[(di + 1) * 3 + (dj + 1)] * hx[(lbase + (int64_t)rr * cols + c2) * 6 + c];
                            }
                        }
                        v = (1.0 - P->chi) * v + P->chi * conv;
                    }
                    z[c] = v;
                }
                double nA[4], nB[4], nC[4];
                philox_normals(P->seed, gid, in->step, TAG_FT_A, nA);
                philox_normals(P->seed, gid, in->step, TAG_FT_B, nB);
                philox_normals(P->seed, gid, in->step, TAG_FT_C, nC);
                double drift_n[6] = {nA[0], nA[1], nA[2], nA[3], nB[0], nB[1]};
                double white_n[6] = {nB[2], nB[3], nC[0], nC[1], nC[2], nC[3]};
                uint32_t wst[4];
                philox_draw(P->seed, gid, st->episode[e], TAG_STUCK, wst);
                int dead = (st->flags[jg] >> 1) & 1;
                for (int c = 0; c < 6; ++c) {
                    size_t si = (size_t)(1 + c) * T + jg;
                    out->ft_noisy[(size_t)c * T + jg] = base_noise(&P->ft, z[c], white_n[c], drift_n[c], &st->drift[si], dead, or_uniform(wst[1]));
                }
                /* per-link sums (clean and noisy) and agg_force (Eq. 32) */
                for (int a = 0; a < 3; ++a) {
                    Fc[a] += out->ft_clean[(size_t)a * T + jg];
                    Tc[a] += out->ft_clean[(size_t)(3 + a) * T + jg];
                    Fn[a] += out->ft_noisy[(size_t)a * T + jg];
                    Tn[a] += out->ft_noisy[(size_t)(3 + a) * T + jg];
                }
                double nrm[3] = {S->nx[jg], S->ny[jg], S->nz[jg]};
                for (int a = 0; a < 3; ++a) {
                    Ac[a] += out->depth_clean[jg] * nrm[a];
                    An[a] += out->depth_noisy[jg] * nrm[a];
                }
                cnt_c += out->contact_clean[jg];
                cnt_n += out->contact_noisy[jg];
            }
        }
        double* rec = out->link_sums + ((size_t)e * L + l) * OR_LINK_REC;
        for (int a = 0; a < 3; ++a) {
            rec[a] = Fc[a]; rec[3 + a] = Tc[a]; rec[6 + a] = Fn[a]; rec[9 + a] = Tn[a];
            /* 1e4 * P_ZYX: reversed axis order */
            rec[12 + a] = 1e4 * Ac[2 - a];
            rec[15 + a] = 1e4 * An[2 - a];
        }
        out->link_counts[((size_t)e * L + l) * 2] = cnt_c;
        out->link_counts[((size_t)e * L + l) * 2 + 1] = cnt_n;
        lbase += nl;
    }
    /* absent links: zero records */
    for (int32_t l = 0; l < L; ++l) {
        if (S->link_rows[e * L + l] * S->link_cols[e * L + l] != 0) continue;
        double* rec = out->link_sums + ((size_t)e * L + l) * OR_LINK_REC;
        for (int a = 0; a < OR_LINK_REC; ++a) rec[a] = 0.0;
        out->link_counts[((size_t)e * L + l) * 2] = 0;
        out->link_counts[((size_t)e * L + l) * 2 + 1] = 0;
    }
    free(hx); free(fclean); free(active);
}

int or_step(const or_scene* S, const or_inputs* in, or_state* st, or_outputs* out, int32_t threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t e = 0; e < S->n_envs; ++e) env_step(S, in, st, out, e);
    return 0;
}

/* ======================================================================== */
/* ElastomerTaxel dilation (Eqs. 18-21) on planar marker pads: marker depth  */
/* h_i = max(0, -phi(q_i)) (no radius), then for each marker j the sum over */
/* sources i within `radius` markers of s_d (r_ij w_ij + n h_i^alpha g),   */
/* w_ij = h_i (c g / g_bar + (1 - c) rho / rho_bar), r_ij = Pi_n(x_j - x_i). */
/* ======================================================================== */
static void env_markers(const or_scene* S, const or_pads* pads, const or_inputs* in, double* u, double* h_out, int32_t e) {
    const int32_t L = S->max_links, P = pads->pads_per_env, M = pads->rows * pads->cols;
    double scale = in->env_params ? in->env_params[3 * e + 2] : 1.0;
    if (S->params.dr_on) {
        double v[3];
        or_dr_draw(&S->params, (uint32_t)S->env_gid[e], in->step, v);
        scale = v[2];
    }
    const or_object* obj = &S->objects[in->obj_id[e]];
    double pC0[3], qC0[4], vC[3], wC[3], pC[3], RC[9];
    for (int a = 0; a < 3; ++a) pC0[a] = in->obj_pose[7 * e + a];
    for (int a = 0; a < 4; ++a) qC0[a] = in->obj_pose[7 * e + 3 + a];
    for (int a = 0; a < 3; ++a) { vC[a] = in->obj_vel[6 * e + a]; wC[a] = in->obj_vel[6 * e + 3 + a]; }
    or_advance_pose(pC0, qC0, vC, wC, in->pose_dt, pC, RC);
    const double gbar = exp(-0.5) / sqrt(2.0 * pads->lambda_d);
    const double rbar = 1.0 / (2.0 * pads->eps);
    double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    double* hs = (double*)malloc(sizeof(double) * (size_t)M);
    for (int32_t p = 0; p < P; ++p) {
        int32_t l = pads->pad_link[e * P + p];
        const float* fr = pads->pad_frame + ((size_t)e * P + p) * 9;
        double o[3] = {fr[0], fr[1], fr[2]}, n[3] = {fr[3], fr[4], fr[5]}, tu[3] = {fr[6], fr[7], fr[8]}, tv[3];
        cross3(n, tu, tv);
        const float* lp = in->link_pose + ((size_t)e * L + l) * 7;
        const float* lv = in->link_vel + ((size_t)e * L + l) * 6;
        double pL0[3], qL0[4], vL[3], wL[3], pL[3], RL[9];
        for (int a = 0; a < 3; ++a) pL0[a] = lp[a];
        for (int a = 0; a < 4; ++a) qL0[a] = lp[3 + a];
        for (int a = 0; a < 3; ++a) { vL[a] = lv[a]; wL[a] = lv[3 + a]; }
        or_advance_pose(pL0, qL0, vL, wL, in->pose_dt, pL, RL);
        for (int32_t m = 0; m < M; ++m) {
            int32_t ra = m / pads->cols, cb = m % pads->cols;
            double sa = (ra - 0.5 * (pads->rows - 1)) * pads->pitch, sb = (cb - 0.5 * (pads->cols - 1)) * pads->pitch;
            double x[3], q[3], dq[3], qh[3], g[3];
            for (int a = 0; a < 3; ++a) x[a] = o[a] + sa * tu[a] + sb * tv[a];
            for (int a = 0; a < 3; ++a) xs[3 * m + a] = x[a];
            matvec(RL, x, q);
            for (int a = 0; a < 3; ++a) q[a] += pL[a];
            sub3(q, pC, dq);
            matTvec(RC, dq, qh);
            for (int a = 0; a < 3; ++a) qh[a] /= scale;
            /* a learned SDF's markers read its fallback grid, as its proximity rays do */
            double phi = scale * (obj->kind == OR_NEURAL ? or_sdf_grid(obj, qh, g) : or_sdf_object(obj, qh, g));
            hs[m] = phi < 0.0 ? -phi : 0.0;
            if (h_out) h_out[((size_t)e * P + p) * M + m] = hs[m];
        }
        for (int32_t j = 0; j < M; ++j) {
            int32_t rj = j / pads->cols, cj = j % pads->cols;
            double acc[3] = {0, 0, 0};
            for (int32_t di = -pads->radius; di <= pads->radius; ++di)
                for (int32_t dj = -pads->radius; dj <= pads->radius; ++dj) {
                    int32_t ri = rj + di, ci = cj + dj;
                    if (ri < 0 || ri >= pads->rows || ci < 0 || ci >= pads->cols) continue;
                    int32_t i = ri * pads->cols + ci;
                    double h = hs[i];
                    if (h == 0.0) continue;
                    double dx[3], r[3];
                    sub3(&xs[3 * j], &xs[3 * i], dx);
                    double dn = dot3(dx, n);
                    for (int a = 0; a < 3; ++a) r[a] = dx[a] - dn * n[a];
                    double r2 = dot3(r, r);
                    double gk = or_marker_kernel_g(pads->lambda_d, r2);
                    double rho = 1.0 / (r2 + pads->eps * pads->eps);
                    double w = h * (pads->c * gk / gbar + (1.0 - pads->c) * rho / rbar);
                    double hn = pow(h, pads->alpha) * gk;
                    for (int a = 0; a < 3; ++a) acc[a] += pads->s_d * (r[a] * w + n[a] * hn);
                }
            double* uo = u + (((size_t)e * P + p) * M + j) * 3;
            uo[0] = dot3(acc, n);
            uo[1] = dot3(acc, tu);
            uo[2] = dot3(acc, tv);
        }
    }
    free(xs);
    free(hs);
}

/* Point-cloud ProximityTaxel (Appendix A "ProximityTaxel"): the env's
   object is tracked by its surface points p_i; taxel j at q_j with normal a_j
   and sensing radius R collects P_ij = R - |p_i - q_j| from every point inside
   its sphere, the point's velocity relative to the taxel's with the normal
   component removed (v_t), and reports in the link frame
   f = k rho sum P a + ks rho sum P v_t,  tau = k rho sum P (p - q) x a,
   rho = density / max(N, 1).  Every point is tested (brute force). */
static void env_pc_prox(const or_scene* S, const or_pcprox* pc, const or_inputs* in, double* ft, int32_t e) {
    const int32_t L = S->max_links;
    const int64_t T = S->taxel_offsets[S->n_envs];
    double scale = in->env_params ? in->env_params[3 * e + 2] : 1.0;
    if (S->params.dr_on) {
        double v[3];
        or_dr_draw(&S->params, (uint32_t)S->env_gid[e], in->step, v);
        scale = v[2];
    }
    int32_t oid = in->obj_id[e];
    if (oid < 0) oid = 0;
    if (oid > S->n_objects - 1) oid = S->n_objects - 1;
    const float* pts = pc->cloud + 3 * pc->cloud_off[oid];
    const int64_t N = pc->cloud_off[oid + 1] - pc->cloud_off[oid];
    const double rho = pc->density / (double)(N > 1 ? N : 1);
    const double R = pc->radius;
    double pC0[3], qC0[4], vC[3], wC[3], pC[3], RC[9];
    for (int a = 0; a < 3; ++a) pC0[a] = in->obj_pose[7 * e + a];
    for (int a = 0; a < 4; ++a) qC0[a] = in->obj_pose[7 * e + 3 + a];
    for (int a = 0; a < 3; ++a) { vC[a] = in->obj_vel[6 * e + a]; wC[a] = in->obj_vel[6 * e + 3 + a]; }
    or_advance_pose(pC0, qC0, vC, wC, in->pose_dt, pC, RC);
    /* world positions and velocities of the tracked points */
    double* pw = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double* vw = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        double ph[3] = {scale * pts[3 * i], scale * pts[3 * i + 1], scale * pts[3 * i + 2]}, r[3], w[3];
        matvec(RC, ph, r);
        for (int a = 0; a < 3; ++a) pw[3 * i + a] = pC[a] + r[a];
        cross3(wC, r, w);
        for (int a = 0; a < 3; ++a) vw[3 * i + a] = vC[a] + w[a];
    }
    int64_t j = S->taxel_offsets[e];
    for (int32_t l = 0; l < L; ++l) {
        int32_t nl = S->link_rows[e * L + l] * S->link_cols[e * L + l];
        if (nl == 0) continue;
        const float* lp = in->link_pose + ((size_t)e * L + l) * 7;
        const float* lv = in->link_vel + ((size_t)e * L + l) * 6;
        double pL0[3], qL0[4], vL[3], wL[3], pL[3], RL[9];
        for (int a = 0; a < 3; ++a) pL0[a] = lp[a];
        for (int a = 0; a < 4; ++a) qL0[a] = lp[3 + a];
        for (int a = 0; a < 3; ++a) { vL[a] = lv[a]; wL[a] = lv[3 + a]; }
        or_advance_pose(pL0, qL0, vL, wL, in->pose_dt, pL, RL);
        for (int32_t m_ = 0; m_ < nl; ++m_, ++j) {
            double fw[3] = {0, 0, 0}, tw[3] = {0, 0, 0};
            if (S->R[j] > 0.0) {
                double x[3] = {S->x[j], S->y[j], S->z[j]}, nl_[3] = {S->nx[j], S->ny[j], S->nz[j]};
                double q[3], a_[3], rq[3], vt_[3], vtax[3];
                matvec(RL, x, rq);
                for (int a = 0; a < 3; ++a) q[a] = pL[a] + rq[a];
                matvec(RL, nl_, a_);
                cross3(wL, rq, vt_);
                for (int a = 0; a < 3; ++a) vtax[a] = vL[a] + vt_[a];
                for (int64_t i = 0; i < N; ++i) {
                    double dlt[3];
                    sub3(&pw[3 * i], q, dlt);
                    double dist = sqrt(dot3(dlt, dlt));
                    if (!(dist < R)) continue;
                    double P = R - dist, vr[3], vt[3], c[3];
                    sub3(&vw[3 * i], vtax, vr);
                    double vn = dot3(vr, a_);
                    for (int a = 0; a < 3; ++a) vt[a] = vr[a] - a_[a] * vn;
                    cross3(dlt, a_, c);
                    for (int a = 0; a < 3; ++a) {
                        fw[a] += pc->k * rho * P * a_[a] + pc->ks * rho * P * vt[a];
                        tw[a] += pc->k * rho * P * c[a];
                    }
                }
            }
            double fl[3], tl[3];
            matTvec(RL, fw, fl);
            matTvec(RL, tw, tl);
            for (int a = 0; a < 3; ++a) {
                ft[(size_t)a * T + j] = fl[a];
                ft[(size_t)(3 + a) * T + j] = tl[a];
            }
        }
    }
    free(pw);
    free(vw);
}

/* ElastomerTaxel shear anchors (Eqs. 19-20).  For every pad: each tracked
   point of the env object is taken into the sensor frame, z = (z_t, z_b, z_n)
   in the pad's tangent, bitangent and normal; its elastomer SDF is that of
   the box under the pad; an unanchored point whose SDF is below -eta_enter
   anchors at e = (z_t, z_b), an anchored one whose SDF is above +eta_exit
   lets go.  Every anchored point with penetration h = max(0, -SDF) > 0 then
   moves marker j (pad position x_j = (a_j, b_j, 0)) by
   s_s Pi_n(z - e) h exp(-lambda_s |Pi_n(x_j - z)|^2). */
static void env_shear(const or_scene* S, const or_pads* pads, const or_shear* sh, const or_inputs* in,
                      double* anchors, int32_t* anchor_obj, double* u, int32_t* n_anchored, double* margin,
                      double* drag, int32_t e) {
    const int32_t L = S->max_links, P = pads->pads_per_env, M = pads->rows * pads->cols;
    double scale = in->env_params ? in->env_params[3 * e + 2] : 1.0;
    if (S->params.dr_on) {
        double v[3];
        or_dr_draw(&S->params, (uint32_t)S->env_gid[e], in->step, v);
        scale = v[2];
    }
    int32_t oid = in->obj_id[e];
    if (oid < 0) oid = 0;
    if (oid > S->n_objects - 1) oid = S->n_objects - 1;
    const float* pts = sh->cloud + 3 * sh->cloud_off[oid];
    const int64_t N = sh->cloud_off[oid + 1] - sh->cloud_off[oid];
    double pC0[3], qC0[4], vC[3], wC[3], pC[3], RC[9];
    for (int a = 0; a < 3; ++a) pC0[a] = in->obj_pose[7 * e + a];
    for (int a = 0; a < 4; ++a) qC0[a] = in->obj_pose[7 * e + 3 + a];
    for (int a = 0; a < 3; ++a) { vC[a] = in->obj_vel[6 * e + a]; wC[a] = in->obj_vel[6 * e + 3 + a]; }
    or_advance_pose(pC0, qC0, vC, wC, in->pose_dt, pC, RC);
    /* the elastomer box: centre (0, 0, -thickness / 2) in pad coordinates */
    const double half[3] = {0.5 * pads->rows * pads->pitch, 0.5 * pads->cols * pads->pitch, 0.5 * sh->thickness};
    double* con = (double*)malloc(sizeof(double) * 4 * (size_t)(N > 0 ? N : 1));
    for (int32_t p = 0; p < P; ++p) {
        const size_t ep = (size_t)e * P + p;
        double* an = anchors + ep * (size_t)sh->n_max * 2;
        if (anchor_obj[ep] != oid) {
            for (int64_t i = 0; i < 2 * sh->n_max; ++i) an[i] = NAN;
            anchor_obj[ep] = oid;
        }
        int32_t l = pads->pad_link[ep];
        const float* fr = pads->pad_frame + ep * 9;
        double o[3] = {fr[0], fr[1], fr[2]}, n[3] = {fr[3], fr[4], fr[5]}, tu[3] = {fr[6], fr[7], fr[8]}, tv[3];
        cross3(n, tu, tv);
        const float* lp = in->link_pose + ((size_t)e * L + l) * 7;
        const float* lv = in->link_vel + ((size_t)e * L + l) * 6;
        double pL0[3], qL0[4], vL[3], wL[3], pL[3], RL[9];
        for (int a = 0; a < 3; ++a) pL0[a] = lp[a];
        for (int a = 0; a < 4; ++a) qL0[a] = lp[3 + a];
        for (int a = 0; a < 3; ++a) { vL[a] = lv[a]; wL[a] = lv[3 + a]; }
        or_advance_pose(pL0, qL0, vL, wL, in->pose_dt, pL, RL);
        int32_t count = 0;
        int64_t K = 0;
        double mg = INFINITY, dg = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double ph[3] = {scale * pts[3 * i], scale * pts[3 * i + 1], scale * pts[3 * i + 2]}, w[3], d[3], xl[3], r[3];
            matvec(RC, ph, w);
            for (int a = 0; a < 3; ++a) w[a] += pC[a];
            sub3(w, pL, d);
            matTvec(RL, d, xl);
            sub3(xl, o, r);
            const double z[3] = {dot3(r, tu), dot3(r, tv), dot3(r, n)};
            const double zb[3] = {z[0], z[1], z[2] + half[2]};
            double g[3];
            const double sdf = or_sdf_box(half, zb, g);
            int anchored = !isnan(an[2 * i]);
            /* the decision this point faces: entering if free, leaving if anchored */
            mg = fmin(mg, anchored ? fabs(sdf - sh->eta_exit) : fabs(sdf + sh->eta_enter));
            if (!anchored && sdf < -sh->eta_enter) {
                an[2 * i] = z[0];
                an[2 * i + 1] = z[1];
                anchored = 1;
            } else if (anchored && sdf > sh->eta_exit) {
                an[2 * i] = an[2 * i + 1] = NAN;
                anchored = 0;
            }
            count += anchored;
            const double h = sdf < 0.0 ? -sdf : 0.0;
            if (anchored && sdf < 1e-6)
                dg += sh->s_s * (h + hypot(z[0] - an[2 * i], z[1] - an[2 * i + 1]));
            if (anchored && h > 0.0) {
                con[4 * K] = z[0];
                con[4 * K + 1] = z[1];
                con[4 * K + 2] = sh->s_s * (z[0] - an[2 * i]) * h;
                con[4 * K + 3] = sh->s_s * (z[1] - an[2 * i + 1]) * h;
                ++K;
            }
        }
        for (int32_t j = 0; j < M; ++j) {
            int32_t ra = j / pads->cols, cb = j % pads->cols;
            double sa = (ra - 0.5 * (pads->rows - 1)) * pads->pitch, sb = (cb - 0.5 * (pads->cols - 1)) * pads->pitch;
            double ut = 0.0, ub = 0.0;
            for (int64_t k = 0; k < K; ++k) {
                const double da = sa - con[4 * k], db = sb - con[4 * k + 1];
                const double gk = exp(-sh->lambda_s * (da * da + db * db));
                ut += con[4 * k + 2] * gk;
                ub += con[4 * k + 3] * gk;
            }
            double* uo = u + (ep * M + j) * 3;
            uo[0] = 0.0;
            uo[1] = ut;
            uo[2] = ub;
        }
        n_anchored[ep] = count;
        margin[ep] = mg;
        drag[ep] = dg;
    }
    free(con);
}

void or_shear_step(const or_scene* S, const or_pads* pads, const or_shear* sh, const or_inputs* in, double* anchors,
                   int32_t* anchor_obj, double* u, int32_t* n_anchored, double* margin, double* drag,
                   int32_t threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t e = 0; e < S->n_envs; ++e)
        env_shear(S, pads, sh, in, anchors, anchor_obj, u, n_anchored, margin, drag, e);
}

void or_pc_prox(const or_scene* S, const or_pcprox* pc, const or_inputs* in, double* ft, int32_t threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t e = 0; e < S->n_envs; ++e) env_pc_prox(S, pc, in, ft, e);
}

void or_markers(const or_scene* S, const or_pads* pads, const or_inputs* in, double* u, double* h_out, int32_t threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t e = 0; e < S->n_envs; ++e) env_markers(S, pads, in, u, h_out, e);
}
