// geom.cuh -- signed distance queries in the object frame (Appendix A, Eq. 2:
// depth from phi_g, contact normal from grad phi_g).
//
// Evaluations per object kind:
//   sdf_fast    FP32 phi and unit gradient (proximity rays, markers)
//   sdf_phi_fast  the same FP32 phi without the gradient; enough for every
//               taxel whose probe sphere is clear of the surface (depth = 0
//               exactly) and for the surface-distance output.
//   sdf_refine  phi as a compensated float pair from a compensated query
//               point, gradient in FP32 at the compensated cell / feature.
//               Used only for taxels within a guard band of contact, so the
//               depth (and k * depth) carries ~1e-14 relative error.
#pragma once
#include <cuda_fp16.h>

#include "df.cuh"
#include "internal.h"

namespace tg {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize_or(float3 v, float3 fallback) {
    float n2 = dot(v, v);
    if (n2 > 0.0f) {
        float inv = rsqrtf(n2);
        return v * inv;
    }
    return fallback;
}

// ------------------------------------------------------------------ grids
// Grid values are re-read by every env that holds the object, while the
// per-taxel state streams through L2 once per step: grid loads carry an
// evict-last L2 policy so the grids stay resident under the stream.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// The 8 corner values of cell (i, j, k), read from the cell-major copy of
// the grid (one 16-byte record per cell for binary16, two for float): one
// vector load per query instead of eight scattered ones.
__device__ __forceinline__ uint4 ld_cell16(const uint4* p, uint64_t pol) {
    uint4 v;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ float2 h2f2(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

struct Corners {
    float v000, v100, v010, v110, v001, v101, v011, v111;
};

__device__ __forceinline__ Corners grid_corners(const ObjDev& o, int i, int j, int k) {
    const size_t cell = ((size_t)k * (o.dims[1] - 1) + j) * (o.dims[0] - 1) + i;
    const uint64_t pol = l2_evict_last_policy();
    Corners c;
    if (o.fp16) {
        const uint4 v = ld_cell16(reinterpret_cast<const uint4*>(o.cells) + cell, pol);
        float2 a = h2f2(v.x), b = h2f2(v.y), d = h2f2(v.z), e = h2f2(v.w);
        c.v000 = a.x; c.v100 = a.y; c.v010 = b.x; c.v110 = b.y;
        c.v001 = d.x; c.v101 = d.y; c.v011 = e.x; c.v111 = e.y;
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(o.cells) + 2 * cell;
        const uint4 v = ld_cell16(p, pol), w = ld_cell16(p + 1, pol);
        c.v000 = __uint_as_float(v.x); c.v100 = __uint_as_float(v.y);
        c.v010 = __uint_as_float(v.z); c.v110 = __uint_as_float(v.w);
        c.v001 = __uint_as_float(w.x); c.v101 = __uint_as_float(w.y);
        c.v011 = __uint_as_float(w.z); c.v111 = __uint_as_float(w.w);
    }
    return c;
}

// analytic gradient of the trilinear interpolant (per unit of the cell)
__device__ __forceinline__ float3 trilinear_grad(const Corners& c, float fx, float fy, float fz) {
    float gx = ((c.v100 - c.v000) * (1.0f - fy) + (c.v110 - c.v010) * fy) * (1.0f - fz) +
               ((c.v101 - c.v001) * (1.0f - fy) + (c.v111 - c.v011) * fy) * fz;
    float gy = ((c.v010 - c.v000) * (1.0f - fx) + (c.v110 - c.v100) * fx) * (1.0f - fz) +
               ((c.v011 - c.v001) * (1.0f - fx) + (c.v111 - c.v101) * fx) * fz;
    float gz = ((c.v001 - c.v000) * (1.0f - fx) + (c.v101 - c.v100) * fx) * (1.0f - fy) +
               ((c.v011 - c.v010) * (1.0f - fx) + (c.v111 - c.v110) * fx) * fy;
    return f3(gx, gy, gz);
}

__device__ __forceinline__ float grid_fast(const ObjDev& o, float3 q, float3* g) {
    float c[3] = {fminf(fmaxf(q.x, o.lo[0]), o.hi[0]), fminf(fmaxf(q.y, o.lo[1]), o.hi[1]),
                  fminf(fmaxf(q.z, o.lo[2]), o.hi[2])};
    int i[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = (c[a] - o.lo[a]) * o.inv_h_hi[a];
        int ii = (int)floorf(u);
        ii = min(max(ii, 0), o.dims[a] - 2);
        i[a] = ii;
        f[a] = u - (float)ii;
    }
    Corners v = grid_corners(o, i[0], i[1], i[2]);
    float fx = f[0], fy = f[1], fz = f[2];
    float c00 = v.v000 + fx * (v.v100 - v.v000), c10 = v.v010 + fx * (v.v110 - v.v010);
    float c01 = v.v001 + fx * (v.v101 - v.v001), c11 = v.v011 + fx * (v.v111 - v.v011);
    float c0 = c00 + fy * (c10 - c00), c1 = c01 + fy * (c11 - c01);
    float phi = c0 + fz * (c1 - c0);
    float3 gr = trilinear_grad(v, fx, fy, fz);
    gr = f3(gr.x * o.inv_h_hi[0], gr.y * o.inv_h_hi[1], gr.z * o.inv_h_hi[2]);
    *g = normalize_or(gr, normalize_or(q, f3(0.f, 0.f, 1.f)));
    float3 out = f3(q.x - c[0], q.y - c[1], q.z - c[2]);
    return phi + sqrtf(dot(out, out));
}

// phi alone, for the pass that only decides whether a taxel is near contact:
// the same FP32 interpolation as grid_fast without the gradient
__device__ __forceinline__ float grid_phi_fast(const ObjDev& o, float3 q) {
    float c[3] = {fminf(fmaxf(q.x, o.lo[0]), o.hi[0]), fminf(fmaxf(q.y, o.lo[1]), o.hi[1]),
                  fminf(fmaxf(q.z, o.lo[2]), o.hi[2])};
    int i[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = (c[a] - o.lo[a]) * o.inv_h_hi[a];
        int ii = (int)floorf(u);
        ii = min(max(ii, 0), o.dims[a] - 2);
        i[a] = ii;
        f[a] = u - (float)ii;
    }
    Corners v = grid_corners(o, i[0], i[1], i[2]);
    float fx = f[0], fy = f[1], fz = f[2];
    float c00 = v.v000 + fx * (v.v100 - v.v000), c10 = v.v010 + fx * (v.v110 - v.v010);
    float c01 = v.v001 + fx * (v.v101 - v.v001), c11 = v.v011 + fx * (v.v111 - v.v011);
    float c0 = c00 + fy * (c10 - c00), c1 = c01 + fy * (c11 - c01);
    float phi = c0 + fz * (c1 - c0);
    // distance to the box for points outside it (0 inside); only points
    // outside the padded box, far from any surface, get a non-zero term, and
    // the hardware reciprocal square root is accurate enough there
    float3 out = f3(q.x - c[0], q.y - c[1], q.z - c[2]);
    const float o2 = dot(out, out);
    return phi + o2 * rsqrtf(fmaxf(o2, 1e-30f));
}

// a + f (b - a) for corner values a, b (floats) at a compensated fraction f:
// b - a as an exact pair, then one compensated product and sum
__device__ __forceinline__ df df_lerp_ff(float a, float b, df f) {
    return df_add_f(df_mul(f, two_sum(b, -a)), a);
}
// the same between compensated values (sums with the absolute bound of
// df_add_abs: the values are distances of a few centimetres at most)
__device__ __forceinline__ df df_lerp_abs(df a, df b, df f) {
    return df_add_abs(a, df_mul(f, df_add_abs(b, df_neg(a))));
}

// Compensated phi at a compensated query point (near-contact taxels): the
// cell and in-cell fractions from the compensated point, the trilinear
// interpolant of the stored corner values with compensated products and
// sums (~1e-15 m absolute), the FP32 gradient of the interpolant.  Points
// outside the box add their compensated distance to it.
__device__ __forceinline__ df grid_refine(const ObjDev& o, df3 q, float3* g) {
    df qa[3] = {q.x, q.y, q.z};
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) inside = inside && !df_lt(qa[a], df_from(o.lo[a])) && !df_gt(qa[a], df_from(o.hi[a]));
    df out2 = df_from(0.0f);
    if (!inside) {  // (no near-contact probe of a padded box lies here)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            df ca = qa[a];
            if (df_lt(ca, df_from(o.lo[a]))) ca = df_from(o.lo[a]);
            if (df_gt(ca, df_from(o.hi[a]))) ca = df_from(o.hi[a]);
            const df d = df_sub(qa[a], ca);
            out2 = df_add(out2, df_mul(d, d));
            qa[a] = ca;
        }
    }
    int i[3];
    df f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const df u = df_mul(df_add_f(qa[a], -o.lo[a]), df{o.inv_h_hi[a], o.inv_h_lo[a]});
        int ii = df_floor_int(u);
        ii = min(max(ii, 0), o.dims[a] - 2);
        i[a] = ii;
        f[a] = df_add_f(u, -(float)ii);
    }
    const Corners v = grid_corners(o, i[0], i[1], i[2]);
    const df c00 = df_lerp_ff(v.v000, v.v100, f[0]);
    const df c10 = df_lerp_ff(v.v010, v.v110, f[0]);
    const df c01 = df_lerp_ff(v.v001, v.v101, f[0]);
    const df c11 = df_lerp_ff(v.v011, v.v111, f[0]);
    const df c0 = df_lerp_abs(c00, c10, f[1]);
    const df c1 = df_lerp_abs(c01, c11, f[1]);
    const df phi = df_lerp_abs(c0, c1, f[2]);
    float3 gr = trilinear_grad(v, f[0].hi, f[1].hi, f[2].hi);
    gr = f3(gr.x * o.inv_h_hi[0], gr.y * o.inv_h_hi[1], gr.z * o.inv_h_hi[2]);
    *g = normalize_or(gr, normalize_or(f3(q.x.hi, q.y.hi, q.z.hi), f3(0.f, 0.f, 1.f)));
    return inside ? phi : df_add(phi, df_sqrt(out2));
}

// ------------------------------------------------------------------ analytic
static __device__ __noinline__ float box_fast(const ObjDev& o, float3 q, float3* g) {
    float d[3] = {fabsf(q.x) - o.half[0], fabsf(q.y) - o.half[1], fabsf(q.z) - o.half[2]};
    float qa[3] = {q.x, q.y, q.z};
    float oo[3] = {fmaxf(d[0], 0.f), fmaxf(d[1], 0.f), fmaxf(d[2], 0.f)};
    float outside = sqrtf(oo[0] * oo[0] + oo[1] * oo[1] + oo[2] * oo[2]);
    if (outside > 0.0f) {
        *g = f3(copysignf(oo[0], qa[0]), copysignf(oo[1], qa[1]), copysignf(oo[2], qa[2])) * (1.0f / outside);
        return outside;
    }
    int am = 0;
    if (d[1] > d[am]) am = 1;
    if (d[2] > d[am]) am = 2;
    float gg[3] = {0.f, 0.f, 0.f};
    gg[am] = qa[am] < 0.f ? -1.f : 1.f;
    *g = f3(gg[0], gg[1], gg[2]);
    return d[am];
}

__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.f ? df_neg(a) : a; }

static __device__ __noinline__ df box_refine(const ObjDev& o, df3 q, float3* g) {
    df qa[3] = {q.x, q.y, q.z};
    df d[3];
    df o2 = df_from(0.f);
    bool out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] = df_add_f(df_abs(qa[a]), -o.half[a]);
        if (d[a].hi > 0.f) { out = true; o2 = df_add(o2, df_mul(d[a], d[a])); }
    }
    if (out) {
        df dist = df_sqrt(o2);
        float3 v = f3(d[0].hi > 0.f ? copysignf(d[0].hi, qa[0].hi) : 0.f,
                      d[1].hi > 0.f ? copysignf(d[1].hi, qa[1].hi) : 0.f,
                      d[2].hi > 0.f ? copysignf(d[2].hi, qa[2].hi) : 0.f);
        *g = normalize_or(v, f3(0.f, 0.f, 1.f));
        return dist;
    }
    int am = 0;
    if (df_gt(d[1], d[am])) am = 1;
    if (df_gt(d[2], d[am])) am = 2;
    float gg[3] = {0.f, 0.f, 0.f};
    gg[am] = qa[am].hi < 0.f ? -1.f : 1.f;
    *g = f3(gg[0], gg[1], gg[2]);
    return d[am];
}

// ------------------------------------------------------------------ meshes
// Closest point on a triangle by Voronoi-region classification (Ericson,
// Real-Time Collision Detection, 5.1.5), generic over float and the
// compensated pair.  Returns the squared distance and the region
// (0 face, 1..3 vertex, 4..6 edge).
struct dfn {
    df v;
};
__device__ __forceinline__ dfn operator+(dfn a, dfn b) { return dfn{df_add(a.v, b.v)}; }
__device__ __forceinline__ dfn operator-(dfn a, dfn b) { return dfn{df_sub(a.v, b.v)}; }
__device__ __forceinline__ dfn operator*(dfn a, dfn b) { return dfn{df_mul(a.v, b.v)}; }
__device__ __forceinline__ dfn operator/(dfn a, dfn b) { return dfn{df_div(a.v, b.v)}; }
__device__ __forceinline__ bool operator<=(dfn a, float b) { return !df_gt(a.v, df_from(b)); }
__device__ __forceinline__ bool operator>=(dfn a, float b) { return !df_lt(a.v, df_from(b)); }
__device__ __forceinline__ bool operator<=(dfn a, dfn b) { return !df_gt(a.v, b.v); }
__device__ __forceinline__ dfn mk(float a) { return dfn{df_from(a)}; }
__device__ __forceinline__ float mkf(float a) { return a; }

template <class S>
struct V3 {
    S x, y, z;
};
template <class S>
__device__ __forceinline__ S vdot(V3<S> a, V3<S> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S>
__device__ __forceinline__ V3<S> vsub(V3<S> a, V3<S> b) { return V3<S>{a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S>
__device__ __forceinline__ V3<S> vmad(V3<S> a, V3<S> d, S t) { return V3<S>{a.x + d.x * t, a.y + d.y * t, a.z + d.z * t}; }

template <class S>
__device__ __forceinline__ S closest_point_tri(V3<S> p, V3<S> a, V3<S> b, V3<S> c, V3<S>* cp, int* region) {
    V3<S> ab = vsub(b, a), ac = vsub(c, a), ap = vsub(p, a);
    S d1 = vdot(ab, ap), d2 = vdot(ac, ap);
    V3<S> q;
    if (d1 <= 0.0f && d2 <= 0.0f) { q = a; *region = 1; }
    else {
        V3<S> bp = vsub(p, b);
        S d3 = vdot(ab, bp), d4 = vdot(ac, bp);
        if (d3 >= 0.0f && d4 <= d3) { q = b; *region = 2; }
        else {
            S vc = d1 * d4 - d3 * d2;
            if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
                q = vmad(a, ab, d1 / (d1 - d3)); *region = 4;
            } else {
                V3<S> cpv = vsub(p, c);
                S d5 = vdot(ab, cpv), d6 = vdot(ac, cpv);
                if (d6 >= 0.0f && d5 <= d6) { q = c; *region = 3; }
                else {
                    S vb = d5 * d2 - d1 * d6;
                    if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
                        q = vmad(a, ac, d2 / (d2 - d6)); *region = 5;
                    } else {
                        S va = d3 * d6 - d5 * d4;
                        S e43 = d4 - d3, e56 = d5 - d6;
                        if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
                            q = vmad(b, vsub(c, b), e43 / (e43 + e56)); *region = 6;
                        } else {
                            S den = va + vb + vc;
                            S v = vb / den, w = vc / den;
                            q = vmad(vmad(a, ab, v), ac, w); *region = 0;
                        }
                    }
                }
            }
        }
    }
    *cp = q;
    V3<S> dd = vsub(p, q);
    return vdot(dd, dd);
}

__device__ __forceinline__ V3<float> tri_vert(const float* t, int f, int v) {
    const float* p = t + (size_t)f * 9 + v * 3;
    return V3<float>{__ldg(p), __ldg(p + 1), __ldg(p + 2)};
}

// solid angle of a triangle seen from p (Van Oosterom and Strackee, 1983)
__device__ __forceinline__ float solid_angle(V3<float> A, V3<float> B, V3<float> C) {
    float la = sqrtf(vdot(A, A)), lb = sqrtf(vdot(B, B)), lc = sqrtf(vdot(C, C));
    float num = A.x * (B.y * C.z - B.z * C.y) + A.y * (B.z * C.x - B.x * C.z) + A.z * (B.x * C.y - B.y * C.x);
    float den = la * lb * lc + vdot(A, B) * lc + vdot(B, C) * la + vdot(C, A) * lb;
    return 2.0f * atan2f(num, den);
}

// FP32 pass over all faces: min squared distance, nearest face, winding number
static __device__ __noinline__ void mesh_scan(const ObjDev& o, float3 qf, float* dmin2, int* best, float* wind) {
    V3<float> p{qf.x, qf.y, qf.z};
    float bd = INFINITY, w = 0.f;
    int bf = 0;
    for (int f = 0; f < o.n_faces; ++f) {
        V3<float> a = tri_vert(o.tri, f, 0), b = tri_vert(o.tri, f, 1), c = tri_vert(o.tri, f, 2);
        V3<float> cp;
        int reg;
        float d2 = closest_point_tri<float>(p, a, b, c, &cp, &reg);
        if (d2 < bd) { bd = d2; bf = f; }
        w += solid_angle(vsub(a, p), vsub(b, p), vsub(c, p));
    }
    *dmin2 = bd;
    *best = bf;
    *wind = w * 0.079577471545947668f;  // 1 / (4 pi)
}

static __device__ __noinline__ float mesh_fast(const ObjDev& o, float3 q, float3* g) {
    float d2, w;
    int bf;
    mesh_scan(o, q, &d2, &bf, &w);
    float sign = w > 0.5f ? -1.0f : 1.0f;
    V3<float> cp;
    int reg;
    closest_point_tri<float>(V3<float>{q.x, q.y, q.z}, tri_vert(o.tri, bf, 0), tri_vert(o.tri, bf, 1),
                             tri_vert(o.tri, bf, 2), &cp, &reg);
    float d = sqrtf(d2);
    if (reg == 0 || !(d > 0.f)) {
        *g = f3(__ldg(o.tri_n + 3 * bf), __ldg(o.tri_n + 3 * bf + 1), __ldg(o.tri_n + 3 * bf + 2));
    } else {
        *g = normalize_or(f3(q.x - cp.x, q.y - cp.y, q.z - cp.z) * sign, f3(0.f, 0.f, 1.f));
    }
    return sign * d;
}

// FP32 scan, then every face within a guard of the FP32 minimum re-evaluated
// with the compensated closest point; the smallest compensated distance wins.
static __device__ __noinline__ df mesh_refine(const ObjDev& o, df3 q, float3* g) {
    float3 qf = f3(q.x.hi, q.y.hi, q.z.hi);
    float d2, w;
    int bf;
    mesh_scan(o, qf, &d2, &bf, &w);
    float sign = w > 0.5f ? -1.0f : 1.0f;
    float guard = sqrtf(d2) + 1e-6f;
    float guard2 = guard * guard;
    V3<dfn> p{dfn{q.x}, dfn{q.y}, dfn{q.z}};
    df best = df_from(INFINITY);
    int best_face = bf, best_reg = 0;
    V3<dfn> best_cp{mk(0.f), mk(0.f), mk(0.f)};
    V3<float> pf{qf.x, qf.y, qf.z};
    for (int f = 0; f < o.n_faces; ++f) {
        V3<float> a = tri_vert(o.tri, f, 0), b = tri_vert(o.tri, f, 1), c = tri_vert(o.tri, f, 2);
        V3<float> cpf;
        int reg;
        float e2 = closest_point_tri<float>(pf, a, b, c, &cpf, &reg);
        if (e2 > guard2) continue;
        V3<dfn> A{mk(a.x), mk(a.y), mk(a.z)}, B{mk(b.x), mk(b.y), mk(b.z)}, C{mk(c.x), mk(c.y), mk(c.z)};
        V3<dfn> cp;
        dfn dd2 = closest_point_tri<dfn>(p, A, B, C, &cp, &reg);
        if (df_lt(dd2.v, best)) { best = dd2.v; best_face = f; best_reg = reg; best_cp = cp; }
    }
    df dist = df_sqrt(best);
    if (best_reg == 0 || !(dist.hi > 0.f)) {
        *g = f3(__ldg(o.tri_n + 3 * best_face), __ldg(o.tri_n + 3 * best_face + 1), __ldg(o.tri_n + 3 * best_face + 2));
    } else {
        df3 dv = df3{df_sub(q.x, best_cp.x.v), df_sub(q.y, best_cp.y.v), df_sub(q.z, best_cp.z.v)};
        *g = normalize_or(f3(dv.x.hi, dv.y.hi, dv.z.hi) * sign, f3(0.f, 0.f, 1.f));
    }
    return sign < 0.f ? df_neg(dist) : dist;
}

// ------------------------------------------------------------------ dispatch
__device__ __forceinline__ float sdf_fast(const ObjDev& o, float3 q, float3* g) {
    switch (o.kind) {
    case TG_OBJ_SPHERE: {
        float n = sqrtf(dot(q, q));
        *g = normalize_or(q, f3(0.f, 0.f, 1.f));
        return n - o.radius;
    }
    case TG_OBJ_BOX: return box_fast(o, q, g);
    case TG_OBJ_PLANE: *g = f3(0.f, 0.f, 1.f); return q.z;
    case TG_OBJ_MESH: return mesh_fast(o, q, g);
    case TG_OBJ_GRID:
    case TG_OBJ_NEURAL: return grid_fast(o, q, g);  // a learned SDF's fallback grid (proximity, markers)
    default: *g = f3(0.f, 0.f, 1.f); return __int_as_float(0x7fc00000);
    }
}

// FP32 phi without the gradient (equal to sdf_fast's phi)
__device__ __forceinline__ float sdf_phi_fast(const ObjDev& o, float3 q) {
    float3 g;
    switch (o.kind) {
    case TG_OBJ_SPHERE: return sqrtf(dot(q, q)) - o.radius;
    case TG_OBJ_BOX: return box_fast(o, q, &g);
    case TG_OBJ_PLANE: return q.z;
    case TG_OBJ_MESH: return mesh_fast(o, q, &g);
    case TG_OBJ_GRID:
    case TG_OBJ_NEURAL: return grid_phi_fast(o, q);
    default: return __int_as_float(0x7fc00000);
    }
}

__device__ __forceinline__ df sdf_refine(const ObjDev& o, df3 q, float3* g) {
    switch (o.kind) {
    case TG_OBJ_SPHERE: {
        df n = df_sqrt(df_dot3(q, q));
        *g = normalize_or(f3(q.x.hi, q.y.hi, q.z.hi), f3(0.f, 0.f, 1.f));
        return df_add_f(n, -o.radius);
    }
    case TG_OBJ_BOX: return box_refine(o, q, g);
    case TG_OBJ_PLANE: *g = f3(0.f, 0.f, 1.f); return q.z;
    case TG_OBJ_MESH: return mesh_refine(o, q, g);
    case TG_OBJ_GRID:
    case TG_OBJ_NEURAL: return grid_refine(o, q, g);
    default: *g = f3(0.f, 0.f, 1.f); return df_from(__int_as_float(0x7fc00000));
    }
}

}  // namespace tg
