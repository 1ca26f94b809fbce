// mesh_kernel.cuh -- the exact mesh signed-distance kernel shared by the
// allocating entry points (mesh.cu: grid bake and point queries) and the
// non-allocating point query (mesh_noalloc.cu).
//
// Per point: an FP32 pass over all faces (closest point by Voronoi regions,
// Ericson 5.1.5; generalised winding number from Van Oosterom-Strackee solid
// angles) finds the nearest distance and the inside/outside sign; a second
// pass re-evaluates, with compensated arithmetic, every face whose FP32
// distance lies within a guard band of the minimum.  The result is rounded
// once, to float or to binary16, from the compensated value.  Faces are
// staged through shared memory in tiles that every thread of the CTA reuses.
#pragma once
#include <cuda_fp16.h>

#include "df.cuh"
#include "geom.cuh"
#include "internal.h"

namespace tg {

constexpr int kMeshThreads = 128;
constexpr int kFaceTile = 256;

struct MeshSrc {
    const float* points;   // mode 0: [n][3]
    int64_t n;
    int dims[3];           // mode 1: grid nodes
    float lo_hi[3], lo_lo[3], h_hi[3], h_lo[3];
    int mode;
};

__device__ __forceinline__ df3 mesh_point(const MeshSrc& s, int64_t idx) {
    if (s.mode == 0) return df3_from(s.points[3 * idx], s.points[3 * idx + 1], s.points[3 * idx + 2]);
    const int64_t nx = s.dims[0], ny = s.dims[1];
    const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / (nx * ny));
    const int ii[3] = {i, j, k};
    df c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = df_add(df{s.lo_hi[a], s.lo_lo[a]}, df_mul_f(df{s.h_hi[a], s.h_lo[a]}, (float)ii[a]));
    return df3{c[0], c[1], c[2]};
}

// round a compensated value to binary16 as if from the exact sum hi + lo
__device__ __forceinline__ __half df_to_half_rn(df v) {
    const float a = fabsf(v.hi);
    bool tie;
    float lower;  // the half of smaller magnitude around a tie
    if (a >= 6.103515625e-05f) {  // normal binary16 range: 10 fraction bits
        const uint32_t bits = __float_as_uint(a);
        tie = (bits & 0x1FFFu) == 0x1000u;
        lower = __uint_as_float(bits & ~0x1FFFu);
    } else {                      // subnormal binary16: multiples of 2^-24
        const float t = a * 33554432.0f;  // 2^25, exact
        tie = (t == floorf(t)) && (fmodf(t, 2.0f) == 1.0f);
        lower = (t - 1.0f) * 2.98023223876953125e-08f;
    }
    if (!tie || v.lo == 0.0f) return __float2half_rn(v.hi);
    const bool away = (v.lo > 0.0f) == (v.hi > 0.0f);
    const float mag = away ? lower + 2.0f * (a - lower) : lower;
    return __float2half_rn(copysignf(mag, v.hi));
}

template <int NT>
__global__ void __launch_bounds__(NT) mesh_sdf_kernel(const float* __restrict__ tri, const float* __restrict__ tri_n,
                                                      int nf, MeshSrc src, float* phi_out, float* grad_out,
                                                      void* grid_out, int fp16) {
    __shared__ float st[kFaceTile * 9];
    const int64_t idx = (int64_t)blockIdx.x * NT + threadIdx.x;
    const bool live = idx < src.n;
    const df3 p = live ? mesh_point(src, idx) : df3_from(0.f, 0.f, 0.f);
    const V3<float> pf{p.x.hi, p.y.hi, p.z.hi};

    // pass 1: FP32 minimum and winding number
    float best2 = INFINITY, wsum = 0.0f;
    for (int f0 = 0; f0 < nf; f0 += kFaceTile) {
        const int nt = min(kFaceTile, nf - f0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt * 9; i += NT) st[i] = tri[(size_t)f0 * 9 + i];
        __syncthreads();
        if (live) {
            for (int f = 0; f < nt; ++f) {
                const float* t = st + 9 * f;
                V3<float> a{t[0], t[1], t[2]}, b{t[3], t[4], t[5]}, c{t[6], t[7], t[8]};
                V3<float> cp;
                int reg;
                float d2 = closest_point_tri<float>(pf, a, b, c, &cp, &reg);
                best2 = fminf(best2, d2);
                wsum += solid_angle(vsub(a, pf), vsub(b, pf), vsub(c, pf));
            }
        }
    }
    const float sign = wsum * 0.079577471545947668f > 0.5f ? -1.0f : 1.0f;
    const float guard = sqrtf(best2) + 1e-6f;
    const float guard2 = guard * guard;

    // pass 2: compensated re-evaluation of the faces near the minimum
    V3<dfn> pd{dfn{p.x}, dfn{p.y}, dfn{p.z}};
    df best = df_from(INFINITY);
    int best_face = 0, best_reg = 0;
    V3<dfn> best_cp{mk(0.f), mk(0.f), mk(0.f)};
    for (int f0 = 0; f0 < nf; f0 += kFaceTile) {
        const int nt = min(kFaceTile, nf - f0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt * 9; i += NT) st[i] = tri[(size_t)f0 * 9 + i];
        __syncthreads();
        if (live) {
            for (int f = 0; f < nt; ++f) {
                const float* t = st + 9 * f;
                V3<float> a{t[0], t[1], t[2]}, b{t[3], t[4], t[5]}, c{t[6], t[7], t[8]};
                V3<float> cpf;
                int reg;
                float e2 = closest_point_tri<float>(pf, a, b, c, &cpf, &reg);
                if (e2 > guard2) continue;
                V3<dfn> A{mk(a.x), mk(a.y), mk(a.z)}, B{mk(b.x), mk(b.y), mk(b.z)}, C{mk(c.x), mk(c.y), mk(c.z)};
                V3<dfn> cp;
                dfn d2 = closest_point_tri<dfn>(pd, A, B, C, &cp, &reg);
                if (df_lt(d2.v, best)) { best = d2.v; best_face = f0 + f; best_reg = reg; best_cp = cp; }
            }
        }
    }
    if (!live) return;
    df dist = df_sqrt(best);
    df phi = sign < 0.0f ? df_neg(dist) : dist;
    if (grid_out) {
        if (fp16) reinterpret_cast<__half*>(grid_out)[idx] = df_to_half_rn(phi);
        else reinterpret_cast<float*>(grid_out)[idx] = phi.hi;
    }
    if (phi_out) phi_out[idx] = phi.hi;
    if (grad_out) {
        float3 g;
        if (best_reg == 0 || !(dist.hi > 0.f)) {
            g = f3(tri_n[3 * best_face], tri_n[3 * best_face + 1], tri_n[3 * best_face + 2]);
        } else {
            float3 dv = f3(df_sub(p.x, best_cp.x.v).hi, df_sub(p.y, best_cp.y.v).hi, df_sub(p.z, best_cp.z.v).hi);
            g = normalize_or(dv * sign, f3(0.f, 0.f, 1.f));
        }
        grad_out[3 * idx] = g.x;
        grad_out[3 * idx + 1] = g.y;
        grad_out[3 * idx + 2] = g.z;
    }
}

}  // namespace tg
