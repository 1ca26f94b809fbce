// nsdf.cuh -- device side of the learned signed-distance surrogate: the
// multiresolution hash encoding (16 levels x 2 binary16 features, 2^16
// entries per level; Mueller et al. 2022) and the 32 -> 64 -> 64 -> 1 ReLU MLP
// with bfloat16 weights, whose output is the distance in millimetres.
//
// Geometry of the encoding: level l has N_l = floor(16 * 2^(l/3)) cells per
// axis over the object's box; vertex (i, j, k) is entry i + (N+1)(j + (N+1)k)
// while (N+1)^3 <= 2^16 (levels 0-3), else (i ^ j * 2654435761 ^
// k * 805459861) mod 2^16.  Outside the box the distance is extended as
// phi(clamp q) + |q - clamp q|, as for the SDF grids.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace tg {

constexpr int kNsdfLevels = 16;
constexpr int kNsdfTable = 1 << 16;
constexpr int kNsdfHidden = 64;
constexpr int kNsdfIn = 32;
constexpr int kNsdfWeights = kNsdfHidden * kNsdfIn + kNsdfHidden * kNsdfHidden + kNsdfHidden;  // 6,208
constexpr int64_t kNsdfTableEntries = (int64_t)kNsdfLevels * kNsdfTable;                       // half2 each
constexpr int kNsdfDenseLevels = 4;  // (N+1)^3 <= 2^16 for N = 16, 20, 25, 32

// N_l = floor(16 * 2^(l/3)), l = 0..15
__device__ __forceinline__ int nsdf_res(int l) {
    switch (l) {
    case 0: return 16;   case 1: return 20;   case 2: return 25;   case 3: return 32;
    case 4: return 40;   case 5: return 50;   case 6: return 64;   case 7: return 80;
    case 8: return 101;  case 9: return 128;  case 10: return 161; case 11: return 203;
    case 12: return 256; case 13: return 322; case 14: return 406; default: return 512;
    }
}

__device__ __forceinline__ uint32_t nsdf_entry(int l, int n1, uint32_t i, uint32_t j, uint32_t k) {
    if (l < kNsdfDenseLevels) return i + (uint32_t)n1 * (j + (uint32_t)n1 * k);
    return (i ^ (j * 2654435761u) ^ (k * 805459861u)) & (uint32_t)(kNsdfTable - 1);
}

// The cell of level l holding u (in [0,1]^3): base vertex and fractions.
struct NsdfCell {
    uint32_t i, j, k;
    float fx, fy, fz;
    int n1;
};

__device__ __forceinline__ NsdfCell nsdf_cell(int l, float ux, float uy, float uz) {
    const int N = nsdf_res(l);
    const float px = ux * (float)N, py = uy * (float)N, pz = uz * (float)N;
    const int ix = min((int)floorf(px), N - 1), iy = min((int)floorf(py), N - 1), iz = min((int)floorf(pz), N - 1);
    NsdfCell c;
    c.i = (uint32_t)max(ix, 0);
    c.j = (uint32_t)max(iy, 0);
    c.k = (uint32_t)max(iz, 0);
    c.fx = px - (float)(int)c.i;
    c.fy = py - (float)(int)c.j;
    c.fz = pz - (float)(int)c.k;
    c.n1 = N + 1;
    return c;
}

__device__ __forceinline__ float2 nsdf_feat(const uint32_t* table, int l, uint32_t e) {
    const uint32_t v = __ldg(table + (size_t)l * kNsdfTable + e);
    return __half22float2(*reinterpret_cast<const __half2*>(&v));
}

// Object-frame point -> clamped point, u in [0,1]^3 and |q - clamp q|.
__device__ __forceinline__ float nsdf_clamp(const ObjDev& o, float3 q, float* u) {
    const float cx = fminf(fmaxf(q.x, o.nlo[0]), o.nhi[0]);
    const float cy = fminf(fmaxf(q.y, o.nlo[1]), o.nhi[1]);
    const float cz = fminf(fmaxf(q.z, o.nlo[2]), o.nhi[2]);
    u[0] = (cx - o.nlo[0]) * o.ninv_ext[0];
    u[1] = (cy - o.nlo[1]) * o.ninv_ext[1];
    u[2] = (cz - o.nlo[2]) * o.ninv_ext[2];
    const float dx = q.x - cx, dy = q.y - cy, dz = q.z - cz;
    return sqrtf(dx * dx + dy * dy + dz * dz);
}

// Encoding values of levels l0 .. l0 + NL - 1 of u into enc[0 .. 2 NL)
// (FP32 sums of the 8 weighted corner features).
template <int NL>
__device__ __forceinline__ void nsdf_encode_levels(const uint32_t* table, const float* u, int l0, float* enc) {
#pragma unroll
    for (int jl = 0; jl < NL; ++jl) {
        const int l = l0 + jl;
        const NsdfCell c = nsdf_cell(l, u[0], u[1], u[2]);
        float e0 = 0.f, e1 = 0.f;
#pragma unroll
        for (int corner = 0; corner < 8; ++corner) {
            const uint32_t dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
            const float w = (dx ? c.fx : 1.f - c.fx) * (dy ? c.fy : 1.f - c.fy) * (dz ? c.fz : 1.f - c.fz);
            const float2 f = nsdf_feat(table, l, nsdf_entry(l, c.n1, c.i + dx, c.j + dy, c.k + dz));
            e0 = fmaf(w, f.x, e0);
            e1 = fmaf(w, f.y, e1);
        }
        enc[2 * jl] = e0;
        enc[2 * jl + 1] = e1;
    }
}

// The 32 encoding values of u.
__device__ __forceinline__ void nsdf_encode(const uint32_t* table, const float* u, float* enc) {
    nsdf_encode_levels<kNsdfLevels>(table, u, 0, enc);
}

__device__ __forceinline__ float bf16f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

}  // namespace tg
