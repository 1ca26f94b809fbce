// nsdf.cu -- the learned signed-distance surrogate on the GPU: inference on
// tensor cores, the input gradient of near-contact queries, the training
// forward/backward, and Adam.
//
// Inference (tiles of 128 points, 8 warps): each point's 32 encoding values
// are gathered from the binary16 table and rounded to bfloat16; the two
// hidden layers run as warp-level bfloat16 MMAs with FP32 accumulation (one
// warp per 16 points; the accumulator fragments of layer 1 are re-packed in
// registers as the A operand of layer 2); ReLU outputs are rounded to
// bfloat16; the output layer is an FP32 dot product of the rounded h2 with
// W3.  tg_nsdf_eval's gradient is the analytic d phi / d q in FP32 (one warp
// per point); contact normals in a step use a central-difference stencil.
//
// Training (tiles of 128 points, one thread per point for the per-point
// vectors): FP32 activations on the stored binary16 / bfloat16 parameters,
// backward of the mean L1 loss; weight gradients as per-CTA partial sums
// reduced by a second kernel, table gradients by float2 atomics.
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "geom.cuh"
#include "nsdf.cuh"
#include "rng.cuh"

namespace tg {

namespace {

constexpr int kRows = 128;
constexpr int kInferThreads = 256;
constexpr uint32_t kTagNsdfBatch = 48, kTagNsdfInit = 49;

// Operand tiles in the tensor cores' no-swizzle K-major layout: core
// matrices of 8 rows x 16 bytes (8 bfloat16 along K); element (r, k) of an
// operand with R rows at byte ((k / 8) (R / 8) + r / 8) 128 + (r % 8) 16 +
// (k % 8) 2.  Core matrices adjacent along K are (R / 8) 128 bytes apart
// (the descriptor's leading byte offset), adjacent 8-row groups 128 bytes
// (its stride byte offset).
__host__ __device__ constexpr uint32_t core_off(int r, int k, int R) {
    return (uint32_t)(((k >> 3) * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct __align__(128) SmemInfer {
    unsigned char a1[kRows * kNsdfIn * 2];          // encoding tile, 128 x 32 (8 KB)
    unsigned char a2[kRows * kNsdfHidden * 2];      // h1 tile, 128 x 64 (16 KB)
    unsigned char w1[kNsdfHidden * kNsdfIn * 2];    // W1 as the B operand, 64 x 32 (4 KB)
    unsigned char w2[kNsdfHidden * kNsdfHidden * 2];  // W2, 64 x 64 (8 KB)
    uint32_t h2pos[2][kRows];                       // h2 > 0 per unit (column halves), for the analytic gradient
    float w3[kNsdfHidden];
    float outp[2][kRows];                           // the two column halves of W3 . h2
    float u[kRows][3];
    float ext[kRows];
    float out[kRows];
    float q[kRows][3];
    int64_t gidx[kRows];   // destination index of each row (-1: padding)
    float scale[kRows];
    int16_t queue[kRows];
    int nq;
    uint64_t mbar;         // MMA completion barrier
    uint32_t tmem;         // TMEM base: columns [0, 64) layer 1, [64, 128) layer 2
    uint32_t phase;        // completions so far (parity of the next wait)
    // sized to ~61 KB: 3 CTAs per SM (384 of the 512 TMEM columns) with the
    // shared-memory carveout leaving ~60 KB of L1 for the table gathers; a
    // sweep on GB300 (1M queries) gave 0.92 ms at 4 CTAs / 49 KB, 0.48 ms here,
    // 0.90 ms at 3 CTAs / 73 KB (carveout 228 KB, L1 28 KB), 0.60 ms at 2 CTAs
    unsigned char pad_l1[16384];
};
static_assert(sizeof(SmemInfer) * 4 > 228 * 1024, "at most 3 CTAs per SM (3 x 128 TMEM columns)");

__device__ __forceinline__ float bf16_at(const unsigned char* tile, int r, int k, int R) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(tile + core_off(r, k, R)));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ void load_weights(SmemInfer& S, const uint16_t* w) {
    for (int j = threadIdx.x; j < kNsdfHidden * kNsdfIn; j += blockDim.x)
        *reinterpret_cast<uint16_t*>(S.w1 + core_off(j / kNsdfIn, j % kNsdfIn, kNsdfHidden)) = w[j];
    for (int j = threadIdx.x; j < kNsdfHidden * kNsdfHidden; j += blockDim.x)
        *reinterpret_cast<uint16_t*>(S.w2 + core_off(j / kNsdfHidden, j % kNsdfHidden, kNsdfHidden)) =
            w[kNsdfHidden * kNsdfIn + j];
    for (int j = threadIdx.x; j < kNsdfHidden; j += blockDim.x)
        S.w3[j] = bf16f(w[kNsdfHidden * kNsdfIn + kNsdfHidden * kNsdfHidden + j]);
}

// ---- tcgen05 plumbing (inline PTX) -------------------------------------------
// shared-memory operand descriptor: start, leading byte offset (K-adjacent
// core matrices), stride byte offset (row groups), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator, bfloat16 A and B, both
// K-major, N = 64, M = 128
constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kIdescM128N64), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        (uint32_t)__cvta_generic_to_shared(mbar)));
}

// bounded wait for the barrier phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(mbar);
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

// TMEM (128 columns) and the MMA barrier for this CTA; warp 0 allocates.
__device__ void tc_setup(SmemInfer& S) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&S.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        S.phase = 0;
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
            (uint32_t)__cvta_generic_to_shared(&S.tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ void tc_teardown(SmemInfer& S) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(S.tmem));
}

// Forward of the 128 rows whose u[] is set: S.out[r] (mm); h1 (a2) and h2 kept.
// Both hidden layers on the tensor cores (M = 128 rows, N = 64, K = 32 / 64 in
// steps of 16), accumulators in TMEM; 8 warps read them back, warp w the lanes
// 32 (w % 4) .. + 31 and the column half w / 4.  Returns false (the same in
// every thread) if an MMA did not complete within the wait limit.
__device__ bool infer_tile(SmemInfer& S, const uint32_t* table) {
    const int tid = threadIdx.x;
    const uint32_t ph = S.phase;  // MMA completions so far: this tile waits for ph and ph + 1
    {   // encoding: two threads per row, 8 levels each, two 16-byte stores each
        const int r = tid >> 1, half = tid & 1;
        float enc[16];
        nsdf_encode_levels<8>(table, S.u[r], 8 * half, enc);
        uint4 v0, v1;
        v0.x = pack_bf16(enc[0], enc[1]);   v0.y = pack_bf16(enc[2], enc[3]);
        v0.z = pack_bf16(enc[4], enc[5]);   v0.w = pack_bf16(enc[6], enc[7]);
        v1.x = pack_bf16(enc[8], enc[9]);   v1.y = pack_bf16(enc[10], enc[11]);
        v1.z = pack_bf16(enc[12], enc[13]); v1.w = pack_bf16(enc[14], enc[15]);
        *reinterpret_cast<uint4*>(S.a1 + core_off(r, 16 * half, kRows)) = v0;
        *reinterpret_cast<uint4*>(S.a1 + core_off(r, 16 * half + 8, kRows)) = v1;
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        for (int ks = 0; ks < kNsdfIn / 16; ++ks)
            tc_mma(S.tmem, smem_desc(S.a1 + ks * 2 * (kRows / 8) * 128, (kRows / 8) * 128, 128),
                   smem_desc(S.w1 + ks * 2 * (kNsdfHidden / 8) * 128, (kNsdfHidden / 8) * 128, 128), ks > 0);
        tc_commit(&S.mbar);
    }
    const int warp = tid >> 5, lane = tid & 31;
    const int r = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);
    const uint32_t lane_addr = S.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    bool ok = mbar_wait(&S.mbar, ph & 1u);
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
    {   // layer-1 epilogue: ReLU, bfloat16, into the h1 operand tile
        float z[32];
        tmem_ld32(lane_addr + c0, z);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint4 v;
            v.x = pack_bf16(fmaxf(z[8 * j], 0.f), fmaxf(z[8 * j + 1], 0.f));
            v.y = pack_bf16(fmaxf(z[8 * j + 2], 0.f), fmaxf(z[8 * j + 3], 0.f));
            v.z = pack_bf16(fmaxf(z[8 * j + 4], 0.f), fmaxf(z[8 * j + 5], 0.f));
            v.w = pack_bf16(fmaxf(z[8 * j + 6], 0.f), fmaxf(z[8 * j + 7], 0.f));
            *reinterpret_cast<uint4*>(S.a2 + core_off(r, c0 + 8 * j, kRows)) = v;
        }
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        for (int ks = 0; ks < kNsdfHidden / 16; ++ks)
            tc_mma(S.tmem + 64, smem_desc(S.a2 + ks * 2 * (kRows / 8) * 128, (kRows / 8) * 128, 128),
                   smem_desc(S.w2 + ks * 2 * (kNsdfHidden / 8) * 128, (kNsdfHidden / 8) * 128, 128), ks > 0);
        tc_commit(&S.mbar);
    }
    ok = mbar_wait(&S.mbar, (ph + 1u) & 1u);
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
    {   // layer-2 epilogue: ReLU, bfloat16, the half dot product with W3; keep h2
        float z[32];
        tmem_ld32(lane_addr + 64 + c0, z);
        float s = 0.f;
        uint32_t pos = 0;
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(z[j], 0.f), fmaxf(z[j + 1], 0.f));
            const float lo = __low2float(h), hi = __high2float(h);
            pos |= (lo > 0.f ? 1u : 0u) << j;
            pos |= (hi > 0.f ? 1u : 0u) << (j + 1);
            s = fmaf(lo, S.w3[c0 + j], s);
            s = fmaf(hi, S.w3[c0 + j + 1], s);
        }
        S.outp[warp >> 2][r] = s;
        S.h2pos[warp >> 2][r] = pos;
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) S.phase = ph + 2u;  // read again only after the caller's next barrier
    if (tid < kRows) S.out[tid] = S.outp[0][tid] + S.outp[1][tid];
    return true;
}

// d phi / d q (object frame, raw) of row r, by one warp.
__device__ float3 row_grad(const SmemInfer& S, const uint32_t* table, const ObjDev& o, int r) {
    const int lane = threadIdx.x & 31;
    // g_z2 = [h2 > 0] W3 for units lane, lane + 32
    const float gz2a = ((S.h2pos[0][r] >> lane) & 1u) ? S.w3[lane] : 0.f;
    const float gz2b = ((S.h2pos[1][r] >> lane) & 1u) ? S.w3[lane + 32] : 0.f;
    float gh1a = 0.f, gh1b = 0.f;  // units lane, lane + 32
#pragma unroll 8
    for (int oo = 0; oo < kNsdfHidden; ++oo) {
        const float v = __shfl_sync(0xffffffffu, oo < 32 ? gz2a : gz2b, oo & 31);
        gh1a = fmaf(v, bf16_at(S.w2, oo, lane, kNsdfHidden), gh1a);
        gh1b = fmaf(v, bf16_at(S.w2, oo, lane + 32, kNsdfHidden), gh1b);
    }
    const float gz1a = bf16_at(S.a2, r, lane, kRows) > 0.f ? gh1a : 0.f;
    const float gz1b = bf16_at(S.a2, r, lane + 32, kRows) > 0.f ? gh1b : 0.f;
    float genc = 0.f;  // d out / d enc[lane]
#pragma unroll 8
    for (int i = 0; i < kNsdfHidden; ++i) {
        const float v = __shfl_sync(0xffffffffu, i < 32 ? gz1a : gz1b, i & 31);
        genc = fmaf(v, bf16_at(S.w1, i, lane, kNsdfHidden), genc);
    }
    const float ge0 = __shfl_sync(0xffffffffu, genc, (2 * lane) & 31);
    const float ge1 = __shfl_sync(0xffffffffu, genc, (2 * lane + 1) & 31);
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (lane < kNsdfLevels) {
        const int l = lane;
        const NsdfCell c = nsdf_cell(l, S.u[r][0], S.u[r][1], S.u[r][2]);
        const float N = (float)(c.n1 - 1);
#pragma unroll
        for (int corner = 0; corner < 8; ++corner) {
            const uint32_t dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
            const float tx = dx ? c.fx : 1.f - c.fx, ty = dy ? c.fy : 1.f - c.fy, tz = dz ? c.fz : 1.f - c.fz;
            const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
            const float2 f = nsdf_feat(table, l, nsdf_entry(l, c.n1, c.i + dx, c.j + dy, c.k + dz));
            const float fe = ge0 * f.x + ge1 * f.y;
            gx = fmaf(sx * ty * tz * N, fe, gx);
            gy = fmaf(tx * sy * tz * N, fe, gy);
            gz = fmaf(tx * ty * sz * N, fe, gz);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, off);
        gy += __shfl_xor_sync(0xffffffffu, gy, off);
        gz += __shfl_xor_sync(0xffffffffu, gz, off);
    }
    return make_float3(1e-3f * gx * o.ninv_ext[0], 1e-3f * gy * o.ninv_ext[1], 1e-3f * gz * o.ninv_ext[2]);
}

__device__ __forceinline__ void set_row(SmemInfer& S, const ObjDev& o, int r, float3 q) {
    S.ext[r] = nsdf_clamp(o, q, S.u[r]);
}

__global__ void __launch_bounds__(kInferThreads) nsdf_eval_kernel(const ObjDev o, const float* pts, int64_t n,
                                                                  float* phi, float* grad, unsigned* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemInfer& S = *reinterpret_cast<SmemInfer*>(smem_raw);
    load_weights(S, o.nweights);
    tc_setup(S);
    const int64_t n_tiles = (n + kRows - 1) / kRows;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t base = tile * kRows;
        if (threadIdx.x < kRows) {
            const int64_t i = base + threadIdx.x;
            float3 q = make_float3(0.f, 0.f, 0.f);
            if (i < n) q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
            else q = make_float3(o.nlo[0], o.nlo[1], o.nlo[2]);
            set_row(S, o, threadIdx.x, q);
        }
        __syncthreads();
        if (!infer_tile(S, o.ntable)) {
            if (threadIdx.x == 0) atomicAdd(err, 1u);
            break;
        }
        __syncthreads();
        if (threadIdx.x < kRows && base + threadIdx.x < n) phi[base + threadIdx.x] = 1e-3f * S.out[threadIdx.x] + S.ext[threadIdx.x];
        if (grad) {
            const int warp = threadIdx.x >> 5;
            for (int r = warp; r < kRows && base + r < n; r += kInferThreads / 32) {
                const float3 gr = row_grad(S, o.ntable, o, r);
                if ((threadIdx.x & 31) == 0) {
                    grad[3 * (base + r)] = gr.x;
                    grad[3 * (base + r) + 1] = gr.y;
                    grad[3 * (base + r) + 2] = gr.z;
                }
            }
        }
        __syncthreads();
    }
    tc_teardown(S);
}

constexpr int kQueryLinks = 32;
constexpr float kNormalStep = 2.5e-4f;  // stencil half-width h of the contact normal (object frame, m)
constexpr float kNeuralBand = 1e-3f;    // the network answers where phi_grid <= R + this (m)

// The object-frame point and scale of taxel i of the item (link records in smem).
__device__ __forceinline__ float3 taxel_point(const StepArgs& a, const float (*rec_s)[kLinkRec], const int* start_s,
                                              int64_t g, int i, float* scale) {
    int l = 0;
    while (i >= start_s[l + 1]) ++l;
    const float* rec = rec_s[l];
    const float x0 = a.x[g], x1 = a.y[g], x2 = a.z[g];
    *scale = rec[38];
    return make_float3(fmaf(rec[0], x0, fmaf(rec[1], x1, fmaf(rec[2], x2, rec[18]))),
                       fmaf(rec[3], x0, fmaf(rec[4], x1, fmaf(rec[5], x2, rec[19]))),
                       fmaf(rec[6], x0, fmaf(rec[7], x1, fmaf(rec[8], x2, rec[20]))));
}

// Per work item whose env holds a learned-SDF object: phi (scaled) of every
// taxel -- the fallback grid's where it puts the probe more than 1 mm beyond
// contact (phi_grid > R + 1 mm), the network's elsewhere -- and, for the
// taxels within 1 um of contact (those the step kernel refines), the contact
// normal by the tetrahedral central difference sum_k v_k phi(q + h v_k) / (4 h),
// v_k = (1,-1,-1), (-1,-1,1), (-1,1,-1), (1,1,1): the analytic gradient of
// the hash encoding jumps at every cell face of its finest levels, the
// stencil averages over a few cells.  Network points go through the
// tensor-core tiles (the near-field taxels, then 32 stencil taxels per tile).
__global__ void __launch_bounds__(kInferThreads) nsdf_step_query_kernel(const StepArgs a, float* phi_out,
                                                                        float* grad_out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemInfer& S = *reinterpret_cast<SmemInfer*>(smem_raw);
    __shared__ float rec_s[kQueryLinks][kLinkRec];
    __shared__ int start_s[kQueryLinks + 1];
    __shared__ float cq_pt[kItemCap][3];   // object-frame points of the near-contact taxels
    __shared__ int64_t cq_g[kItemCap];
    __shared__ int16_t near_i[kItemCap];   // taxels the network answers
    __shared__ int ncq, nnear;
    const Item it = a.items_sorted ? a.items_sorted[blockIdx.x] : a.items[blockIdx.x];
    const int e = it.env, L = a.max_links, lb = it.link_begin, nl = it.link_end - it.link_begin, n = it.n_taxels;
    const int oid = min(max(a.items_sorted ? it.pad : a.obj_id[e], 0), a.n_objects - 1);
    const ObjDev& o = a.objects[oid];
    if (o.kind != TG_OBJ_NEURAL) return;
    const int64_t T = a.n_taxels;
    load_weights(S, o.nweights);
    for (int i = threadIdx.x; i < nl * kLinkRec; i += kInferThreads)
        rec_s[i / kLinkRec][i % kLinkRec] = a.link_rec[(size_t)(e * L + lb + i / kLinkRec) * kLinkRec + i % kLinkRec];
    if ((int)threadIdx.x <= nl) {
        const int base = a.lattice[e * L + lb].env_offset;
        start_s[threadIdx.x] = (int)threadIdx.x < nl ? a.lattice[e * L + lb + threadIdx.x].env_offset - base : n;
    }
    if (threadIdx.x == 0) {
        ncq = 0;
        nnear = 0;
    }
    tc_setup(S);  // (its barrier also publishes the loads above)
    // pass 1a: the fallback grid for every taxel; near-field taxels are listed
    //          (a thread's four taxels at once, so that their loads and
    //          their grid-cell loads are in flight together)
    static_assert(kItemCap <= 4 * kInferThreads, "four taxels per thread cover an item");
    {
        constexpr int U = 4;
        float px[U][3], pr[U];
        int64_t pgid[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kInferThreads;
            pgid[u] = it.taxel_begin + (i < n ? i : 0);
            pr[u] = 0.0f;
            if (i < n) {
                px[u][0] = a.x[pgid[u]];
                px[u][1] = a.y[pgid[u]];
                px[u][2] = a.z[pgid[u]];
                pr[u] = a.R[pgid[u]];
            }
        }
        float pg[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kInferThreads;
            pg[u] = 0.0f;
            if (i < n) {
                int lo = 0, hi = nl - 1;  // link of taxel i: last start <= i
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (start_s[mid] <= i) lo = mid;
                    else hi = mid - 1;
                }
                const float* rec = rec_s[lo];
                const float3 q = make_float3(fmaf(rec[0], px[u][0], fmaf(rec[1], px[u][1], fmaf(rec[2], px[u][2], rec[18]))),
                                             fmaf(rec[3], px[u][0], fmaf(rec[4], px[u][1], fmaf(rec[5], px[u][2], rec[19]))),
                                             fmaf(rec[6], px[u][0], fmaf(rec[7], px[u][1], fmaf(rec[8], px[u][2], rec[20]))));
                pg[u] = rec[38] * grid_phi_fast(o, q);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kInferThreads;
            if (i >= n) break;
            if (pr[u] > 0.0f && !(pg[u] > pr[u] + kNeuralBand)) near_i[atomicAdd(&nnear, 1)] = (int16_t)i;
            else phi_out[pgid[u]] = pg[u];
        }
    }
    __syncthreads();
    bool failed = false;
    // pass 1b: the network for the listed taxels
    const int nn = nnear;
    for (int base = 0; base < nn; base += kRows) {
        if (threadIdx.x < kRows) {
            const int k = base + threadIdx.x;
            float3 q = make_float3(o.nlo[0], o.nlo[1], o.nlo[2]);
            S.gidx[threadIdx.x] = -1;
            S.scale[threadIdx.x] = 0.f;
            if (k < nn) {
                const int i = near_i[k];
                const int64_t g = it.taxel_begin + i;
                float scale;
                q = taxel_point(a, rec_s, start_s, g, i, &scale);
                S.gidx[threadIdx.x] = g;
                S.scale[threadIdx.x] = scale;
            }
            S.q[threadIdx.x][0] = q.x;
            S.q[threadIdx.x][1] = q.y;
            S.q[threadIdx.x][2] = q.z;
            set_row(S, o, threadIdx.x, q);
        }
        __syncthreads();
        if (!infer_tile(S, o.ntable)) {
            failed = true;
            break;
        }
        __syncthreads();
        if (threadIdx.x < kRows) {
            const int64_t g = S.gidx[threadIdx.x];
            if (g >= 0) {
                const float p = S.scale[threadIdx.x] * (1e-3f * S.out[threadIdx.x] + S.ext[threadIdx.x]);
                phi_out[g] = p;
                const float R = a.R[g];
                if (R > 0.0f && p < R + 1e-6f + a.P.rho) {  // (the noisy radius reaches R + rho)
                    const int k = atomicAdd(&ncq, 1);
                    cq_g[k] = g;
                    cq_pt[k][0] = S.q[threadIdx.x][0];
                    cq_pt[k][1] = S.q[threadIdx.x][1];
                    cq_pt[k][2] = S.q[threadIdx.x][2];
                }
            }
        }
        __syncthreads();
    }
    // pass 2: stencil normals, 4 points per near-contact taxel
    const int nc = failed ? 0 : ncq;
    for (int c0 = 0; c0 < nc; c0 += kRows / 4) {
        if (threadIdx.x < kRows) {
            const int t = c0 + (threadIdx.x >> 2), k = threadIdx.x & 3;
            float3 q = make_float3(o.nlo[0], o.nlo[1], o.nlo[2]);
            if (t < nc) {
                const float vx = (k == 0 || k == 3) ? 1.f : -1.f;
                const float vy = (k >= 2) ? 1.f : -1.f;
                const float vz = (k == 1 || k == 3) ? 1.f : -1.f;
                q = make_float3(cq_pt[t][0] + kNormalStep * vx, cq_pt[t][1] + kNormalStep * vy,
                                cq_pt[t][2] + kNormalStep * vz);
            }
            set_row(S, o, threadIdx.x, q);
        }
        __syncthreads();
        if (!infer_tile(S, o.ntable)) {
            failed = true;
            break;
        }
        __syncthreads();
        if (threadIdx.x < kRows / 4) {
            const int t = c0 + threadIdx.x;
            if (t < nc) {
                float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int r = 4 * threadIdx.x + k;
                    const float ph = 1e-3f * S.out[r] + S.ext[r];
                    gx += ((k == 0 || k == 3) ? ph : -ph);
                    gy += ((k >= 2) ? ph : -ph);
                    gz += ((k == 1 || k == 3) ? ph : -ph);
                }
                const float inv = 1.0f / (4.0f * kNormalStep);
                const int64_t g = cq_g[t];
                grad_out[g] = gx * inv;
                grad_out[T + g] = gy * inv;
                grad_out[2 * T + g] = gz * inv;
            }
        }
        __syncthreads();
    }
    if (failed && threadIdx.x == 0) atomicAdd(a.err + 1, 1u);
    tc_teardown(S);
}

// ---------------------------------------------------------------- training
constexpr int kTrainThreads = 128;

struct SmemTrain {
    float w1[kNsdfHidden][kNsdfIn + 1];
    float w2[kNsdfHidden][kNsdfHidden + 1];
    float w3[kNsdfHidden];
    float enc[kRows][kNsdfIn + 1];
    float h1[kRows][kNsdfHidden + 1];   // h1, later g_z1
    float h2[kRows][kNsdfHidden + 1];   // h2, later g_z2
    float gout[kRows];
    float red[kTrainThreads / 32];
};

__global__ void __launch_bounds__(kTrainThreads) nsdf_train_kernel(const ObjDev o, const float* pts,
                                                                   const float* labels, const uint32_t* idx,
                                                                   int64_t n, float* g_part, float* g_table,
                                                                   float* loss_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemTrain& S = *reinterpret_cast<SmemTrain*>(smem_raw);
    const int p = threadIdx.x;
    for (int j = p; j < kNsdfHidden * kNsdfIn; j += kTrainThreads) S.w1[j / kNsdfIn][j % kNsdfIn] = bf16f(o.nweights[j]);
    for (int j = p; j < kNsdfHidden * kNsdfHidden; j += kTrainThreads)
        S.w2[j / kNsdfHidden][j % kNsdfHidden] = bf16f(o.nweights[kNsdfHidden * kNsdfIn + j]);
    if (p < kNsdfHidden) S.w3[p] = bf16f(o.nweights[kNsdfHidden * kNsdfIn + kNsdfHidden * kNsdfHidden + p]);
    const int64_t b = (int64_t)blockIdx.x * kRows + p;
    const bool valid = b < n;
    const int64_t src = valid ? (idx ? (int64_t)idx[b] : b) : 0;
    float u[3];
    {
        const float3 q = make_float3(pts[3 * src], pts[3 * src + 1], pts[3 * src + 2]);
        nsdf_clamp(o, q, u);
    }
    float enc[kNsdfIn];
    nsdf_encode(o.ntable, u, enc);
#pragma unroll
    for (int k = 0; k < kNsdfIn; ++k) S.enc[p][k] = enc[k];
    __syncthreads();
    // forward, one row per thread, FP32
    for (int oo = 0; oo < kNsdfHidden; ++oo) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kNsdfIn; ++k) s = fmaf(S.w1[oo][k], enc[k], s);
        S.h1[p][oo] = fmaxf(s, 0.f);
    }
    float out = 0.f;
    for (int oo = 0; oo < kNsdfHidden; ++oo) {
        float s = 0.f;
#pragma unroll 16
        for (int i = 0; i < kNsdfHidden; ++i) s = fmaf(S.w2[oo][i], S.h1[p][i], s);
        s = fmaxf(s, 0.f);
        S.h2[p][oo] = s;
        out = fmaf(S.w3[oo], s, out);
    }
    const float res = valid ? out - labels[src] : 0.f;
    const float go = res > 0.f ? 1.f : (res < 0.f ? -1.f : 0.f);
    S.gout[p] = go;
    // loss partial
    float l = fabsf(res);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((p & 31) == 0) S.red[p >> 5] = l;
    __syncthreads();
    if (p == 0) {
        float s = 0.f;
        for (int w = 0; w < kTrainThreads / 32; ++w) s += S.red[w];
        loss_part[blockIdx.x] = s;
    }
    float* gp = g_part + (size_t)blockIdx.x * kNsdfWeights;
    // dW3[i] = sum_p gout[p] h2[p][i]
    if (p < kNsdfHidden) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s = fmaf(S.gout[r], S.h2[r][p], s);
        gp[kNsdfHidden * kNsdfIn + kNsdfHidden * kNsdfHidden + p] = s;
    }
    __syncthreads();
    // g_z2 = [h2 > 0] gout W3 (in place, own row)
    for (int oo = 0; oo < kNsdfHidden; ++oo) S.h2[p][oo] = S.h2[p][oo] > 0.f ? go * S.w3[oo] : 0.f;
    __syncthreads();
    {   // dW2[o][i] = sum_p g_z2[p][o] h1[p][i]: thread -> o = p / 2, i in 32 columns
        const int oo = p >> 1, i0 = (p & 1) * 32;
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.f;
        for (int r = 0; r < kRows; ++r) {
            const float gz = S.h2[r][oo];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = fmaf(gz, S.h1[r][i0 + j], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) gp[kNsdfHidden * kNsdfIn + oo * kNsdfHidden + i0 + j] = acc[j];
    }
    __syncthreads();
    // g_z1 = [h1 > 0] W2^T g_z2 (in place, own row)
    for (int i = 0; i < kNsdfHidden; ++i) {
        float s = 0.f;
#pragma unroll 16
        for (int oo = 0; oo < kNsdfHidden; ++oo) s = fmaf(S.h2[p][oo], S.w2[oo][i], s);
        S.h1[p][i] = S.h1[p][i] > 0.f ? s : 0.f;
    }
    __syncthreads();
    {   // dW1[o][k] = sum_p g_z1[p][o] enc[p][k]: thread -> o = p / 2, k in 16 columns
        const int oo = p >> 1, k0 = (p & 1) * 16;
        float acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = 0.f;
        for (int r = 0; r < kRows; ++r) {
            const float gz = S.h1[r][oo];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = fmaf(gz, S.enc[r][k0 + j], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) gp[oo * kNsdfIn + k0 + j] = acc[j];
    }
    // d loss / d enc for this row, then the table entries it read
    if (!valid || go == 0.f) return;
    float genc[kNsdfIn];
#pragma unroll
    for (int k = 0; k < kNsdfIn; ++k) genc[k] = 0.f;
    for (int oo = 0; oo < kNsdfHidden; ++oo) {
        const float gz = S.h1[p][oo];
        if (gz == 0.f) continue;
#pragma unroll
        for (int k = 0; k < kNsdfIn; ++k) genc[k] = fmaf(gz, S.w1[oo][k], genc[k]);
    }
    float2* gt = reinterpret_cast<float2*>(g_table);
#pragma unroll 1
    for (int lv = 0; lv < kNsdfLevels; ++lv) {
        const NsdfCell c = nsdf_cell(lv, u[0], u[1], u[2]);
#pragma unroll
        for (int corner = 0; corner < 8; ++corner) {
            const uint32_t dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
            const float w = (dx ? c.fx : 1.f - c.fx) * (dy ? c.fy : 1.f - c.fy) * (dz ? c.fz : 1.f - c.fz);
            const uint32_t e = nsdf_entry(lv, c.n1, c.i + dx, c.j + dy, c.k + dz);
            atomicAdd(gt + (size_t)lv * kNsdfTable + e, make_float2(w * genc[2 * lv], w * genc[2 * lv + 1]));
        }
    }
}

// g_w[j] = scale * sum over CTAs of g_part[cta][j]
__global__ void nsdf_reduce_kernel(const float* g_part, int n_part, float scale, float* g_w) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kNsdfWeights) return;
    float s = 0.f;
    for (int b = 0; b < n_part; ++b) s += g_part[(size_t)b * kNsdfWeights + j];
    g_w[j] = s * scale;
}

__global__ void nsdf_sample_kernel(uint64_t seed, uint32_t step, int64_t n_points, int32_t batch, uint32_t* idx) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const uint4 w = draw(seed, (uint64_t)b, step, kTagNsdfBatch);
    idx[b] = (uint32_t)(((uint64_t)w.x * (uint64_t)n_points) >> 32);
}

__device__ __forceinline__ uint16_t to_bf16_bits(float x) {
    const __nv_bfloat16 v = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&v);
}

// Adam over the weights (j < 6208) and the table entries (two features each).
__global__ void nsdf_adam_kernel(float* master, float* m, float* v, const float* g_w, const float* g_table,
                                 uint16_t* weights, uint32_t* table, float lr, float c1, float c2, float gscale) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float b1 = 0.9f, b2 = 0.99f, eps = 1e-15f;
    if (j < kNsdfWeights) {
        const float g = g_w[j] * gscale;
        const float mm = b1 * m[j] + (1.f - b1) * g, vv = b2 * v[j] + (1.f - b2) * g * g;
        m[j] = mm;
        v[j] = vv;
        const float th = master[j] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        master[j] = th;
        weights[j] = to_bf16_bits(th);
        return;
    }
    const int64_t e = j - kNsdfWeights;
    if (e >= kNsdfTableEntries) return;
    float th[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const int64_t k = kNsdfWeights + 2 * e + f;
        const float g = g_table[2 * e + f] * gscale;
        const float mm = b1 * m[k] + (1.f - b1) * g, vv = b2 * v[k] + (1.f - b2) * g * g;
        m[k] = mm;
        v[k] = vv;
        th[f] = master[k] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        master[k] = th[f];
    }
    const __half2 h = __floats2half2_rn(th[0], th[1]);
    table[e] = *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void nsdf_init_kernel(uint64_t seed, float* master, float* m, float* v, uint16_t* weights,
                                 uint32_t* table) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < kNsdfWeights) {
        const float lim = j < kNsdfHidden * kNsdfIn
                              ? sqrtf(6.f / (kNsdfIn + kNsdfHidden))
                              : (j < kNsdfHidden * kNsdfIn + kNsdfHidden * kNsdfHidden ? sqrtf(6.f / (2 * kNsdfHidden))
                                                                                      : sqrtf(6.f / (kNsdfHidden + 1)));
        const float th = lim * (2.f * u24(draw(seed, (uint64_t)j, 0u, kTagNsdfInit).x) - 1.f);
        master[j] = th;
        m[j] = 0.f;
        v[j] = 0.f;
        weights[j] = to_bf16_bits(th);
        return;
    }
    const int64_t e = j - kNsdfWeights;
    if (e >= kNsdfTableEntries) return;
    const uint4 w = draw(seed, (uint64_t)j, 0u, kTagNsdfInit);
    float th[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const int64_t k = kNsdfWeights + 2 * e + f;
        th[f] = 1e-4f * (2.f * u24(f ? w.y : w.x) - 1.f);
        master[k] = th[f];
        m[k] = 0.f;
        v[k] = 0.f;
    }
    const __half2 h = __floats2half2_rn(th[0], th[1]);
    table[e] = *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void nsdf_sync_masters_kernel(float* master, float* m, float* v, const uint16_t* weights,
                                         const uint32_t* table) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < kNsdfWeights) {
        master[j] = bf16f(weights[j]);
        m[j] = v[j] = 0.f;
        return;
    }
    const int64_t e = j - kNsdfWeights;
    if (e >= kNsdfTableEntries) return;
    const uint32_t t = table[e];
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&t));
    master[kNsdfWeights + 2 * e] = f.x;
    master[kNsdfWeights + 2 * e + 1] = f.y;
    m[kNsdfWeights + 2 * e] = m[kNsdfWeights + 2 * e + 1] = 0.f;
    v[kNsdfWeights + 2 * e] = v[kNsdfWeights + 2 * e + 1] = 0.f;
}

constexpr int64_t kParamCount = kNsdfWeights + 2 * kNsdfTableEntries;
constexpr int64_t kUpdateCount = kNsdfWeights + kNsdfTableEntries;  // Adam threads

// shared-memory limits of the three kernels on the current device (per device, once)
cudaError_t configure() {
    cudaError_t e = raise_smem_limit((const void*)nsdf_eval_kernel, sizeof(SmemInfer));
    if (e == cudaSuccess) e = raise_smem_limit((const void*)nsdf_step_query_kernel, sizeof(SmemInfer));
    if (e == cudaSuccess) e = raise_smem_limit((const void*)nsdf_train_kernel, sizeof(SmemTrain));
    return e;
}

}  // namespace

cudaError_t nsdf_alloc(NsdfNet* n) {
    cudaError_t e = cudaMalloc(&n->table, sizeof(uint32_t) * kNsdfTableEntries);
    if (e == cudaSuccess) e = cudaMalloc(&n->weights, sizeof(uint16_t) * kNsdfWeights);
    if (e == cudaSuccess) e = cudaMalloc(&n->master, sizeof(float) * kParamCount);
    if (e == cudaSuccess) e = cudaMalloc(&n->adam_m, sizeof(float) * kParamCount);
    if (e == cudaSuccess) e = cudaMalloc(&n->adam_v, sizeof(float) * kParamCount);
    if (e == cudaSuccess) e = configure();
    n->adam_t = 0;
    return e;
}

void nsdf_free(NsdfNet* n) {
    cudaFree(n->table);
    cudaFree(n->weights);
    cudaFree(n->master);
    cudaFree(n->adam_m);
    cudaFree(n->adam_v);
    n->table = nullptr;
    n->weights = nullptr;
    n->master = n->adam_m = n->adam_v = nullptr;
}

cudaError_t nsdf_init(NsdfNet* n, uint64_t seed, cudaStream_t s) {
    nsdf_init_kernel<<<(unsigned)((kUpdateCount + 255) / 256), 256, 0, s>>>(seed, n->master, n->adam_m, n->adam_v,
                                                                           n->weights, n->table);
    n->adam_t = 0;
    return cudaGetLastError();
}

cudaError_t nsdf_sync_masters(NsdfNet* n, cudaStream_t s) {
    nsdf_sync_masters_kernel<<<(unsigned)((kUpdateCount + 255) / 256), 256, 0, s>>>(n->master, n->adam_m, n->adam_v,
                                                                                   n->weights, n->table);
    n->adam_t = 0;
    return cudaGetLastError();
}

cudaError_t launch_nsdf_eval(const ObjDev& o, const float* pts, int64_t n, float* phi, float* grad, unsigned* err,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = configure();
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + kRows - 1) / kRows;
    const unsigned grid = (unsigned)(tiles < 152 * 3 ? tiles : 152 * 3);
    nsdf_eval_kernel<<<grid, kInferThreads, sizeof(SmemInfer), s>>>(o, pts, n, phi, grad, err);
    return cudaGetLastError();
}

cudaError_t launch_nsdf_step_query(const StepArgs& a, int n_items, float* phi, float* grad, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    cudaError_t e = configure();
    if (e != cudaSuccess) return e;
    nsdf_step_query_kernel<<<n_items, kInferThreads, sizeof(SmemInfer), s>>>(a, phi, grad);
    return cudaGetLastError();
}

int nsdf_train_ctas(int64_t n) { return (int)((n + kRows - 1) / kRows); }

cudaError_t launch_nsdf_train_step(const ObjDev& o, const float* pts, const float* labels, const uint32_t* idx,
                                   int64_t n, float* g_part, float* g_w, float* g_table, float* loss_part,
                                   cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = configure();
    if (e != cudaSuccess) return e;
    const int ctas = nsdf_train_ctas(n);
    nsdf_train_kernel<<<ctas, kTrainThreads, sizeof(SmemTrain), s>>>(o, pts, labels, idx, n, g_part, g_table,
                                                                     loss_part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nsdf_reduce_kernel<<<(kNsdfWeights + 255) / 256, 256, 0, s>>>(g_part, ctas, 1.0f, g_w);
    return cudaGetLastError();
}

cudaError_t launch_nsdf_sample(uint64_t seed, uint32_t step, int64_t n_points, int32_t batch, uint32_t* idx,
                               cudaStream_t s) {
    nsdf_sample_kernel<<<(batch + 255) / 256, 256, 0, s>>>(seed, step, n_points, batch, idx);
    return cudaGetLastError();
}

cudaError_t launch_nsdf_adam(NsdfNet* n, const float* g_w, const float* g_table, float lr, float gscale,
                             cudaStream_t s) {
    n->adam_t += 1;
    const double c1 = 1.0 - std::pow(0.9, (double)n->adam_t), c2 = 1.0 - std::pow(0.99, (double)n->adam_t);
    nsdf_adam_kernel<<<(unsigned)((kUpdateCount + 255) / 256), 256, 0, s>>>(
        n->master, n->adam_m, n->adam_v, g_w, g_table, n->weights, n->table, lr, (float)c1, (float)c2, gscale);
    return cudaGetLastError();
}

}  // namespace tg
