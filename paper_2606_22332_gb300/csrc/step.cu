// step.cu -- the fused per-taxel sensor step (Appendix A) and the episode
// reset.
//
// One work item per CTA at a time: a run of whole links of one env (at most
// kItemCap taxels, kItemMaxLinks links); items are taken in an object-sorted
// order so that concurrently running CTAs share one or two SDF grids in L2.
// Either every item gets its own CTA (grid schedule) or a resident grid takes
// items from an atomic counter (persistent schedule); the autotuner picks.  Per-taxel
// arrays are SoA in HBM, read and written coalesced with streaming
// (evict-first) cache operators.
//   phase A1 per taxel: FP32 object-frame query; taxels clear of the surface
//            finish here (depth 0, no contact, no force), the others queue
//   phase A2 queued near-contact taxels, compacted onto whole warps:
//            compensated query point and SDF, depth, Schmitt bit, force/torque
//            (position, radius and flags come from shared memory, where A1
//            left them)
//   phase N  per taxel: noise state (gain, hysteresis, depth base noise, dead)
//            with all state loads independent of the geometry; alongside it,
//            per (link, quantity), the clean force/torque sums and clean
//            contact counts (their inputs are final after A2)
//   phase B  per taxel: 3x3 crosstalk from shared memory, drift/white noise,
//            quantisation, dead override -> noisy force/torque; alongside it
//            the agg_force sums and noisy contact counts (final after N)
//   phase C2 per (link, quantity, half): noisy force/torque sums
// Link sums are compensated (Kahan) sums in a fixed order (link_sum), so
// results are deterministic run to run.
#include <cstdint>

#include "step_common.cuh"

namespace tg {

struct SmemStep {
    float rec[kItemMaxLinks][kLinkRec];
    int start[kItemMaxLinks + 1];       // first taxel of each link, relative to the item
    int rows[kItemMaxLinks], cols[kItemMaxLinks], wrap[kItemMaxLinks];
    ObjDev obj;
    float hx[6][kItemCap];              // force/torque after gain + hysteresis (A1-A2: near-taxel inputs)
    float fc[6][kItemCap];              // clean force/torque, later noisy force/torque
    // 0 clean depth, 1 noisy depth (with probe-radius noise, until phase N,
    // the perturbed radius's depth), 2-4 probe normal (from phase N; in A1-A2
    // rows 2-3 hold the near-contact queue); agg_force terms d n are formed
    // in the link sums
    float dn[5][kItemCap];
    uint8_t bits[kItemCap];             // BIT_* flags
    int nq;
    unsigned int slot;                  // persistent schedule: the item being run
    uint32_t episode;                   // the env's episode counter
    int rdelay;                         // read delay of the env at this step (steps)
    // when every link of the item has the same lattice (rows x cols, wrap)
    // and holds rows * cols taxels: that taxel count (else 0), the lattice,
    // and 1/count, 1/cols for the index arithmetic below
    int uni_len, uni_rows, uni_cols, uni_wrap;
    float uni_inv_len, uni_inv_cols;
};

// three items' shared memory (and the 1 KB the SM reserves per CTA) fit in
// the SM's 228 KB, for the 384 x 3 shape
static_assert(3 * (sizeof(SmemStep) + 1024) <= 228 * 1024, "three step-kernel CTAs per SM");

// L2 prefetch of the SDF grid of the object whose run of items begins two
// waves of resident CTAs after `slot` in the object-sorted order.  Each env
// queries cells no other env touches, so without it every query's cell is a
// random HBM sector whose latency the geometry phase waits for; with it the
// grid streams into L2 (evict-last) once per object and step, ahead of the
// CTAs that read it.  A hint only: results do not depend on it.
constexpr uint32_t kGridPrefetchChunk = 64 * 1024;

__device__ __forceinline__ void prefetch_grid_ahead(const StepArgs& a, int slot) {
    const int t = slot + 2 * a.resident_ctas;  // one wave ahead measured 1 % slower, half a wave 3 %
    if (t <= 0 || t >= a.n_items) return;
    const int k = a.items_sorted[t].pad;
    if (k == a.items_sorted[t - 1].pad) return;
    const ObjDev& o = a.objects[min(max(k, 0), a.n_objects - 1)];
    if ((o.kind != TG_OBJ_GRID && o.kind != TG_OBJ_NEURAL) || !o.cells) return;
    const uint64_t bytes = (uint64_t)(o.dims[0] - 1) * (uint64_t)(o.dims[1] - 1) * (uint64_t)(o.dims[2] - 1) *
                           (o.fp16 ? 16u : 32u);
    const char* base = static_cast<const char*>(o.cells);
    const uint64_t pol = l2_evict_last_policy();
    for (uint64_t off = 0; off < bytes; off += kGridPrefetchChunk) {
        const uint32_t len = (uint32_t)min((uint64_t)kGridPrefetchChunk, bytes - off);  // a multiple of 16
        asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(base + off), "r"(len),
                     "l"(pol)
                     : "memory");
    }
}

// One work item: every phase of the step for its taxels.  GRID: the form
// for scenes whose objects are all plain SDF grids (no kind dispatch, no
// query kernel ahead of this one).
template <int NT, bool RADIUS, bool GRID>
__device__ __forceinline__ void step_item(const StepArgs& a, SmemStep& S, int slot, uint32_t step) {
    const Item it = a.items_sorted ? a.items_sorted[slot] : a.items[slot];
    const int e = it.env;
    const int L = a.max_links;
    const int lb = it.link_begin;
    const int nl = it.link_end - it.link_begin;
    const int n = it.n_taxels;
    const int tid = threadIdx.x;

    // ---- prologue: link records (the item's links are consecutive: one
    //      contiguous block of 16-byte vectors), lattice, object
    static_assert(kLinkRec % 4 == 0 && kItemCap <= 1024, "vector copy of link records; uni_div range");
    {
        const float4* src = reinterpret_cast<const float4*>(a.link_rec + (size_t)(e * L + lb) * kLinkRec);
        float4* dst = reinterpret_cast<float4*>(&S.rec[0][0]);
        for (int v = tid; v < nl * (kLinkRec / 4); v += NT) dst[v] = src[v];
    }
    if (tid < 32) {  // uniform-lattice test over the item's (at most 32) links
        const bool act = tid < nl;
        LinkLattice lat{};
        if (act) lat = a.lattice[e * L + lb + tid];
        int next = __shfl_down_sync(0xffffffffu, lat.env_offset, 1);
        if (tid == nl - 1) next = a.lattice[e * L + lb].env_offset + n;
        const int cnt = act ? next - lat.env_offset : 0;
        const int r0 = __shfl_sync(0xffffffffu, (int)lat.rows, 0), c0 = __shfl_sync(0xffffffffu, (int)lat.cols, 0);
        const int w0 = __shfl_sync(0xffffffffu, (int)lat.wrap, 0);
        const bool same = !act || ((int)lat.rows == r0 && (int)lat.cols == c0 && (int)lat.wrap == w0 && cnt == r0 * c0);
        const bool uni = __all_sync(0xffffffffu, same) && r0 * c0 > 0;
        if (tid == 0) {
            S.uni_len = uni ? r0 * c0 : 0;
            S.uni_rows = r0;
            S.uni_cols = c0;
            S.uni_wrap = w0;
            S.uni_inv_len = uni ? 1.0f / (float)(r0 * c0) : 0.0f;
            S.uni_inv_cols = uni ? 1.0f / (float)c0 : 0.0f;
        }
    }
    if (tid <= nl) {
        // the lattice table holds each link's first taxel relative to the env
        const int base = a.lattice[e * L + lb].env_offset;
        if (tid < nl) {
            const LinkLattice lat = a.lattice[e * L + lb + tid];
            S.rows[tid] = lat.rows;
            S.cols[tid] = lat.cols;
            S.wrap[tid] = lat.wrap;
            S.start[tid] = lat.env_offset - base;
        } else {
            S.start[nl] = n;
        }
    }
    // the object descriptor, 16 bytes per thread of warp 1
    static_assert(sizeof(ObjDev) % 16 == 0 && sizeof(ObjDev) / 16 <= 32 && NT >= 64, "object copy by one warp");
    if (tid >= 32 && tid < 32 + (int)(sizeof(ObjDev) / 16)) {
        // the sorted copy of the items carries the object (one load fewer
        // on the prologue's dependent chain)
        int oid = a.items_sorted ? it.pad : a.obj_id[e];
        oid = min(max(oid, 0), a.n_objects - 1);
        reinterpret_cast<uint4*>(&S.obj)[tid - 32] = reinterpret_cast<const uint4*>(a.objects + oid)[tid - 32];
    }
    if (tid == 0) {
        S.nq = 0;
        S.episode = a.episode[e];
        S.rdelay = a.P.ring_k > 1 ? read_delay(a.P, (uint64_t)(a.env_gid0 + e), step) : 0;
    }
    __syncthreads();

    const uint32_t ep = S.episode;
    const ObjDev& obj = S.obj;
    // near-contact taxels for phase A2 (rows 2-3 of dn are free until phase N)
    int16_t* queue = reinterpret_cast<int16_t*>(&S.dn[2][0]);
    static_assert(2 * kItemCap * sizeof(float) >= kItemCap * sizeof(int16_t), "queue fits");

    // ---- phase A1 (geometry): FP32 query of every taxel; those clear of the
    //      surface finish here, those within 1 um of contact are queued.  A
    //      thread takes its taxels in pairs so both load chains (taxel, then
    //      grid cell) are in flight together.
    int l = 0;
    for (int i0 = tid; i0 < n; i0 += 2 * NT) {
        const int i1 = i0 + NT;
        const bool has1 = i1 < n;
        const tidx g0 = (tidx)(it.taxel_begin + i0), g1 = (tidx)(it.taxel_begin + (has1 ? i1 : i0));
        const float R0 = __ldcs(a.R + g0), R1 = has1 ? __ldcs(a.R + g1) : 0.0f;
        const float x00 = __ldcs(a.x + g0), x01 = __ldcs(a.y + g0), x02 = __ldcs(a.z + g0);
        const float x10 = __ldcs(a.x + g1), x11 = __ldcs(a.y + g1), x12 = __ldcs(a.z + g1);
        const uint8_t fl0 = __ldcs(a.flags + g0), fl1 = __ldcs(a.flags + g1);
        int l0, l1;
        if (S.uni_len) {
            l0 = uni_div(i0, S.uni_inv_len);
            l1 = has1 ? uni_div(i1, S.uni_inv_len) : l0;
        } else {
            while (i0 >= S.start[l + 1]) ++l;
            l0 = l1 = l;
            if (has1)
                while (i1 >= S.start[l1 + 1]) ++l1;
        }
        float phi0 = 0.0f, phi1 = 0.0f;
        if (!GRID && phi_precomputed(obj, a.P)) {  // from the learned-SDF or raycast query kernel
            if (R0 > 0.0f) phi0 = a.nq_phi[g0];
            if (R1 > 0.0f) phi1 = a.nq_phi[g1];
        } else {
            if (R0 > 0.0f) phi0 = fast_query<GRID>(S.rec[l0], obj, x00, x01, x02);
            if (R1 > 0.0f) phi1 = fast_query<GRID>(S.rec[l1], obj, x10, x11, x12);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (u == 1 && !has1) break;
            const int i = u ? i1 : i0;
            const tidx g = u ? g1 : g0;
            const float R = u ? R1 : R0, phi = u ? phi1 : phi0;
            if (R > 0.0f && !isfinite(phi)) atomicAdd(a.err, 1u);
            // (with probe-radius noise the noisy readout's radius reaches R + rho)
            if (R > 0.0f && phi < R + 1e-6f + (RADIUS ? a.P.rho : 0.0f)) {
                queue[atomicAdd(&S.nq, 1)] = (int16_t)i;
                // A2's inputs, kept on chip (hx is not used before phase N)
                float* st = &S.hx[0][0];
                st[i] = u ? x10 : x00;
                st[kItemCap + i] = u ? x11 : x01;
                st[2 * kItemCap + i] = u ? x12 : x02;
                st[3 * kItemCap + i] = R;
                st[4 * kItemCap + i] = __uint_as_float(u ? fl1 : fl0);
                continue;
            }
            S.bits[i] = clear_taxel(a, g, R, u ? fl1 : fl0, !GRID && raycast_obj(obj, a.P) ? R : phi);
#pragma unroll
            for (int c = 0; c < 6; ++c) S.fc[c][i] = 0.f;
            S.dn[0][i] = 0.f;
        }
        l = l1;
    }
    __syncthreads();

    // ---- phase A2: near-contact taxels, compacted onto whole warps
    const int nq = S.nq;
    for (int k = tid; k < nq; k += NT) {
        const int i = queue[k];
        int lo = 0, hi = nl - 1;  // link of taxel i: last start <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.start[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const float* st = &S.hx[0][0];
        const CleanReading cr = refine_taxel<RADIUS, GRID>(a, S.rec[lo], obj, (tidx)(it.taxel_begin + i), st[i], st[kItemCap + i],
                                             st[2 * kItemCap + i], st[3 * kItemCap + i],
                                             (uint8_t)__float_as_uint(st[4 * kItemCap + i]), step);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            S.fc[c][i] = cr.f[c];
            S.fc[3 + c][i] = cr.tq[c];
        }
        S.dn[0][i] = cr.d;
        S.bits[i] = cr.bits;
        if constexpr (RADIUS) {  // the noisy chain's depth and force, for phase N (slots free until then)
            S.dn[1][i] = cr.dn;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                S.hx[c][i] = cr.fn[c];
                S.hx[3 + c][i] = cr.tqn[c];
            }
        }
    }
    __syncthreads();

    // ---- phase N: noise state of every taxel (independent state loads);
    //      the clean force/torque sums and clean counts (final after A2) run
    //      here too, while a thread's first taxel's state loads are in flight
    {
        const int ntask = nl * 7;
        int i = tid;
        NoiseIn s0{};
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
        uint8_t b0 = 0;
        tidx g0 = 0;
        if (i < n) {
            g0 = (tidx)(it.taxel_begin + i);
            b0 = S.bits[i];
            if (b0 & BIT_ACTIVE) {
                s0 = noise_load(a, g0);
                m0 = __ldcs(a.nx + g0); m1 = __ldcs(a.ny + g0); m2 = __ldcs(a.nz + g0);
            }
        }
        for (int t = tid; t < ntask; t += NT) {
            const int ll = t % nl, q = t / nl;
            link_quantity(a, S, S.fc, (size_t)(e * L + lb + ll), S.start[ll], S.start[ll + 1], q < 6 ? q : 12);
        }
        if (i < n) {
            if (b0 & BIT_ACTIVE) noise_apply<RADIUS>(a, S, i, g0, ep, step, b0, m0, m1, m2, s0);
            else noise_state_filler(a, S, i, g0);
        }
        for (i = tid + NT; i < n; i += NT) {
            const tidx g = (tidx)(it.taxel_begin + i);
            const uint8_t bits = S.bits[i];
            if (bits & BIT_ACTIVE)
                noise_state<RADIUS>(a, S, i, g, ep, step, bits, __ldcs(a.nx + g), __ldcs(a.ny + g), __ldcs(a.nz + g));
            else noise_state_filler(a, S, i, g);
        }
    }
    __syncthreads();

    // ---- phase B: crosstalk, base noise, dead override -> noisy force/torque
    //      (written over the clean values in fc, summed in phase N); the
    //      agg_force sums and noisy counts (final after N) run here too
    l = 0;
    {
        const int ntask = nl * 7;
        for (int t = tid; t < ntask; t += NT) {
            const int ll = t % nl, q = t / nl;
            link_quantity(a, S, S.fc, (size_t)(e * L + lb + ll), S.start[ll], S.start[ll + 1], q < 6 ? 6 + q : 13);
        }
        if (a.items_sorted && tid == NT - 1) prefetch_grid_ahead(a, slot);
    }
    for (int i = tid; i < n; i += NT) {
        if (S.uni_len) {
            const int base = uni_div(i, S.uni_inv_len) * S.uni_len;
            const int j = i - base;
            const int r = uni_div(j, S.uni_inv_cols);
            noisy_ft(a, S, S.fc, i, (tidx)(it.taxel_begin + i), ep, step, S.bits[i], base, r, j - r * S.uni_cols,
                     S.uni_rows, S.uni_cols, S.uni_wrap != 0);
            continue;
        }
        while (i >= S.start[l + 1]) ++l;
        const int j = i - S.start[l], cols = S.cols[l];
        const int r = j / cols;
        noisy_ft(a, S, S.fc, i, (tidx)(it.taxel_begin + i), ep, step, S.bits[i], S.start[l], r, j - r * cols, S.rows[l],
                 cols, S.wrap[l] != 0);
    }
    __syncthreads();

    // ---- phase C2: noisy force/torque link sums, two threads (adjacent
    //      lanes) per (link, quantity), a half of the link each, joined
    //      through a shuffle as link_sum_halves joins them
    static_assert(kItemMaxLinks * 12 <= NT, "one pass of C2");
    if (tid < nl * 12) {
        const int task = tid >> 1, half = tid & 1;
        const int ll = task % nl, q = task / nl;
        const int s0 = S.start[ll], s1 = S.start[ll + 1], mid = link_mid(s0, s1);
        const Acc h = link_acc(S.fc[q], half ? mid : s0, half ? s1 : mid);
        // (pairs are whole: nl * 12 is even, and a pair's lanes are adjacent)
        const unsigned m = __activemask();
        const float os = __shfl_down_sync(m, h.s, 1), oc = __shfl_down_sync(m, h.c, 1);
        if (!half) a.link_out[(size_t)(e * L + lb + ll) * kLinkOut + 6 + q] = acc_join(h, Acc{os, oc});
    }
}

// Grid schedule: CTA b runs item slot b.  Persistent schedule: a grid sized
// to the resident CTAs takes item slots from an atomic counter (zeroed
// before the launch) until none are left.
template <int NT, int MINB, bool PERSISTENT, bool RADIUS, bool GRID>
__global__ void __launch_bounds__(NT, MINB) step_kernel(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemStep& S = *reinterpret_cast<SmemStep*>(smem_raw);
    const uint32_t step = a.step_from_ctl ? a.ctl->step : a.step;
    if constexpr (!PERSISTENT) {
        step_item<NT, RADIUS, GRID>(a, S, blockIdx.x, step);
    } else {
        for (;;) {
            if (threadIdx.x == 0) S.slot = atomicAdd(&a.ctl->counter, 1u);
            __syncthreads();
            const int slot = (int)S.slot;
            if (slot >= a.n_items) break;
            step_item<NT, RADIUS, GRID>(a, S, slot, step);
            __syncthreads();  // shared memory is reused by the next item
        }
    }
}

// Reset of the envs whose mask byte is set: dead mask drawn from
// (seed, taxel id, episode), hysteresis / drift / Schmitt state zeroed, and
// the clean depth and force/torque outputs zeroed (with prev_out they are
// the hysteresis x_{t-1}).
__global__ void reset_kernel(const StepArgs a, const uint8_t* env_mask, uint32_t episode, uint32_t* episode_arr) {
    const Item it = a.items[blockIdx.x];
    const int e = it.env;
    if (env_mask && !env_mask[e]) return;
    if (threadIdx.x == 0) episode_arr[e] = episode;
    const int64_t T = a.n_taxels;
    for (int i = threadIdx.x; i < it.n_taxels; i += blockDim.x) {
        const tidx g = (tidx)(it.taxel_begin + i);
        const uint64_t gid = (uint64_t)(a.gid0 + g);
        const bool active = a.R[g] > 0.0f;
        bool dead = false;
        if (active) dead = bernoulli24(draw(a.P.seed, gid, episode, TAG_EPISODE).x, a.P.dead_threshold24);
        a.flags[g] = dead ? 2u : 0u;
        for (int c = 0; c < 8; ++c) {
            a.hyst_prev[c * T + g] = 0.f;
            a.hyst_xi[c * T + g] = 0.f;
            a.drift[c * T + g] = 0.f;
        }
        a.depth_clean[g] = 0.f;
        for (int c = 0; c < 6; ++c) a.ft_clean[c * T + g] = 0.f;
        for (int c = 0; a.P.ring_k > 1 && c < a.P.ring_k * 8; ++c) a.ring[c * T + g] = 0.f;
    }
}

__global__ void unpack_contact_kernel(const uint8_t* flags, int64_t n, int bit, uint8_t* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (flags[i] >> bit) & 1u;
}

// Every form of the step kernel for one CTA shape: PERSISTENT x RADIUS x GRID.
template <int NT, int MINB>
struct StepForms {
    static const void* fn(int k) {
        const void* f[8] = {(const void*)step_kernel<NT, MINB, false, false, false>,
                            (const void*)step_kernel<NT, MINB, true, false, false>,
                            (const void*)step_kernel<NT, MINB, false, true, false>,
                            (const void*)step_kernel<NT, MINB, true, true, false>,
                            (const void*)step_kernel<NT, MINB, false, false, true>,
                            (const void*)step_kernel<NT, MINB, true, false, true>,
                            (const void*)step_kernel<NT, MINB, false, true, true>,
                            (const void*)step_kernel<NT, MINB, true, true, true>};
        return f[k];
    }
    static void launch(const StepArgs& a, int blocks, bool persistent, size_t smem, cudaStream_t s) {
        const bool r = a.P.rho > 0.0f, g = a.all_grid != 0;
#define TG_STEP_LAUNCH(P, R, G) step_kernel<NT, MINB, P, R, G><<<blocks, NT, smem, s>>>(a)
        if (persistent) {
            if (r) { if (g) TG_STEP_LAUNCH(true, true, true); else TG_STEP_LAUNCH(true, true, false); }
            else { if (g) TG_STEP_LAUNCH(true, false, true); else TG_STEP_LAUNCH(true, false, false); }
        } else {
            if (r) { if (g) TG_STEP_LAUNCH(false, true, true); else TG_STEP_LAUNCH(false, true, false); }
            else { if (g) TG_STEP_LAUNCH(false, false, true); else TG_STEP_LAUNCH(false, false, false); }
        }
#undef TG_STEP_LAUNCH
    }
};
static_assert(kStepShapeThreads[0] == 512 && kStepShapeBlocks[0] == 2 && kStepShapeThreads[1] == 384 &&
                  kStepShapeBlocks[1] == 3, "step kernel shapes");
using StepForms0 = StepForms<512, 2>;
using StepForms1 = StepForms<384, 3>;

cudaError_t configure_step_kernels() {
    const int smem = (int)sizeof(SmemStep);
    for (int k = 0; k < 8; ++k)
        for (int shape = 0; shape < kStepShapes; ++shape) {
            const void* f = shape == 0 ? StepForms0::fn(k) : StepForms1::fn(k);
            cudaError_t err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            // 384 x 3: the whole carveout, so that three items' shared memory
            // fits on an SM (512 x 2 keeps the rest of the SM's 256 KB as L1)
            if (err == cudaSuccess && shape == 1)
                err = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared);
            if (err != cudaSuccess) return err;
        }
    return cudaSuccess;
}

int step_kernel_resident_ctas(int shape) {
    int dev = 0, sms = 0, per_sm = 0;
    if (shape < 0 || shape >= kStepShapes) return 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const void* f = shape == 0 ? StepForms0::fn(1) : StepForms1::fn(1);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kStepShapeThreads[shape], sizeof(SmemStep)) !=
        cudaSuccess)
        return 0;
    return sms * per_sm;
}

cudaError_t launch_step(const StepArgs& a, int n_items, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    if (a.shape < 0 || a.shape >= kStepShapes) return cudaErrorInvalidValue;
    const size_t smem = sizeof(SmemStep);
    int blocks = n_items;
    if (a.persistent) {
        if (!a.ctl || a.n_items != n_items) return cudaErrorInvalidValue;
        const int ctas = a.resident_ctas;
        if (ctas <= 0) return cudaErrorInvalidConfiguration;
        cudaError_t err = cudaMemsetAsync(&a.ctl->counter, 0, sizeof(uint32_t), s);
        if (err != cudaSuccess) return err;
        blocks = min(ctas, n_items);
    }
    if (a.shape == 0) StepForms0::launch(a, blocks, a.persistent != 0, smem, s);
    else StepForms1::launch(a, blocks, a.persistent != 0, smem, s);
    return cudaGetLastError();
}

__global__ void set_ctl_kernel(StepCtl* ctl, StepCtl value) { *ctl = value; }

// last node of a captured step: the next replay runs the next step
__global__ void advance_ctl_kernel(StepCtl* ctl) {
    ctl->step += 1u;
    ctl->replay += 1u;
}

cudaError_t launch_set_ctl(StepCtl* ctl, StepCtl value, cudaStream_t s) {
    set_ctl_kernel<<<1, 1, 0, s>>>(ctl, value);
    return cudaGetLastError();
}

cudaError_t launch_advance_ctl(StepCtl* ctl, cudaStream_t s) {
    advance_ctl_kernel<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

// Counting sort of the work items by the object their env holds this step:
// CTAs launched together then read one or two object grids, which stay in L2
// while the per-taxel state streams past.  Order within an object is
// arbitrary; every item's result is independent of it.
// Counting sort of the items by the object their env holds this step, into
// a copy of the items (so a CTA reads its item with one load).  One CTA: the
// items' objects are read once, a thread's items at once (their dependent
// loads in flight together), and kept in shared memory when they fit
// (cache != 0); the order within an object is that of the atomics (results do
// not depend on it: every item is computed the same wherever it runs).
__global__ void order_items_kernel(const Item* items, int n_items, const int32_t* obj_id, int n_objects, int cache,
                                   Item* sorted) {
    extern __shared__ int cnt[];  // [n_objects], then [n_items] uint16 objects when cached
    uint16_t* oc = reinterpret_cast<uint16_t*>(cnt + n_objects);
    for (int k = threadIdx.x; k < n_objects; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    constexpr int U = 8;
    for (int i0 = threadIdx.x; i0 < n_items; i0 += U * blockDim.x) {
        int env[U], obj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            env[u] = i < n_items ? items[i].env : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) obj[u] = env[u] >= 0 ? obj_id[env[u]] : 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= n_items) break;
            const int k = min(max(obj[u], 0), n_objects - 1);
            atomicAdd(&cnt[k], 1);
            if (cache) oc[i] = (uint16_t)k;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < n_objects; ++k) {
            const int c = cnt[k];
            cnt[k] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_items; i += blockDim.x) {
        Item it = items[i];
        const int k = cache ? (int)oc[i] : min(max(obj_id[it.env], 0), n_objects - 1);
        it.pad = k;  // the env's object this step
        sorted[atomicAdd(&cnt[k], 1)] = it;
    }
}

cudaError_t launch_order_items(const Item* items, int n_items, const int32_t* obj_id, int n_objects, Item* sorted,
                               cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    constexpr size_t kCap = 160 * 1024;
    const size_t base = (size_t)n_objects * sizeof(int);
    const size_t with_cache = base + (size_t)n_items * sizeof(uint16_t);
    const int cache = with_cache <= kCap && n_objects <= 65535 ? 1 : 0;
    const size_t smem = cache ? with_cache : base;
    if (smem > 48 * 1024) {
        const cudaError_t e = raise_smem_limit((const void*)order_items_kernel, kCap);
        if (e != cudaSuccess) return e;
    }
    order_items_kernel<<<1, 1024, smem, s>>>(items, n_items, obj_id, n_objects, cache, sorted);
    return cudaGetLastError();
}

cudaError_t launch_reset(const StepArgs& a, int n_items, const uint8_t* env_mask, uint32_t episode,
                         uint32_t* episode_arr, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    reset_kernel<<<n_items, 256, 0, s>>>(a, env_mask, episode, episode_arr);
    return cudaGetLastError();
}

// Cell-major copy of a grid: the 8 corner values of every cell in one record
// (v000 v100 v010 v110 v001 v101 v011 v111), so a query reads one record.
template <class V>
__global__ void build_cells_kernel(const V* values, int nx, int ny, int nz, V* cells) {
    const int64_t ncx = nx - 1, ncy = ny - 1, ncz = nz - 1;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncx * ncy * ncz) return;
    const int i = (int)(c % ncx), j = (int)((c / ncx) % ncy), k = (int)(c / (ncx * ncy));
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t b = k * sz + j * sy + i;
    V* o = cells + 8 * c;
    o[0] = values[b];
    o[1] = values[b + sx];
    o[2] = values[b + sy];
    o[3] = values[b + sy + sx];
    o[4] = values[b + sz];
    o[5] = values[b + sz + sx];
    o[6] = values[b + sz + sy];
    o[7] = values[b + sz + sy + sx];
}

cudaError_t launch_build_cells(const void* values, const int dims[3], int fp16, void* cells, cudaStream_t s) {
    const int64_t n = (int64_t)(dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (fp16)
        build_cells_kernel<<<blocks, 256, 0, s>>>(static_cast<const uint16_t*>(values), dims[0], dims[1], dims[2],
                                                  static_cast<uint16_t*>(cells));
    else
        build_cells_kernel<<<blocks, 256, 0, s>>>(static_cast<const float*>(values), dims[0], dims[1], dims[2],
                                                  static_cast<float*>(cells));
    return cudaGetLastError();
}

cudaError_t launch_unpack_contact(const uint8_t* flags, int64_t n, int bit, uint8_t* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unpack_contact_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(flags, n, bit, out);
    return cudaGetLastError();
}

}  // namespace tg
