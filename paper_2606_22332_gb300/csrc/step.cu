// step.cu -- the fused per-taxel sensor step (Appendix A) and the episode
// reset.
//
// One CTA per work item: a run of whole links of one env (at most kItemCap
// taxels, kItemMaxLinks links); items are taken in an object-sorted order so
// that concurrently running CTAs share one or two SDF grids in L2.  Per-taxel
// arrays are SoA in HBM, read and written coalesced with streaming
// (evict-first) cache operators.
//   phase A1 per taxel: FP32 object-frame query; taxels clear of the surface
//            finish here (depth 0, no contact, no force), the others queue
//   phase A2 queued near-contact taxels, compacted onto whole warps:
//            compensated query point and SDF, depth, Schmitt bit, force/torque
//   phase N  per taxel: noise state (gain, hysteresis, depth base noise, dead)
//            with all state loads independent of the geometry; agg_force terms
//   phase C1 per (link, quantity): clean sums, agg_force, contact counts
//   phase B  per taxel: 3x3 crosstalk from shared memory, drift/white noise,
//            quantisation, dead override -> noisy force/torque
//   phase C2 per (link, quantity): noisy sums
// Link sums are sequential compensated (Neumaier) sums in lattice order, so
// results are deterministic run to run.
#include <cstdint>

#include "step_common.cuh"

namespace tg {

constexpr int kItemMaxLinks = 32;

struct SmemStep {
    float rec[kItemMaxLinks][kLinkRec];
    int start[kItemMaxLinks + 1];       // first taxel of each link, relative to the item
    int rows[kItemMaxLinks], cols[kItemMaxLinks], wrap[kItemMaxLinks];
    ObjDev obj;
    float hx[6][kItemCap];              // force/torque after gain + hysteresis
    float fc[6][kItemCap];              // clean force/torque, later noisy force/torque
    float ag[6][kItemCap];              // clean depth, then agg_force terms d n: clean xyz, noisy xyz
    uint8_t bits[kItemCap];             // BIT_* flags
    int16_t queue[kItemCap];            // near-contact taxels for phase A2
    int nq;
};

template <int NT>
__global__ void __launch_bounds__(NT, kStepMinBlocks) step_kernel(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemStep& S = *reinterpret_cast<SmemStep*>(smem_raw);
    const Item it = a.items[a.item_order ? a.item_order[blockIdx.x] : blockIdx.x];
    const int e = it.env;
    const int L = a.max_links;
    const int lb = it.link_begin;
    const int nl = it.link_end - it.link_begin;
    const int n = it.n_taxels;
    const int tid = threadIdx.x;

    // ---- prologue: link records, lattice, object
    for (int i = tid; i < nl * kLinkRec; i += NT) {
        int l = i / kLinkRec, f = i % kLinkRec;
        S.rec[l][f] = a.link_rec[(size_t)(e * L + lb + l) * kLinkRec + f];
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
    if (tid == 0) {
        int oid = a.obj_id[e];
        oid = min(max(oid, 0), a.n_objects - 1);
        S.obj = a.objects[oid];
        S.nq = 0;
    }
    __syncthreads();

    const uint32_t ep = a.episode[e];
    const ObjDev& obj = S.obj;

    // ---- phase A1 (geometry): FP32 query of every taxel; those clear of the
    //      surface finish here, those within 1 um of contact are queued
    int l = 0;
    for (int i = tid; i < n; i += NT) {
        while (i >= S.start[l + 1]) ++l;
        const int64_t g = it.taxel_begin + i;
        const float R = __ldcs(a.R + g);
        const float x0 = __ldcs(a.x + g), x1 = __ldcs(a.y + g), x2 = __ldcs(a.z + g);
        const uint8_t flags = __ldcs(a.flags + g);
        float phi = 0.0f;
        bool near = false;
        if (R > 0.0f) {
            phi = fast_query(S.rec[l], obj, x0, x1, x2);
            if (!isfinite(phi)) atomicAdd(a.err, 1u);
            near = phi < R + 1e-6f;
        }
        if (near) {
            S.queue[atomicAdd(&S.nq, 1)] = (int16_t)i;
            continue;
        }
        S.bits[i] = clear_taxel(a, g, R, flags, phi);
#pragma unroll
        for (int c = 0; c < 6; ++c) S.fc[c][i] = 0.f;
        S.ag[0][i] = 0.f;
    }
    __syncthreads();

    // ---- phase A2: near-contact taxels, compacted onto whole warps
    const int nq = S.nq;
    for (int k = tid; k < nq; k += NT) {
        const int i = S.queue[k];
        int lo = 0, hi = nl - 1;  // link of taxel i: last start <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.start[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const CleanReading cr = refine_taxel(a, S.rec[lo], obj, it.taxel_begin + i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            S.fc[c][i] = cr.f[c];
            S.fc[3 + c][i] = cr.tq[c];
        }
        S.ag[0][i] = cr.d;
        S.bits[i] = cr.bits;
    }
    __syncthreads();

    // ---- phase N: noise state of every taxel (independent state loads)
    for (int i = tid; i < n; i += NT) {
        const int64_t g = it.taxel_begin + i;
        const uint8_t bits = S.bits[i];
        if (bits & BIT_ACTIVE) noise_state(a, S, i, g, ep, bits);
        else noise_state_filler(a, S, i, g);
    }
    __syncthreads();

    // ---- phase C1: clean link sums, agg_force (clean and noisy), contact counts
    for (int t = tid; t < nl * 14; t += NT) {
        const int ll = t % nl;
        link_quantity(a, S, S.fc, (size_t)(e * L + lb + ll), S.start[ll], S.start[ll + 1], t / nl);
    }
    __syncthreads();

    // ---- phase B: crosstalk, base noise, dead override -> noisy force/torque
    //      (written over the clean values in fc, which C1 has consumed)
    l = 0;
    for (int i = tid; i < n; i += NT) {
        while (i >= S.start[l + 1]) ++l;
        const int j = i - S.start[l], cols = S.cols[l];
        const int r = j / cols;
        noisy_ft(a, S, S.fc, i, it.taxel_begin + i, ep, S.bits[i], S.start[l], r, j - r * cols, S.rows[l], cols,
                 S.wrap[l] != 0);
    }
    __syncthreads();

    // ---- phase C2: noisy force/torque link sums
    for (int t = tid; t < nl * 6; t += NT) {
        const int ll = t % nl;
        link_quantity(a, S, S.fc, (size_t)(e * L + lb + ll), S.start[ll], S.start[ll + 1], 14 + t / nl);
    }
}

// Reset of the envs whose mask byte is set: dead mask drawn from
// (seed, taxel id, episode), hysteresis / drift / Schmitt state zeroed.
__global__ void reset_kernel(const StepArgs a, const uint8_t* env_mask, uint32_t episode, uint32_t* episode_arr) {
    const Item it = a.items[blockIdx.x];
    const int e = it.env;
    if (env_mask && !env_mask[e]) return;
    if (threadIdx.x == 0) episode_arr[e] = episode;
    const int64_t T = a.n_taxels;
    for (int i = threadIdx.x; i < it.n_taxels; i += blockDim.x) {
        const int64_t g = it.taxel_begin + i;
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
    }
}

__global__ void unpack_contact_kernel(const uint8_t* flags, int64_t n, int noisy, uint8_t* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (flags[i] >> (noisy ? 2 : 0)) & 1u;
}

cudaError_t launch_step(const StepArgs& a, int n_items, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    const size_t smem = sizeof(SmemStep);
    static bool configured = false;
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(step_kernel<kStepThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        configured = true;
    }
    step_kernel<kStepThreads><<<n_items, kStepThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Counting sort of the work items by the object their env holds this step:
// CTAs launched together then read one or two object grids, which stay in L2
// while the per-taxel state streams past.  Order within an object is
// arbitrary; every item's result is independent of it.
__global__ void order_items_kernel(const Item* items, int n_items, const int32_t* obj_id, int n_objects,
                                   int32_t* order) {
    extern __shared__ int cnt[];
    for (int k = threadIdx.x; k < n_objects; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n_items; i += blockDim.x) {
        const int k = min(max(obj_id[items[i].env], 0), n_objects - 1);
        atomicAdd(&cnt[k], 1);
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
        const int k = min(max(obj_id[items[i].env], 0), n_objects - 1);
        order[atomicAdd(&cnt[k], 1)] = i;
    }
}

cudaError_t launch_order_items(const Item* items, int n_items, const int32_t* obj_id, int n_objects,
                               int32_t* order, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    order_items_kernel<<<1, 1024, (size_t)n_objects * sizeof(int), s>>>(items, n_items, obj_id, n_objects, order);
    return cudaGetLastError();
}

cudaError_t launch_reset(const StepArgs& a, int n_items, const uint8_t* env_mask, uint32_t episode,
                         uint32_t* episode_arr, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    reset_kernel<<<n_items, 256, 0, s>>>(a, env_mask, episode, episode_arr);
    return cudaGetLastError();
}

cudaError_t launch_unpack_contact(const uint8_t* flags, int64_t n, int noisy, uint8_t* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unpack_contact_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(flags, n, noisy, out);
    return cudaGetLastError();
}

}  // namespace tg
