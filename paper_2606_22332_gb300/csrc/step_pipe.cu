// step_pipe.cu -- the fused per-taxel sensor step (Appendix A) as a
// pipelined persistent kernel.
//
// One CTA per SM runs work items (runs of whole links of one env, in the
// step's order, object-sorted by default) one after another: CTA b takes the
// items of order positions b, b + G, b + 2G, ...  Everything an item reads
// from HBM that does not depend on this step's arithmetic is brought into
// shared memory by bulk copies (cp.async.bulk, completed on mbarriers) ahead
// of the phase that reads it, so the phases compute from shared memory while
// the next item's data streams in:
//   taxel geometry, flags, link pose records, item layout and the object's
//   descriptor of item k+1 -- issued when item k starts (two buffers)
//   hysteresis state and depth drift of item k+1 -- after item k's phase A2N
//   force/torque drift of item k+1 -- after item k's phase B
// The item's order record (SlotRec) is fetched three items ahead with cp.async.
// Phases of an item (each ends at a CTA barrier):
//   A1  FP32 object-frame query of every taxel; taxels clear of the surface
//       finish (depth 0, no contact, no force); near-contact taxels are
//       listed first, clear ones last (warp-aggregated)
//   A2N the near-contact taxels' compensated query, depth, Schmitt bit and
//       force/torque followed by their noise state, while the other threads
//       run the noise state of the clear taxels
//   B   3x3 crosstalk, drift / white noise, quantisation, dead override ->
//       noisy force/torque (kept in registers over a barrier, then in hx)
//   C   every per-link quantity: clean and noisy force/torque, agg_force
//       (ZYX, clean and noisy), contact counts
// Every per-taxel result comes from the same routines (step_common.cuh) as
// the other schedules in step.cu, in the same order of operations, and the
// link sums are the same sequential compensated sums in lattice order, so
// all schedules give bit-identical outputs.
//
// Every mbarrier wait is bounded: a copy that does not complete in time is
// counted in err[2] (reported as TG_ERR_TIMEOUT), the CTA waits (bounded)
// for its other copies in flight and stops.
#include <cstdint>

#include "bulk.cuh"
#include "step_common.cuh"

namespace tg {
namespace {

constexpr int kStride = kItemCap + 4;       // floats per staged channel: a lead-in of up to 3, then the item
constexpr int kFlagStride = kItemCap + 16;  // bytes per staged flag row: a lead-in of up to 15
constexpr int kGeoCh = 7;                   // x y z R nx ny nz
constexpr int kHyCh = 15;                   // hysteresis x_{t-1} 0-6, xi 0-6, depth drift
constexpr int kDrCh = 6;                    // force/torque drift
constexpr int kLinkQuantities = 20;

struct alignas(16) Geo {
    float ch[kGeoCh][kStride];
    uint8_t flags[kFlagStride];
    float rec[kItemMaxLinks][kLinkRec];
    ItemMeta meta;
    ObjDev obj;
};

struct Lead {  // lead-in (elements) of each staged channel of one item
    int geo[kGeoCh + 1];  // float channels, then the flags
    int hy[kHyCh];
    int dr[kDrCh];
};

struct alignas(16) SmemPipe {
    Geo geo[2];
    float hy[kHyCh][kStride];
    float dr[kDrCh][kStride];
    float hx[6][kItemCap];  // force/torque after gain + hysteresis; after B the noisy force/torque
    float fc[6][kItemCap];  // clean force/torque
    float dd[3][kItemCap];  // clean depth, noisy depth
    SlotRec slot[4];        // order records: item k in slot[k & 3]
    Lead lead[2];
    uint8_t bits[kItemCap];
    int16_t order[kItemCap];  // A1: near-contact taxels from the front, clear ones from the back
    uint64_t mbar_geo[2], mbar_hy, mbar_dr;
    int nq, nc, abort;
    int rdelay;             // read delay of the item's env at this step (steps)
};
static_assert(sizeof(SmemPipe) <= 227 * 1024, "one CTA per SM");
static_assert(kStride * 4 % 16 == 0 && kFlagStride % 16 == 0 && sizeof(Geo) % 16 == 0, "bulk copy alignment");

// geometry, flags, link records, item layout and object of the item in `r`
__device__ void issue_geo(const StepArgs& a, SmemPipe& S, int buf, const SlotRec& r) {
    Geo& G = S.geo[buf];
    Lead& L = S.lead[buf];
    uint64_t* m = &S.mbar_geo[buf];
    uint32_t tx = 0;
    const float* src[kGeoCh] = {a.x, a.y, a.z, a.R, a.nx, a.ny, a.nz};
    proxy_fence();
#pragma unroll
    for (int c = 0; c < kGeoCh; ++c) L.geo[c] = stage(G.ch[c], src[c], r.taxel_begin, r.n_taxels, 4, m, tx);
    L.geo[kGeoCh] = stage(G.flags, a.flags, r.taxel_begin, r.n_taxels, 1, m, tx);
    const int nl = r.link_end - r.link_begin;
    bulk_load(G.rec, a.link_rec + ((size_t)r.env * a.max_links + r.link_begin) * kLinkRec,
              (uint32_t)(nl * kLinkRec * 4), m);
    bulk_load(&G.meta, a.metas + r.item, (uint32_t)sizeof(ItemMeta), m);
    bulk_load(&G.obj, a.objects + r.oid, (uint32_t)sizeof(ObjDev), m);
    tx += (uint32_t)(nl * kLinkRec * 4 + sizeof(ItemMeta) + sizeof(ObjDev));
    mbar_expect(m, tx);
}

// hysteresis state and depth drift (the channels the parameters use)
__device__ void issue_hy(const StepArgs& a, SmemPipe& S, int buf, const SlotRec& r) {
    const ParamsDev& P = a.P;
    const int64_t T = a.n_taxels;
    Lead& L = S.lead[buf];
    uint32_t tx = 0;
    proxy_fence();
    const bool hd = hyst_depth_on(P), hf = hyst_ft_on(P), wd = drift_depth_on(P);
    for (int c = 0; c < 7; ++c) {
        if (c == 0 ? !hd : !hf) continue;
        // x_{t-1}: hyst_prev, or with prev_out last step's clean output
        if (P.prev_out)
            L.hy[c] = stage(S.hy[c], c == 0 ? a.depth_clean : a.ft_clean, (c == 0 ? 0 : (c - 1) * T) + r.taxel_begin,
                            r.n_taxels, 4, &S.mbar_hy, tx);
        else
            L.hy[c] = stage(S.hy[c], a.hyst_prev, c * T + r.taxel_begin, r.n_taxels, 4, &S.mbar_hy, tx);
        L.hy[7 + c] = stage(S.hy[7 + c], a.hyst_xi, c * T + r.taxel_begin, r.n_taxels, 4, &S.mbar_hy, tx);
    }
    if (wd) L.hy[14] = stage(S.hy[14], a.drift, r.taxel_begin, r.n_taxels, 4, &S.mbar_hy, tx);
    mbar_expect(&S.mbar_hy, tx);
}

// force/torque drift
__device__ void issue_dr(const StepArgs& a, SmemPipe& S, int buf, const SlotRec& r) {
    const int64_t T = a.n_taxels;
    Lead& L = S.lead[buf];
    uint32_t tx = 0;
    proxy_fence();
    if (drift_ft_on(a.P))
        for (int c = 0; c < kDrCh; ++c)
            L.dr[c] = stage(S.dr[c], a.drift, (1 + c) * T + r.taxel_begin, r.n_taxels, 4, &S.mbar_dr, tx);
    mbar_expect(&S.mbar_dr, tx);
}

// order record of position p into S.slot[ring] (cp.async: the issuing thread waits for it)
__device__ __forceinline__ void fetch_slot(const StepArgs& a, SmemPipe& S, int ring, int p) {
    static_assert(sizeof(SlotRec) == 32, "one 32-byte record");
    cp_async32(&S.slot[ring], a.slots + p);
}
__device__ __forceinline__ void wait_slots() { cp_async_wait(); }

__device__ __forceinline__ int link_of(const ItemMeta& M, int i) { return meta_link_of(M, i); }

// One per-link quantity over taxels [s0, s1) in lattice order, as
// link_quantity in step_common.cuh (same sources, same compensated sums);
// the agg_force terms d n are formed here as single rounded products.
__device__ __forceinline__ void pipe_link_quantity(const StepArgs& a, const SmemPipe& S, const Geo& G, const Lead& L,
                                                   size_t rec, int s0, int s1, int qn) {
    if (qn == 12 || qn == 13) {
        const int bit = qn == 12 ? 0 : 1;
        int cnt = 0;
        for (int i = s0; i < s1; ++i) cnt += (S.bits[i] >> bit) & 1;
        a.link_count[rec * 2 + bit] = cnt;
        return;
    }
    float sum;
    int col;
    float scale = 1.0f;
    if (qn < 6) {
        col = qn;
        sum = link_sum(S.fc[qn], s0, s1);
    } else if (qn >= 14) {
        col = 6 + (qn - 14);
        sum = link_sum_halves(S.hx[qn - 14], s0, s1);
    } else {
        const bool noisy = qn >= 9;
        const int axis = noisy ? 2 - (qn - 9) : 2 - (qn - 6);  // ZYX
        const float* d = S.dd[noisy ? 1 : 0];
        const float* n = G.ch[4 + axis] + L.geo[4 + axis];
        col = noisy ? 15 + (qn - 9) : 12 + (qn - 6);
        scale = 1e4f;
        sum = link_sum_prod(d, n, s0, s1);
    }
    a.link_out[rec * kLinkOut + col] = scale * sum;
}

template <int NT, bool RADIUS>
__global__ void __launch_bounds__(NT, 1) step_pipe_kernel(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemPipe& S = *reinterpret_cast<SmemPipe*>(smem_raw);
    constexpr int kPer = (kItemCap + NT - 1) / NT;  // taxels per thread and phase
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = gridDim.x;
    const int n_items = a.n_items;
    const uint32_t step = a.step_from_ctl ? a.ctl->step : a.step;
    const ParamsDev& P = a.P;
    const int64_t T = a.n_taxels;
    const int Lmax = a.max_links;
    const bool hd = hyst_depth_on(P), hf = hyst_ft_on(P), wd = drift_depth_on(P), wf = drift_ft_on(P);
    const int p0 = blockIdx.x;
    if (p0 >= n_items) return;
    uint32_t pend = 0;      // thread 0: copies issued and not yet waited for (bit 0/1 geo, 2 hy, 3 dr)
    uint32_t issued[4] = {0, 0, 0, 0};  // thread 0: phases issued per barrier

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&S.mbar_geo[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&S.mbar_geo[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&S.mbar_hy)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&S.mbar_dr)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.nq = 0;
        S.nc = 0;
        S.abort = 0;
        for (int q = 0; q < 2; ++q) S.lead[q] = Lead{};  // channels a parameter set leaves off read index 0
    }
    // no thread may poll a barrier before it is initialised
    __syncthreads();
    if (tid == 0) {
        S.slot[0] = a.slots[p0];
        if (p0 + G < n_items) S.slot[1] = a.slots[p0 + G];
        if (p0 + 2 * G < n_items) fetch_slot(a, S, 2, p0 + 2 * G);
        issue_geo(a, S, 0, S.slot[0]);
        issue_hy(a, S, 0, S.slot[0]);
        issue_dr(a, S, 0, S.slot[0]);
        pend = 1u | 4u | 8u;
        issued[0] = issued[2] = issued[3] = 1;
    }
    bool ok = mbar_wait(&S.mbar_geo[0], 0);
    if (!ok && atomicExch(&S.abort, 1) == 0) atomicAdd(a.err + 2, 1u);
    __syncthreads();
    if (tid == 0) pend &= ~1u;

    for (int k = 0;; ++k) {
        if (S.abort) break;
        const int b = k & 1;
        const int pos = p0 + k * G;
        const bool has_next = pos + G < n_items;
        const SlotRec cur = S.slot[k & 3];
        Geo& Gb = S.geo[b];
        const ItemMeta& M = Gb.meta;
        const ObjDev& obj = Gb.obj;
        const Lead& Ld = S.lead[b];
        // (both within their maxima by construction; the clamps keep every
        // shared-memory index inside its array whatever the records hold)
        const int n = min(max(cur.n_taxels, 0), kItemCap);
        const int nl = min(max(M.nl, 1), kItemMaxLinks);
        const uint32_t ep = cur.episode;
        if (tid == 0) {
            S.rdelay = P.ring_k > 1 ? read_delay(P, (uint64_t)(a.env_gid0 + cur.env), step) : 0;
            wait_slots();  // the records of items k+1 and k+2 are in place
            // item k+3 into the entry of item k-1, which no thread reads any more
            if (pos + 3 * G < n_items) fetch_slot(a, S, (k + 3) & 3, pos + 3 * G);
            if (has_next) {
                issue_geo(a, S, b ^ 1, S.slot[(k + 1) & 3]);
                pend |= 1u << (b ^ 1);
                ++issued[b ^ 1];
            }
        }

        // ---- A1: FP32 query of every taxel from the staged geometry
        for (int i0 = tid & ~31; i0 < n; i0 += NT) {
            const int i = i0 + lane;
            const bool act = i < n;
            bool near = false;
            if (act) {
                const tidx g = (tidx)(cur.taxel_begin + i);
                const float x0 = Gb.ch[0][Ld.geo[0] + i], x1 = Gb.ch[1][Ld.geo[1] + i], x2 = Gb.ch[2][Ld.geo[2] + i];
                const float R = Gb.ch[3][Ld.geo[3] + i];
                const uint8_t fl = Gb.flags[Ld.geo[kGeoCh] + i];
                float phi = 0.0f;
                if (R > 0.0f) {
                    if (phi_precomputed(obj, P)) phi = a.nq_phi[g];
                    else phi = fast_query(Gb.rec[link_of(M, i)], obj, x0, x1, x2);
                    if (!isfinite(phi)) atomicAdd(a.err, 1u);
                }
                near = R > 0.0f && phi < R + 1e-6f + (RADIUS ? P.rho : 0.0f);
                if (!near) {
                    S.bits[i] = clear_taxel(a, g, R, fl, raycast_obj(obj, P) ? R : phi);
#pragma unroll
                    for (int c = 0; c < 6; ++c) S.fc[c][i] = 0.f;
                    S.dd[0][i] = 0.f;
                }
            }
            const unsigned mn = __ballot_sync(0xffffffffu, act && near);
            const unsigned mc = __ballot_sync(0xffffffffu, act && !near);
            int bn = 0, bc = 0;
            if (lane == 0) {
                if (mn) bn = atomicAdd(&S.nq, __popc(mn));
                if (mc) bc = atomicAdd(&S.nc, __popc(mc));
            }
            bn = __shfl_sync(0xffffffffu, bn, 0);
            bc = __shfl_sync(0xffffffffu, bc, 0);
            const unsigned lt = (1u << lane) - 1u;
            if (act) {
                if (near) S.order[bn + __popc(mn & lt)] = (int16_t)i;
                else S.order[n - 1 - (bc + __popc(mc & lt))] = (int16_t)i;
            }
        }
        ok = mbar_wait(&S.mbar_hy, (uint32_t)(k & 1));
        if (!ok && atomicExch(&S.abort, 1) == 0) atomicAdd(a.err + 2, 1u);
        __syncthreads();
        if (S.abort) break;
        if (tid == 0) pend &= ~4u;

        // ---- A2N: near-contact refinement + noise state, and the clear taxels' noise state
        const int nq = S.nq;
        for (int j = tid; j < n; j += NT) {
            const int i = S.order[j];
            const tidx g = (tidx)(cur.taxel_begin + i);
            uint8_t bits;
            float d_in = 0.0f, f_in[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (j < nq) {
                const float x0 = Gb.ch[0][Ld.geo[0] + i], x1 = Gb.ch[1][Ld.geo[1] + i], x2 = Gb.ch[2][Ld.geo[2] + i];
                const float R = Gb.ch[3][Ld.geo[3] + i];
                const uint8_t fl = Gb.flags[Ld.geo[kGeoCh] + i];
                const CleanReading cr = refine_compute<RADIUS>(P, a.nq_phi, a.nq_phi_lo, a.nq_grad, T, a.gid0,
                                                               Gb.rec[link_of(M, i)], obj, g, x0, x1, x2, R, fl, step);
                store_clean(a, g, cr);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    S.fc[c][i] = cr.f[c];
                    S.fc[3 + c][i] = cr.tq[c];
                }
                S.dd[0][i] = cr.d;
                bits = cr.bits;
                d_in = RADIUS ? cr.dn : cr.d;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    f_in[c] = RADIUS ? cr.fn[c] : cr.f[c];
                    f_in[3 + c] = RADIUS ? cr.tqn[c] : cr.tq[c];
                }
            } else {
                bits = S.bits[i];
            }
            if (bits & BIT_ACTIVE) {
                NoiseIn s;
                s.prev_d = hd ? S.hy[0][Ld.hy[0] + i] : 0.0f;
                s.xi_d = hd ? S.hy[7][Ld.hy[7] + i] : 0.0f;
                s.drift_d = wd ? S.hy[14][Ld.hy[14] + i] : 0.0f;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    s.pv[c] = hf ? S.hy[1 + c][Ld.hy[1 + c] + i] : 0.0f;
                    s.xv[c] = hf ? S.hy[8 + c][Ld.hy[8 + c] + i] : 0.0f;
                }
                if (P.ring_k > 1) bits = delay_readout(a, g, step, S.rdelay, bits, d_in, f_in);
                const NoiseOut o = noise_core(P, (uint64_t)(a.gid0 + g), ep, step, bits, d_in, f_in, s);
                if (hd) {
                    __stcs(a.hyst_xi + g, o.xi_d);
                    if (!P.prev_out) __stcs(a.hyst_prev + g, o.prev_d);
                }
                if (hf) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        __stcs(a.hyst_xi + (1 + c) * T + g, o.xv[c]);
                        if (!P.prev_out) __stcs(a.hyst_prev + (1 + c) * T + g, o.pv[c]);
                    }
                }
                if (wd) __stcs(a.drift + g, o.drift_d);
                __stcs(a.depth_noisy + g, o.xd);
#pragma unroll
                for (int c = 0; c < 6; ++c) S.hx[c][i] = o.hx[c];
                S.dd[1][i] = o.xd;
            } else {
                __stcs(a.depth_noisy + g, 0.f);
#pragma unroll
                for (int c = 0; c < 6; ++c) S.hx[c][i] = 0.f;
                S.dd[1][i] = 0.f;
            }
            S.bits[i] = bits;
            {  // clean outputs, after the staged copy of last step's (prev_out) has landed
                float fc[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) fc[c] = S.fc[c][i];
                store_clean_out(a, g, S.dd[0][i], fc);
            }
        }
        ok = mbar_wait(&S.mbar_dr, (uint32_t)(k & 1));
        if (!ok && atomicExch(&S.abort, 1) == 0) atomicAdd(a.err + 2, 1u);
        __syncthreads();
        if (S.abort) break;
        if (tid == 0) {
            pend &= ~8u;
            S.nq = 0;
            S.nc = 0;
            if (has_next) {
                issue_hy(a, S, b ^ 1, S.slot[(k + 1) & 3]);
                pend |= 4u;
                ++issued[2];
            }
        }

        // ---- B: crosstalk and the noisy force/torque (kept in registers until hx is free)
        float zk[kPer][6];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int i = tid + u * NT;
            if (i >= n) break;
            const tidx g = (tidx)(cur.taxel_begin + i);
            const uint8_t bits = S.bits[i];
            if (!(bits & BIT_ACTIVE)) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    zk[u][c] = 0.0f;
                    __stcs(a.ft_noisy + c * T + g, 0.f);
                }
                continue;
            }
            int base, r, cc, rows, cols;
            bool wrap;
            if (M.uni_len) {
                base = uni_div(i, M.uni_inv_len) * M.uni_len;
                const int jj = i - base;
                r = uni_div(jj, M.uni_inv_cols);
                cc = jj - r * M.uni_cols;
                rows = M.uni_rows;
                cols = M.uni_cols;
                wrap = M.uni_wrap != 0;
            } else {
                const int l = link_of(M, i);
                base = M.start[l];
                cols = M.cols[l];
                rows = M.rows[l];
                wrap = M.wrap[l] != 0;
                const int jj = i - base;
                r = jj / cols;
                cc = jj - r * cols;
            }
            float dr[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) dr[c] = wf ? S.dr[c][Ld.dr[c] + i] : 0.0f;
            crosstalk(P, S.hx, i, base, r, cc, rows, cols, wrap, zk[u]);
            noisy_core(P, (uint64_t)(a.gid0 + g), ep, step, bits, zk[u], dr);
            if (wf) {
#pragma unroll
                for (int c = 0; c < 6; ++c) __stcs(a.drift + (1 + c) * T + g, dr[c]);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) __stcs(a.ft_noisy + c * T + g, zk[u][c]);
        }
        __syncthreads();
        if (tid == 0 && has_next) {
            issue_dr(a, S, b ^ 1, S.slot[(k + 1) & 3]);
            pend |= 8u;
            ++issued[3];
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int i = tid + u * NT;
            if (i >= n) break;
#pragma unroll
            for (int c = 0; c < 6; ++c) S.hx[c][i] = zk[u][c];
        }
        __syncthreads();

        // ---- C: every per-link quantity
        for (int t = tid; t < nl * kLinkQuantities; t += NT) {
            const int ll = t % nl;
            pipe_link_quantity(a, S, Gb, Ld, (size_t)cur.env * Lmax + cur.link_begin + ll, M.start[ll],
                               M.start[ll + 1], t / nl);
        }
        if (has_next) {
            ok = mbar_wait(&S.mbar_geo[b ^ 1], (uint32_t)(((k + 1) >> 1) & 1));
            if (!ok && atomicExch(&S.abort, 1) == 0) atomicAdd(a.err + 2, 1u);
        }
        __syncthreads();
        if (tid == 0 && has_next && !S.abort) pend &= ~(1u << (b ^ 1));
        if (!has_next) break;
    }
    // after a timeout: let the copies still in flight land before the CTA's
    // shared memory is released (each wait bounded; a phase that already
    // completed returns at once)
    if (S.abort && tid == 0) {
        for (int q = 0; q < 4; ++q) {
            if (!(pend & (1u << q))) continue;
            uint64_t* m = q < 2 ? &S.mbar_geo[q] : (q == 2 ? &S.mbar_hy : &S.mbar_dr);
            mbar_wait(m, (issued[q] - 1u) & 1u);  // the phase of the last copy issued
        }
        wait_slots();
    }
}

template <int NT>
cudaError_t launch_nt(const StepArgs& a, int n_items, cudaStream_t s) {
    const int ctas = min(a.sms, n_items);
    if (ctas <= 0) return cudaErrorInvalidConfiguration;
    if (a.P.rho > 0.0f) step_pipe_kernel<NT, true><<<ctas, NT, sizeof(SmemPipe), s>>>(a);
    else step_pipe_kernel<NT, false><<<ctas, NT, sizeof(SmemPipe), s>>>(a);
    return cudaGetLastError();
}

// Order records of this step: a counting sort by the object each item's env
// holds (sorted != 0; one CTA, counts in shared memory), or env order.
__global__ void slot_records_kernel(const Item* items, int n_items, const int32_t* obj_id, int n_objects,
                                    const uint32_t* episode, int sorted, SlotRec* out) {
    extern __shared__ int cnt[];  // [n_objects]
    auto record = [&](int idx) {
        const Item it = items[idx];
        SlotRec r;
        r.taxel_begin = it.taxel_begin;
        r.n_taxels = it.n_taxels;
        r.env = it.env;
        r.item = idx;
        r.oid = min(max(obj_id[it.env], 0), n_objects - 1);
        r.episode = episode[it.env];
        r.link_begin = it.link_begin;
        r.link_end = it.link_end;
        return r;
    };
    if (!sorted) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_items; i += gridDim.x * blockDim.x)
            out[i] = record(i);
        return;
    }
    for (int k = threadIdx.x; k < n_objects; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n_items; i += blockDim.x)
        atomicAdd(&cnt[min(max(obj_id[items[i].env], 0), n_objects - 1)], 1);
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
        const SlotRec r = record(i);
        out[atomicAdd(&cnt[r.oid], 1)] = r;
    }
}

}  // namespace

cudaError_t configure_pipe_kernels() {
    const void* k[6] = {(const void*)step_pipe_kernel<1024, false>, (const void*)step_pipe_kernel<1024, true>,
                        (const void*)step_pipe_kernel<768, false>,  (const void*)step_pipe_kernel<768, true>,
                        (const void*)step_pipe_kernel<512, false>,  (const void*)step_pipe_kernel<512, true>};
    for (const void* f : k) {
        const cudaError_t e = raise_smem_limit(f, sizeof(SmemPipe));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_step_pipe(const StepArgs& a, int n_items, int threads, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    if (!a.slots || !a.metas || a.n_items != n_items) return cudaErrorInvalidValue;
    switch (threads) {
        case 1024: return launch_nt<1024>(a, n_items, s);
        case 768: return launch_nt<768>(a, n_items, s);
        case 512: return launch_nt<512>(a, n_items, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_slot_records(const Item* items, int n_items, const int32_t* obj_id, int n_objects,
                                const uint32_t* episode, int sorted, SlotRec* out, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    const size_t smem = (size_t)n_objects * sizeof(int);
    if (sorted && smem <= 160 * 1024) {
        if (smem > 48 * 1024) {
            const cudaError_t e = raise_smem_limit((const void*)slot_records_kernel, 160 * 1024);
            if (e != cudaSuccess) return e;
        }
        slot_records_kernel<<<1, 1024, smem, s>>>(items, n_items, obj_id, n_objects, episode, 1, out);
    } else {
        slot_records_kernel<<<(n_items + 255) / 256, 256, 0, s>>>(items, n_items, obj_id, n_objects, episode, 0,
                                                                  out);
    }
    return cudaGetLastError();
}

}  // namespace tg
