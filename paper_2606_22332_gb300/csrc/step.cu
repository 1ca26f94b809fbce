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

#include "df.cuh"
#include "geom.cuh"
#include "internal.h"
#include "rng.cuh"

namespace tg {

constexpr int kItemMaxLinks = 32;

struct SmemStep {
    float rec[kItemMaxLinks][kLinkRec];
    int start[kItemMaxLinks + 1];       // first taxel of each link, relative to the item
    int rows[kItemMaxLinks], cols[kItemMaxLinks], wrap[kItemMaxLinks];
    ObjDev obj;
    float hx[6][kItemCap];              // force/torque after gain + hysteresis
    float fc[6][kItemCap];              // clean force/torque, later noisy force/torque
    float ag[6][kItemCap];              // agg_force terms d n: clean xyz, noisy xyz
    uint8_t bits[kItemCap];             // bit0 clean contact, bit1 noisy contact, bit2 dead, bit3 active
    int16_t queue[kItemCap];            // near-contact taxels for phase A2
    int nq;
};

__device__ __forceinline__ float hyst_update(const NoiseDev& g, float x, float* prev_p, float* xi_p) {
    float xi = g.decay * __ldcs(xi_p) + (x - __ldcs(prev_p));
    __stcs(xi_p, xi);
    __stcs(prev_p, x);
    return x + g.beta * xi;
}

__device__ __forceinline__ float quantise(const NoiseDev& g, float y) {
    return g.quant > 0.0f ? g.quant * rintf(y / g.quant) : y;
}

// compensated accumulation (Neumaier)
struct Acc {
    float s, c;
};
__device__ __forceinline__ void acc_add(Acc& a, float x) {
    float t = a.s + x;
    if (fabsf(a.s) >= fabsf(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}

// Per-link sums: one thread per (link, quantity) adds the link's taxels in
// lattice order with compensated (Neumaier) accumulation, so results are
// deterministic and carry no order-dependent rounding.
//   clean phase: quantities 0-5 clean force/torque, 6-8 clean agg_force
//                (ZYX order), 9-11 noisy agg_force, 12 clean count, 13 noisy count
//   noisy phase: quantities 0-5 noisy force/torque
__device__ __forceinline__ void link_sums(const StepArgs& a, const SmemStep& S, const Item& it, int nl, bool noisy,
                                          int tid, int nt) {
    const int nquant = noisy ? 6 : 14;
    for (int t = tid; t < nl * nquant; t += nt) {
        const int ll = t % nl, qn = t / nl;
        const int s0 = S.start[ll], s1 = S.start[ll + 1];
        const size_t rec = (size_t)(it.env * a.max_links + it.link_begin + ll);
        if (qn >= 12) {
            const int bit = qn - 12;
            int cnt = 0;
            for (int i = s0; i < s1; ++i) cnt += (S.bits[i] >> bit) & 1;
            a.link_count[rec * 2 + bit] = cnt;
            continue;
        }
        const float* src;
        int col;
        if (noisy) { src = S.fc[qn]; col = 6 + qn; }
        else if (qn < 6) { src = S.fc[qn]; col = qn; }
        else if (qn < 9) { src = S.ag[2 - (qn - 6)]; col = 12 + (qn - 6); }      // clean agg, ZYX
        else { src = S.ag[3 + 2 - (qn - 9)]; col = 15 + (qn - 9); }               // noisy agg, ZYX
        Acc acc{0.f, 0.f};
        for (int i = s0; i < s1; ++i) acc_add(acc, src[i]);
        const float v = acc.s + acc.c;
        a.link_out[rec * kLinkOut + col] = (qn >= 6 && !noisy) ? 1e4f * v : v;
    }
}

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
    const ParamsDev& P = a.P;

    // ---- prologue: link records, lattice, object
    for (int i = tid; i < nl * kLinkRec; i += NT) {
        int l = i / kLinkRec, f = i % kLinkRec;
        S.rec[l][f] = a.link_rec[(size_t)(e * L + lb + l) * kLinkRec + f];
    }
    if (tid < nl) {
        LinkLattice lat = a.lattice[e * L + lb + tid];
        S.rows[tid] = lat.rows;
        S.cols[tid] = lat.cols;
        S.wrap[tid] = lat.wrap;
    }
    if (tid == 0) {
        int acc = 0;
        for (int l = 0; l < nl; ++l) {
            LinkLattice lat = a.lattice[e * L + lb + l];
            S.start[l] = acc;
            acc += (int)lat.rows * (int)lat.cols;
        }
        S.start[nl] = acc;
        int oid = a.obj_id[e];
        oid = min(max(oid, 0), a.n_objects - 1);
        S.obj = a.objects[oid];
        S.nq = 0;
    }
    __syncthreads();

    const uint32_t ep = a.episode[e];
    const int64_t T = a.n_taxels;
    const ObjDev& obj = S.obj;

    // ---- phase A1 (geometry): FP32 query of every taxel; those clear of the
    //      surface get depth 0, contact off and zero force here, those within
    //      the guard band of contact are queued for phase A2
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
            const float* rec = S.rec[l];
            float3 q = f3(fmaf(rec[0], x0, fmaf(rec[1], x1, fmaf(rec[2], x2, rec[18]))),
                          fmaf(rec[3], x0, fmaf(rec[4], x1, fmaf(rec[5], x2, rec[19]))),
                          fmaf(rec[6], x0, fmaf(rec[7], x1, fmaf(rec[8], x2, rec[20]))));
            float3 go;
            phi = rec[38] * sdf_fast(obj, q, &go);
            if (!isfinite(phi)) atomicAdd(a.err, 1u);
            near = phi < R + 1e-6f;
        }
        if (near) {
            S.queue[atomicAdd(&S.nq, 1)] = (int16_t)i;
            continue;
        }
        // clear of contact (or an inactive filler: R = 0, all outputs zero)
        __stcs(a.flags + g, (uint8_t)(flags & 2u));
        __stcs(a.depth_clean + g, 0.f);
        if (a.sensors & TG_SENSOR_DIST) __stcs(a.dist + g, R > 0.0f ? phi - R : 0.0f);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            __stcs(a.ft_clean + c * T + g, 0.f);
            S.fc[c][i] = 0.f;
        }
        S.ag[0][i] = 0.f;                          // clean depth 0 (the clean agg terms are d n)
        S.bits[i] = (uint8_t)(((flags & 2u) << 1) | (R > 0.0f ? 8u : 0u));  // bit2 dead, bit3 active
    }
    __syncthreads();

    // ---- phase A2: near-contact taxels, compacted onto whole warps:
    //      compensated query, depth, Schmitt bit, force/torque (Eqs. 2-9)
    const int nq = S.nq;
    for (int k = tid; k < nq; k += NT) {
        const int i = S.queue[k];
        int lo = 0, hi = nl - 1;  // link of taxel i: last start <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.start[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const float* rec = S.rec[lo];
        const int64_t g = it.taxel_begin + i;
        const float R = a.R[g];
        const uint8_t flags = a.flags[g];
        const float x0 = a.x[g], x1 = a.y[g], x2 = a.z[g];
        df qd[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            df acc = df{rec[18 + r], rec[21 + r]};
            acc = df_add(acc, df_mul_f(df{rec[3 * r], rec[9 + 3 * r]}, x0));
            acc = df_add(acc, df_mul_f(df{rec[3 * r + 1], rec[9 + 3 * r + 1]}, x1));
            acc = df_add(acc, df_mul_f(df{rec[3 * r + 2], rec[9 + 3 * r + 2]}, x2));
            qd[r] = acc;
        }
        float3 go;
        const float scale = rec[38];
        const df phid = df_mul_f(sdf_refine(obj, df3{qd[0], qd[1], qd[2]}, &go), scale);
        const df dd = df_add_f(df_neg(phid), R);  // R - phi
        const float d = dd.hi > 0.0f ? dd.hi : 0.0f;
        const bool prev = flags & 1u;
        const bool y = df_gt(dd, df{P.eta_on_hi, P.eta_on_lo}) || (prev && df_gt(dd, df{P.eta_off_hi, P.eta_off_lo}));
        const bool dead = flags & 2u;
        const bool yn = y && !dead;
        __stcs(a.flags + g, (uint8_t)((y ? 1u : 0u) | (flags & 2u) | (yn ? 4u : 0u)));
        float f[3] = {0.f, 0.f, 0.f}, tq[3] = {0.f, 0.f, 0.f};
        if (d > 0.0f) {
            float3 mb = normalize_or(f3(rec[0] * go.x + rec[3] * go.y + rec[6] * go.z,
                                        rec[1] * go.x + rec[4] * go.y + rec[7] * go.z,
                                        rec[2] * go.x + rec[5] * go.y + rec[8] * go.z),
                                     f3(0.f, 0.f, 1.f));
            const float3 xv = f3(x0, x1, x2);
            const float3 V = f3(rec[24], rec[25], rec[26]), Wc = f3(rec[27], rec[28], rec[29]);
            const float3 Wl = f3(rec[30], rec[31], rec[32]), pLC = f3(rec[33], rec[34], rec[35]);
            float3 vrel = V + cross(Wc, xv - pLC) - cross(Wl, xv);
            const float s = (P.alpha == 1.0f) ? d : powf(d, P.alpha);
            const float kk = rec[36], mu = rec[37];
            float vns = dot(vrel, mb);
            float3 vn = mb * vns;
            float3 vt = vrel - vn;
            float3 fn = mb * (kk * s) + vn * (P.c * s);
            float vtn = sqrtf(dot(vt, vt));
            float sc = 1.0f;
            if (mu >= 0.0f && P.k_t * vtn > 0.0f) sc = fminf(1.0f, mu * sqrtf(dot(fn, fn)) / (P.k_t * vtn));
            float3 ff = fn - vt * (P.k_t * sc);
            float3 tt = cross(xv, ff) - mb * (P.k_omega * dot(Wc - Wl, mb));
            f[0] = ff.x; f[1] = ff.y; f[2] = ff.z;
            tq[0] = tt.x; tq[1] = tt.y; tq[2] = tt.z;
        }
        __stcs(a.depth_clean + g, d);
        if (a.sensors & TG_SENSOR_DIST) __stcs(a.dist + g, -dd.hi);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            __stcs(a.ft_clean + c * T + g, f[c]);
            __stcs(a.ft_clean + (3 + c) * T + g, tq[c]);
            S.fc[c][i] = f[c];
            S.fc[3 + c][i] = tq[c];
        }
        S.ag[0][i] = d;  // clean depth, turned into d n in phase N
        S.bits[i] = (uint8_t)((y ? 1u : 0u) | (yn ? 2u : 0u) | (dead ? 4u : 0u) | 8u);
    }
    __syncthreads();

    // ---- phase N: noise state of every taxel (Eqs. 25-30, R12 order):
    //      depth gain, hysteresis, bias + white + drift, quantisation, dead;
    //      force/torque gain and hysteresis, staged for the crosstalk.  The
    //      state loads do not depend on the geometry, so they all issue at once.
    for (int i = tid; i < n; i += NT) {
        const int64_t g = it.taxel_begin + i;
        const uint8_t bits = S.bits[i];
        if (!(bits & 8u)) {  // filler
            __stcs(a.depth_noisy + g, 0.f);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                S.hx[c][i] = 0.f;
                S.ag[c][i] = 0.f;
            }
            continue;
        }
        const float n0 = __ldcs(a.nx + g), n1 = __ldcs(a.ny + g), n2 = __ldcs(a.nz + g);
        const uint64_t gid = (uint64_t)(a.gid0 + g);
        const bool dead = bits & 4u;
        const float d = S.ag[0][i];
        uint4 wep = make_uint4(0, 0, 0, 0);
        if (P.depth.gain_on | P.ft.gain_on) wep = draw(P.seed, gid, ep, TAG_EPISODE);
        const float gain_d = P.depth.gain_on ? P.depth.gain_lo + P.depth.gain_span * u24(wep.y) : 1.0f;
        const float gain_f = P.ft.gain_on ? P.ft.gain_lo + P.ft.gain_span * u24(wep.z) : 1.0f;
        float xd = gain_d * d;
        if (P.depth.beta != 0.0f) xd = hyst_update(P.depth, xd, a.hyst_prev + g, a.hyst_xi + g);
        if (P.ft.beta != 0.0f) {
            float pv[6], xv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                pv[c] = __ldcs(a.hyst_prev + (1 + c) * T + g);
                xv[c] = __ldcs(a.hyst_xi + (1 + c) * T + g);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const float x = gain_f * S.fc[c][i];
                const float xi = P.ft.decay * xv[c] + (x - pv[c]);
                __stcs(a.hyst_xi + (1 + c) * T + g, xi);
                __stcs(a.hyst_prev + (1 + c) * T + g, x);
                S.hx[c][i] = x + P.ft.beta * xi;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) S.hx[c][i] = gain_f * S.fc[c][i];
        }
        if (P.depth.sigma_rw != 0.0f || P.depth.sigma_white != 0.0f) {
            uint4 w = draw(P.seed, gid, a.step, TAG_SCALAR);
            float2 z = box_muller(w.x, w.y);
            float dr = 0.0f;
            if (P.depth.sigma_rw != 0.0f) {
                dr = __ldcs(a.drift + g) + P.depth.sigma_rw * z.x;
                __stcs(a.drift + g, dr);
            }
            xd = xd + P.depth.bias + P.depth.sigma_white * z.y + dr;
        } else {
            xd += P.depth.bias;
        }
        xd = quantise(P.depth, xd);
        if (dead) xd = P.depth.stuck_lo + P.depth.stuck_span * u24(draw(P.seed, gid, ep, TAG_STUCK).x);
        __stcs(a.depth_noisy + g, xd);
        // agg_force terms (Eq. 32): depth times the link-frame probe normal
        S.ag[0][i] = d * n0; S.ag[1][i] = d * n1; S.ag[2][i] = d * n2;
        S.ag[3][i] = xd * n0; S.ag[4][i] = xd * n1; S.ag[5][i] = xd * n2;
    }
    __syncthreads();

    // ---- phase C1: clean link sums, agg_force (clean and noisy), contact counts
    link_sums(a, S, it, nl, false, tid, NT);
    __syncthreads();

    // ---- phase B: crosstalk, base noise, dead override
    l = 0;
    for (int i = tid; i < n; i += NT) {
        while (i >= S.start[l + 1]) ++l;
        const int64_t g = it.taxel_begin + i;
        const uint8_t bits = S.bits[i];
        if (!(bits & 8u)) {  // filler
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                __stcs(a.ft_noisy + c * T + g, 0.f);
                S.fc[c][i] = 0.f;
            }
            continue;
        }
        const uint64_t gid = (uint64_t)(a.gid0 + g);
        const NoiseDev& G = P.ft;
        float dr_prev[6];
        if (G.sigma_rw != 0.0f) {
#pragma unroll
            for (int c = 0; c < 6; ++c) dr_prev[c] = __ldcs(a.drift + (1 + c) * T + g);
        }
        float z[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) z[c] = S.hx[c][i];
        if (P.chi != 0.0f) {
            const int j = i - S.start[l], cols = S.cols[l], rows = S.rows[l];
            const int r = j / cols, cc = j - r * cols;
            float conv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                const int rr = r + di;
                if (rr < 0 || rr >= rows) continue;
#pragma unroll
                for (int dj = -1; dj <= 1; ++dj) {
                    int c2 = cc + dj;
                    if (c2 < 0 || c2 >= cols) {
                        if (!S.wrap[l]) continue;
                        c2 += c2 < 0 ? cols : -cols;
                    }
                    const int nb = S.start[l] + rr * cols + c2;
                    const float w = P.xt_w[(di + 1) * 3 + (dj + 1)];
#pragma unroll
                    for (int c = 0; c < 6; ++c) conv[c] = fmaf(w, S.hx[c][nb], conv[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) z[c] = (1.0f - P.chi) * z[c] + P.chi * conv[c];
        }
        if (G.sigma_rw != 0.0f || G.sigma_white != 0.0f) {
            float nrm[12];
            uint4 wa = draw(P.seed, gid, a.step, TAG_FT_A);
            uint4 wb = draw(P.seed, gid, a.step, TAG_FT_B);
            float2 p0 = box_muller(wa.x, wa.y), p1 = box_muller(wa.z, wa.w);
            float2 p2 = box_muller(wb.x, wb.y);
            nrm[0] = p0.x; nrm[1] = p0.y; nrm[2] = p1.x; nrm[3] = p1.y; nrm[4] = p2.x; nrm[5] = p2.y;
            if (G.sigma_white != 0.0f) {
                uint4 wc = draw(P.seed, gid, a.step, TAG_FT_C);
                float2 p3 = box_muller(wb.z, wb.w), p4 = box_muller(wc.x, wc.y), p5 = box_muller(wc.z, wc.w);
                nrm[6] = p3.x; nrm[7] = p3.y; nrm[8] = p4.x; nrm[9] = p4.y; nrm[10] = p5.x; nrm[11] = p5.y;
            } else {
#pragma unroll
                for (int c = 6; c < 12; ++c) nrm[c] = 0.0f;
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                float dr = 0.0f;
                if (G.sigma_rw != 0.0f) {
                    dr = dr_prev[c] + G.sigma_rw * nrm[c];
                    __stcs(a.drift + (1 + c) * T + g, dr);
                }
                z[c] = z[c] + G.bias + G.sigma_white * nrm[6 + c] + dr;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) z[c] += G.bias;
        }
        const bool dead = bits & 4u;
        float stuck = 0.0f;
        if (dead) stuck = G.stuck_lo + G.stuck_span * u24(draw(P.seed, gid, ep, TAG_STUCK).y);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float v = quantise(G, z[c]);
            if (dead) v = stuck;
            __stcs(a.ft_noisy + c * T + g, v);
            S.fc[c][i] = v;
        }
    }
    __syncthreads();

    // ---- phase C2: noisy force/torque link sums
    link_sums(a, S, it, nl, true, tid, NT);
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
