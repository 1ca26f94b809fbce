// step.cu -- the fused per-taxel sensor step (Appendix A) and the episode
// reset.
//
// One CTA per work item: a run of whole links of one env (at most kItemCap
// taxels, kItemMaxLinks links).  Per-taxel arrays are SoA in HBM and read
// coalesced (consecutive threads, consecutive taxels).
//   phase A  per taxel: object-frame query (FP32, compensated near contact),
//            depth, Schmitt bit, force/torque, depth noise chain, force/
//            torque gain + hysteresis -> shared memory
//   phase C1 per link (one warp): clean sums, contact count, agg_force
//   phase B  per taxel: 3x3 crosstalk from shared memory, drift/white noise,
//            quantisation, dead override -> noisy force/torque
//   phase C2 per link: noisy sums
// Per-link sums use compensated (TwoSum) FP32 accumulation in a fixed lane
// order, so results are deterministic run to run.
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
    float dc[kItemCap], dn[kItemCap];   // clean / noisy depth
    uint8_t bits[kItemCap];             // bit0 clean contact, bit1 noisy contact
};

__device__ __forceinline__ float hyst_update(const NoiseDev& g, float x, float* prev_p, float* xi_p) {
    float xi = g.decay * (*xi_p) + (x - *prev_p);
    *xi_p = xi;
    *prev_p = x;
    return x + g.beta * xi;
}

__device__ __forceinline__ float quantise(const NoiseDev& g, float y) {
    return g.quant > 0.0f ? g.quant * rintf(y / g.quant) : y;
}

// compensated accumulation (Neumaier) and its warp-level combination
struct Acc {
    float s, c;
};
__device__ __forceinline__ void acc_add(Acc& a, float x) {
    float t = a.s + x;
    if (fabsf(a.s) >= fabsf(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}
__device__ __forceinline__ float acc_warp_total(Acc a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        float s2 = __shfl_xor_sync(0xffffffffu, a.s, off);
        float c2 = __shfl_xor_sync(0xffffffffu, a.c, off);
        df t = two_sum(a.s, s2);
        a.s = t.hi;
        a.c = a.c + c2 + t.lo;
    }
    return a.s + a.c;
}

template <int NT>
__global__ void __launch_bounds__(NT) step_kernel(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemStep& S = *reinterpret_cast<SmemStep*>(smem_raw);
    const Item it = a.items[blockIdx.x];
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
    }
    __syncthreads();

    const uint32_t ep = a.episode[e];
    const int64_t T = a.n_taxels;
    const ObjDev& obj = S.obj;

    // ---- phase A
    int l = 0;
    for (int i = tid; i < n; i += NT) {
        while (i >= S.start[l + 1]) ++l;
        const int64_t g = it.taxel_begin + i;
        const uint64_t gid = (uint64_t)(a.gid0 + g);
        const float R = __ldg(a.R + g);
        uint8_t flags = a.flags[g];
        if (!(R > 0.0f)) {  // inactive filler: every output zero, state untouched
            a.depth_clean[g] = 0.f;
            a.depth_noisy[g] = 0.f;
            if (a.sensors & TG_SENSOR_DIST) a.dist[g] = 0.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                a.ft_clean[c * T + g] = 0.f;
                S.hx[c][i] = 0.f;
                S.fc[c][i] = 0.f;
            }
            S.dc[i] = 0.f;
            S.dn[i] = 0.f;
            S.bits[i] = 0;
            a.flags[g] = flags & 2u;
            continue;
        }
        const float* rec = S.rec[l];
        const float x0 = __ldg(a.x + g), x1 = __ldg(a.y + g), x2 = __ldg(a.z + g);
        // object-frame query point, FP32
        float3 q = f3(fmaf(rec[0], x0, fmaf(rec[1], x1, fmaf(rec[2], x2, rec[18]))),
                      fmaf(rec[3], x0, fmaf(rec[4], x1, fmaf(rec[5], x2, rec[19]))),
                      fmaf(rec[6], x0, fmaf(rec[7], x1, fmaf(rec[8], x2, rec[20]))));
        const float scale = rec[38];
        float3 go;
        float phi = scale * sdf_fast(obj, q, &go);
        if (!isfinite(phi)) atomicAdd(a.err, 1u);
        float dist_out = phi - R;
        float d = 0.0f;
        bool y = false;
        const bool prev = flags & 1u;
        if (phi < R + 1e-6f) {
            // near contact: compensated query point and distance
            df qd[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                df acc = df{rec[18 + r], rec[21 + r]};
                acc = df_add(acc, df_mul_f(df{rec[3 * r], rec[9 + 3 * r]}, x0));
                acc = df_add(acc, df_mul_f(df{rec[3 * r + 1], rec[9 + 3 * r + 1]}, x1));
                acc = df_add(acc, df_mul_f(df{rec[3 * r + 2], rec[9 + 3 * r + 2]}, x2));
                qd[r] = acc;
            }
            df phid = df_mul_f(sdf_refine(obj, df3{qd[0], qd[1], qd[2]}, &go), scale);
            df dd = df_add_f(df_neg(phid), R);  // R - phi
            dist_out = -dd.hi;
            if (dd.hi > 0.0f) d = dd.hi;
            y = df_gt(dd, df{P.eta_on_hi, P.eta_on_lo}) || (prev && df_gt(dd, df{P.eta_off_hi, P.eta_off_lo}));
        }
        const bool dead = flags & 2u;
        const bool yn = y && !dead;
        a.flags[g] = (uint8_t)((y ? 1u : 0u) | (flags & 2u) | (yn ? 4u : 0u));

        // kinematic force/torque (Eqs. 4-9 with the Coulomb clamp)
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
        a.depth_clean[g] = d;
        if (a.sensors & TG_SENSOR_DIST) a.dist[g] = dist_out;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.ft_clean[c * T + g] = f[c];
            a.ft_clean[(3 + c) * T + g] = tq[c];
            S.fc[c][i] = f[c];
            S.fc[3 + c][i] = tq[c];
        }

        // noise: per-episode gains
        uint4 wep = make_uint4(0, 0, 0, 0);
        if (P.depth.gain_on | P.ft.gain_on) wep = draw(P.seed, gid, ep, TAG_EPISODE);
        const float gain_d = P.depth.gain_on ? P.depth.gain_lo + P.depth.gain_span * u24(wep.y) : 1.0f;
        const float gain_f = P.ft.gain_on ? P.ft.gain_lo + P.ft.gain_span * u24(wep.z) : 1.0f;
        // depth channel: gain, hysteresis, base noise, dead
        float xd = gain_d * d;
        if (P.depth.beta != 0.0f) xd = hyst_update(P.depth, xd, a.hyst_prev + g, a.hyst_xi + g);
        if (P.depth.sigma_rw != 0.0f || P.depth.sigma_white != 0.0f) {
            uint4 w = draw(P.seed, gid, a.step, TAG_SCALAR);
            float2 z = box_muller(w.x, w.y);
            float dr = 0.0f;
            if (P.depth.sigma_rw != 0.0f) {
                dr = a.drift[g] + P.depth.sigma_rw * z.x;
                a.drift[g] = dr;
            }
            xd = xd + P.depth.bias + P.depth.sigma_white * z.y + dr;
        } else {
            xd += P.depth.bias;
        }
        xd = quantise(P.depth, xd);
        if (dead) xd = P.depth.stuck_lo + P.depth.stuck_span * u24(draw(P.seed, gid, ep, TAG_STUCK).x);
        a.depth_noisy[g] = xd;
        S.dc[i] = d;
        S.dn[i] = xd;
        S.bits[i] = (uint8_t)((y ? 1u : 0u) | (yn ? 2u : 0u) | (dead ? 4u : 0u));
        // force/torque: gain and hysteresis now, crosstalk in phase B
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float v = gain_f * (c < 3 ? f[c] : tq[c - 3]);
            if (P.ft.beta != 0.0f) v = hyst_update(P.ft, v, a.hyst_prev + (1 + c) * T + g, a.hyst_xi + (1 + c) * T + g);
            S.hx[c][i] = v;
        }
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NW = NT / 32;

    // ---- phase C1: clean link sums
    for (int ll = warp; ll < nl; ll += NW) {
        const int s0 = S.start[ll], s1 = S.start[ll + 1];
        Acc acc[6], ag[3];
        for (int c = 0; c < 6; ++c) acc[c] = Acc{0.f, 0.f};
        for (int c = 0; c < 3; ++c) ag[c] = Acc{0.f, 0.f};
        int cnt = 0;
        for (int i = s0 + lane; i < s1; i += 32) {
            for (int c = 0; c < 6; ++c) acc_add(acc[c], S.fc[c][i]);
            const int64_t g = it.taxel_begin + i;
            const float dd = S.dc[i];
            if (dd != 0.0f) {
                acc_add(ag[0], dd * __ldg(a.nz + g));  // agg_force: 1e4 * ZYX(sum d n)
                acc_add(ag[1], dd * __ldg(a.ny + g));
                acc_add(ag[2], dd * __ldg(a.nx + g));
            }
            cnt += S.bits[i] & 1;
        }
        float tot[6], tag[3];
        for (int c = 0; c < 6; ++c) tot[c] = acc_warp_total(acc[c]);
        for (int c = 0; c < 3; ++c) tag[c] = acc_warp_total(ag[c]);
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (lane == 0) {
            float* o = a.link_out + (size_t)(e * L + lb + ll) * kLinkOut;
            for (int c = 0; c < 6; ++c) o[c] = tot[c];
            for (int c = 0; c < 3; ++c) o[12 + c] = 1e4f * tag[c];
            a.link_count[(size_t)(e * L + lb + ll) * 2] = cnt;
        }
    }
    __syncthreads();

    // ---- phase B: crosstalk, base noise, dead override
    l = 0;
    for (int i = tid; i < n; i += NT) {
        while (i >= S.start[l + 1]) ++l;
        const int64_t g = it.taxel_begin + i;
        const uint64_t gid = (uint64_t)(a.gid0 + g);
        const float R = __ldg(a.R + g);
        if (!(R > 0.0f)) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                a.ft_noisy[c * T + g] = 0.f;
                S.fc[c][i] = 0.f;
            }
            continue;
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
                    if (S.wrap[l]) c2 = (c2 + cols) % cols;
                    else if (c2 < 0 || c2 >= cols) continue;
                    const int nb = S.start[l] + rr * cols + c2;
                    const float w = P.xt_w[(di + 1) * 3 + (dj + 1)];
#pragma unroll
                    for (int c = 0; c < 6; ++c) conv[c] = fmaf(w, S.hx[c][nb], conv[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) z[c] = (1.0f - P.chi) * z[c] + P.chi * conv[c];
        }
        const NoiseDev& G = P.ft;
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
                    float* dp = a.drift + (1 + c) * T + g;
                    dr = *dp + G.sigma_rw * nrm[c];
                    *dp = dr;
                }
                z[c] = z[c] + G.bias + G.sigma_white * nrm[6 + c] + dr;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) z[c] += G.bias;
        }
        const bool dead = S.bits[i] & 4u;
        float stuck = 0.0f;
        if (dead) stuck = G.stuck_lo + G.stuck_span * u24(draw(P.seed, gid, ep, TAG_STUCK).y);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float v = quantise(G, z[c]);
            if (dead) v = stuck;
            a.ft_noisy[c * T + g] = v;
            S.fc[c][i] = v;
        }
    }
    __syncthreads();

    // ---- phase C2: noisy link sums
    for (int ll = warp; ll < nl; ll += NW) {
        const int s0 = S.start[ll], s1 = S.start[ll + 1];
        Acc acc[6], ag[3];
        for (int c = 0; c < 6; ++c) acc[c] = Acc{0.f, 0.f};
        for (int c = 0; c < 3; ++c) ag[c] = Acc{0.f, 0.f};
        int cnt = 0;
        for (int i = s0 + lane; i < s1; i += 32) {
            for (int c = 0; c < 6; ++c) acc_add(acc[c], S.fc[c][i]);
            const int64_t g = it.taxel_begin + i;
            const float dd = S.dn[i];
            if (dd != 0.0f) {
                acc_add(ag[0], dd * __ldg(a.nz + g));
                acc_add(ag[1], dd * __ldg(a.ny + g));
                acc_add(ag[2], dd * __ldg(a.nx + g));
            }
            cnt += (S.bits[i] >> 1) & 1;
        }
        float tot[6], tag[3];
        for (int c = 0; c < 6; ++c) tot[c] = acc_warp_total(acc[c]);
        for (int c = 0; c < 3; ++c) tag[c] = acc_warp_total(ag[c]);
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (lane == 0) {
            float* o = a.link_out + (size_t)(e * L + lb + ll) * kLinkOut;
            for (int c = 0; c < 6; ++c) o[6 + c] = tot[c];
            for (int c = 0; c < 3; ++c) o[15 + c] = 1e4f * tag[c];
            a.link_count[(size_t)(e * L + lb + ll) * 2 + 1] = cnt;
        }
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
