// pose.cu -- per-(env, link) pose prologue of a sensor step.
//
// Each link and its env's object are advanced by their constant velocities
// (p += v tau, R = exp([w] tau) R0 by Rodrigues' formula), then reduced to
// what the taxels of the link need (Appendix A, Eqs. 1 and 4-6):
//   q^ = M x + t         object-frame query point of a link-frame probe x,
//                        M = R_C^T R_L / s, t = R_C^T (p_L - p_C) / s
//   v_rel(x) = V + W_C x (x - p_LC) - W_L x x    link-frame relative velocity
//                        V = R_L^T (v_C - v_L), W_C = R_L^T w_C, W_L = R_L^T w_L,
//                        p_LC = R_L^T (p_C - p_L)
// M and t are kept as compensated float pairs: they carry the probe position
// to ~1e-14 relative, which the depth of near-contact taxels needs.
// The per-env mu, k and scale come from the caller, or, with per-step domain
// randomisation, from Philox (tag DR) for this env and step.
#include "df.cuh"
#include "internal.h"
#include "rng.cuh"

namespace tg {

struct dmat {
    df m[9];
};

__device__ dmat quat_to_dmat(const float* q) {
    df w = df_from(q[0]), x = df_from(q[1]), y = df_from(q[2]), z = df_from(q[3]);
    df n2 = df_add(df_add(df_mul(w, w), df_mul(x, x)), df_add(df_mul(y, y), df_mul(z, z)));
    df s = df_div(df_from(2.0f), n2);
    df xx = df_mul(x, x), yy = df_mul(y, y), zz = df_mul(z, z);
    df xy = df_mul(x, y), xz = df_mul(x, z), yz = df_mul(y, z);
    df wx = df_mul(w, x), wy = df_mul(w, y), wz = df_mul(w, z);
    df one = df_from(1.0f);
    dmat R;
    R.m[0] = df_sub(one, df_mul(s, df_add(yy, zz)));
    R.m[1] = df_mul(s, df_sub(xy, wz));
    R.m[2] = df_mul(s, df_add(xz, wy));
    R.m[3] = df_mul(s, df_add(xy, wz));
    R.m[4] = df_sub(one, df_mul(s, df_add(xx, zz)));
    R.m[5] = df_mul(s, df_sub(yz, wx));
    R.m[6] = df_mul(s, df_sub(xz, wy));
    R.m[7] = df_mul(s, df_add(yz, wx));
    R.m[8] = df_sub(one, df_mul(s, df_add(xx, yy)));
    return R;
}

__device__ dmat dmatmul(const dmat& A, const dmat& B) {
    dmat C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C.m[3 * i + j] = df_add(df_add(df_mul(A.m[3 * i], B.m[j]), df_mul(A.m[3 * i + 1], B.m[3 + j])),
                                    df_mul(A.m[3 * i + 2], B.m[6 + j]));
    return C;
}

// C = A^T B
__device__ dmat dmatTmul(const dmat& A, const dmat& B) {
    dmat C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C.m[3 * i + j] = df_add(df_add(df_mul(A.m[i], B.m[j]), df_mul(A.m[3 + i], B.m[3 + j])),
                                    df_mul(A.m[6 + i], B.m[6 + j]));
    return C;
}

// R(tau) = exp([w] tau) R(q0)
__device__ dmat advance_rotation(const float* q0, const float* w, df tau) {
    dmat R0 = quat_to_dmat(q0);
    df w2 = df_add(df_add(two_prod(w[0], w[0]), two_prod(w[1], w[1])), two_prod(w[2], w[2]));
    if (w2.hi == 0.0f || tau.hi == 0.0f) return R0;
    df wn = df_sqrt(w2);
    df k[3] = {df_div(df_from(w[0]), wn), df_div(df_from(w[1]), wn), df_div(df_from(w[2]), wn)};
    df th = df_mul(wn, tau);
    df s, c;
    df_sincos(th, &s, &c);
    df c1 = df_sub(df_from(1.0f), c);
    // E = I + s K + (1 - c) K^2, K^2 = k k^T - I
    dmat E;
    df K[9] = {df_from(0.f), df_neg(k[2]), k[1], k[2], df_from(0.f), df_neg(k[0]), df_neg(k[1]), k[0], df_from(0.f)};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            df kk = df_mul(k[i], k[j]);
            if (i == j) kk = df_add_f(kk, -1.0f);
            df v = df_add(df_mul(s, K[3 * i + j]), df_mul(c1, kk));
            if (i == j) v = df_add_f(v, 1.0f);
            E.m[3 * i + j] = v;
        }
    return dmatmul(E, R0);
}

constexpr int kPoseThreads = 128;

// lo + (hi - lo) u with u = (m + 1/2) 2^-24 (m the top 24 bits of x), formed
// as a float pair and rounded once to binary32: the FP64 value rounded.
__device__ __forceinline__ float dr_value(float lo, float hi, uint32_t x) {
    const df span = two_sum(hi, -lo);
    const df u = df{(float)(x >> 8) * 5.9604644775390625e-08f, 2.98023223876953125e-08f};
    return df_add(df_from(lo), df_mul(span, u)).hi;
}

// One thread per (env, link); the object pose of each env the block touches
// is advanced once, by one thread, into shared memory.
__global__ void __launch_bounds__(kPoseThreads) pose_kernel(const PoseArgs a) {
    __shared__ float s_obj[kPoseThreads][27];  // R_C as 9 float pairs, p_C as 3 float pairs, mu k scale
    const int L = a.max_links;
    const int n = a.n_envs * L;
    const int base = blockIdx.x * kPoseThreads;
    const int idx = base + threadIdx.x;
    const int e0 = base / L;
    const int e_last = min(base + kPoseThreads, n) - 1;
    const int n_env = e_last / L - e0 + 1;
    df tau{a.tau_hi, a.tau_lo};
    uint32_t step = a.step;
    if (a.ctl) {
        const StepCtl c = *a.ctl;
        step = c.step;
        tau = df_add(df{c.tau0_hi, c.tau0_lo}, df_mul_f(df{c.dtau_hi, c.dtau_lo}, (float)c.replay));
    }
    if ((int)threadIdx.x < n_env) {
        const int e = e0 + threadIdx.x;
        const float* op = a.obj_pose + (size_t)e * 7;
        const float* ov = a.obj_vel + (size_t)e * 6;
        float oq[4] = {op[3], op[4], op[5], op[6]}, ow[3] = {ov[3], ov[4], ov[5]};
        dmat RC = advance_rotation(oq, ow, tau);
        float* o = s_obj[threadIdx.x];
#pragma unroll
        for (int i = 0; i < 9; ++i) { o[2 * i] = RC.m[i].hi; o[2 * i + 1] = RC.m[i].lo; }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            df p = df_add(df_from(op[i]), df_mul_f(tau, ov[i]));
            o[18 + 2 * i] = p.hi;
            o[19 + 2 * i] = p.lo;
        }
        float mu = a.def_mu, k = a.def_k, scale = 1.0f;
        if (a.dr_on) {
            const uint4 w = draw(a.seed, (uint64_t)(a.env_gid0 + e), step, TAG_DR);
            mu = dr_value(a.dr_lo[0], a.dr_hi[0], w.x);
            k = dr_value(a.dr_lo[1], a.dr_hi[1], w.y);
            scale = dr_value(a.dr_lo[2], a.dr_hi[2], w.z);
        } else if (a.env_params) {
            mu = a.env_params[3 * e];
            k = a.env_params[3 * e + 1];
            scale = a.env_params[3 * e + 2];
        }
        o[24] = mu;
        o[25] = k;
        o[26] = scale;
    }
    __syncthreads();
    // each thread's record is staged in shared memory; the block's records
    // (one contiguous range) are then written with coalesced 16-byte stores
    __shared__ __align__(16) float s_rec[kPoseThreads * kLinkRec];
    float* rec = s_rec + threadIdx.x * kLinkRec;
    const bool live = idx < n && a.lattice[idx].present;
    if (!live) {
        for (int f = 0; f < kLinkRec; ++f) rec[f] = 0.0f;  // absent links: a zero record
    } else {
        const int e = idx / L;
        const float* lp = a.link_pose + (size_t)idx * 7;
        const float* lv = a.link_vel + (size_t)idx * 6;
        const float* ov = a.obj_vel + (size_t)e * 6;
        const float* o = s_obj[e - e0];
        const float mu = o[24], k = o[25], scale = o[26];
        dmat RC;
#pragma unroll
        for (int i = 0; i < 9; ++i) RC.m[i] = df{o[2 * i], o[2 * i + 1]};
        float lq[4] = {lp[3], lp[4], lp[5], lp[6]};
        float lw[3] = {lv[3], lv[4], lv[5]}, ow[3] = {ov[3], ov[4], ov[5]};
        dmat RL = advance_rotation(lq, lw, tau);
        df dp[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const df pL = df_add(df_from(lp[i]), df_mul_f(tau, lv[i]));
            dp[i] = df_sub(pL, df{o[18 + 2 * i], o[19 + 2 * i]});  // p_L - p_C
        }
        dmat M = dmatTmul(RC, RL);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            df m = df_div_f(M.m[i], scale);
            rec[i] = m.hi;
            rec[9 + i] = m.lo;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            df t = df_add(df_add(df_mul(RC.m[i], dp[0]), df_mul(RC.m[3 + i], dp[1])), df_mul(RC.m[6 + i], dp[2]));
            t = df_div_f(t, scale);
            rec[18 + i] = t.hi;
            rec[21 + i] = t.lo;
        }
        // velocity terms in the link frame (FP32 is enough here)
        float dv[3] = {ov[0] - lv[0], ov[1] - lv[1], ov[2] - lv[2]};
        float nd[3] = {-dp[0].hi - dp[0].lo, -dp[1].hi - dp[1].lo, -dp[2].hi - dp[2].lo};  // p_C - p_L
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float r0 = RL.m[i].hi, r1 = RL.m[3 + i].hi, r2 = RL.m[6 + i].hi;  // column i of R_L
            rec[24 + i] = r0 * dv[0] + r1 * dv[1] + r2 * dv[2];
            rec[27 + i] = r0 * ow[0] + r1 * ow[1] + r2 * ow[2];
            rec[30 + i] = r0 * lw[0] + r1 * lw[1] + r2 * lw[2];
            rec[33 + i] = r0 * nd[0] + r1 * nd[1] + r2 * nd[2];
        }
        rec[36] = k;
        rec[37] = mu;
        rec[38] = scale;
        rec[39] = 0.0f;
    }
    __syncthreads();
    const int n_block = min(kPoseThreads, n - base);  // records of this block
    float4* dst = reinterpret_cast<float4*>(a.link_rec + (size_t)base * kLinkRec);
    const float4* src = reinterpret_cast<const float4*>(s_rec);
    for (int v = threadIdx.x; v < n_block * kLinkRec / 4; v += kPoseThreads) dst[v] = src[v];
}

cudaError_t launch_pose(const PoseArgs& a, cudaStream_t s) {
    const int n = a.n_envs * a.max_links;
    if (n == 0) return cudaSuccess;
    pose_kernel<<<(n + kPoseThreads - 1) / kPoseThreads, kPoseThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tg
