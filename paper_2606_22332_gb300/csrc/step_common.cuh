// step_common.cuh -- per-taxel pieces of the fused sensor step (step.cu).
// Each routine follows one passage of the paper:
//   fast_query      FP32 object-frame query point and SDF (Eqs. 1-2)
//   clear_taxel     outputs of a taxel clear of the surface: depth 0, no
//                   contact, no force (Eqs. 2-3, 8-9 with d = 0)
//   refine_taxel    near-contact taxel: compensated query point and SDF,
//                   depth, Schmitt bit (Eq. 3), force/torque with the Coulomb
//                   clamp (Eqs. 4-9)
//   noise_state     gain, hysteresis (Eqs. 27, 29-30), depth base noise and
//                   dead override (Eqs. 25, 28), agg_force terms (Eq. 32)
//   noisy_ft        3x3 crosstalk (Eq. 31), drift / white noise,
//                   quantisation, dead override of the force/torque channels
// Smem is any shared-memory layout with the per-taxel arrays fc, hx
// ([6][capacity] floats), dn ([5][capacity]: clean depth, noisy depth,
// probe normal) and bits.
#pragma once
#include <cstdint>

#include "df.cuh"
#include "geom.cuh"
#include "internal.h"
#include "rng.cuh"

namespace tg {

// per-taxel bits in shared memory
enum : uint8_t { BIT_CLEAN = 1, BIT_NOISY = 2, BIT_DEAD = 4, BIT_ACTIVE = 8, BIT_NEAR = 16 };

__device__ __forceinline__ float hyst_update(const NoiseDev& g, float x, float* prev_p, float* xi_p) {
    float xi = g.decay * __ldcs(xi_p) + (x - __ldcs(prev_p));
    __stcs(xi_p, xi);
    __stcs(prev_p, x);
    return x + g.beta * xi;
}

// q rint(y / q); the step (q = 0: off) is a parameter of the scene, so the
// division sits behind a branch every thread takes alike
__device__ __forceinline__ float quantise(const NoiseDev& g, float y) {
    if (g.quant > 0.0f) y = g.quant * rintf(y / g.quant);
    return y;
}

// the stuck readout of a dead taxel, lo + span u (one draw; none when the
// span is 0, as when dead taxels read a constant)
__device__ __forceinline__ float stuck_value(const ParamsDev& P, const NoiseDev& g, uint64_t gid, uint32_t ep,
                                             int word) {
    if (g.stuck_span == 0.0f) return g.stuck_lo;
    const uint4 w = draw_rk(P.rk, gid, ep, TAG_STUCK);
    return g.stuck_lo + g.stuck_span * u24(word == 0 ? w.x : (word == 1 ? w.y : w.z));
}

// compensated accumulation (Kahan): the sum's error stays within ~2 eps
// sum |x| whatever the order of magnitudes, at four additions a term
struct Acc {
    float s, c;
};
__device__ __forceinline__ void acc_add(Acc& a, float x) {
    const float y = x - a.c;
    const float t = a.s + y;
    a.c = (t - a.s) - y;
    a.s = t;
}
// the sum, with the last term's lost part put back
__device__ __forceinline__ float acc_value(const Acc& a) { return a.s - a.c; }

// Compensated sum of a link's terms src[s0..s1) (deterministic): Kahan
// accumulators over the even and the odd positions, two independent
// dependency chains side by side, then combined.
__device__ __forceinline__ Acc link_acc(const float* src, int s0, int s1) {
    Acc e{0.f, 0.f}, o{0.f, 0.f};
    int i = s0;
#pragma unroll 4
    for (; i + 1 < s1; i += 2) {
        acc_add(e, src[i]);
        acc_add(o, src[i + 1]);
    }
    if (i < s1) acc_add(e, src[i]);
    acc_add(e, o.s);
    acc_add(e, -o.c);
    return e;
}
__device__ __forceinline__ float link_sum(const float* src, int s0, int s1) { return acc_value(link_acc(src, s0, s1)); }

// the sum of two partial sums, the first then the second
__device__ __forceinline__ float acc_join(Acc e, const Acc& o) {
    acc_add(e, o.s);
    acc_add(e, -o.c);
    return acc_value(e);
}
// the midpoint at which link_sum_halves splits [s0, s1)
__device__ __forceinline__ int link_mid(int s0, int s1) { return s0 + (s1 - s0) / 2; }
// link_sum over the two halves of [s0, s1) apart, then joined: the form of
// the noisy force/torque sums, which the grid and persistent schedules run
// on two threads (a half each, joined through a shuffle)
__device__ __forceinline__ float link_sum_halves(const float* src, int s0, int s1) {
    const int m = link_mid(s0, s1);
    return acc_join(link_acc(src, s0, m), link_acc(src, m, s1));
}

// the same for the terms d[i] n[i], each product rounded on its own
__device__ __forceinline__ float link_sum_prod(const float* d, const float* n, int s0, int s1) {
    Acc e{0.f, 0.f}, o{0.f, 0.f};
    int i = s0;
#pragma unroll 4
    for (; i + 1 < s1; i += 2) {
        acc_add(e, __fmul_rn(d[i], n[i]));
        acc_add(o, __fmul_rn(d[i + 1], n[i + 1]));
    }
    if (i < s1) acc_add(e, __fmul_rn(d[i], n[i]));
    acc_add(e, o.s);
    acc_add(e, -o.c);
    return acc_value(e);
}

// Link of item taxel i (and, in B, its lattice row and column) for a uniform
// item: l = floor((i + 1/2) / len) evaluated as (i + 1/2) * fl(1/len) in
// FP32.  The quotient lies at least 1/(2 len) from an integer while the two
// roundings move it by at most 2^-23 (i + 1/2) / len; for i < 1024 and
// len <= 1024 that is below 1.3e-4 < 1/(2 len), so the floor is exact.
__device__ __forceinline__ int uni_div(int i, float inv) { return (int)(((float)i + 0.5f) * inv); }

// link of item taxel i from the item's static layout
__device__ __forceinline__ int meta_link_of(const ItemMeta& M, int i) {
    if (M.uni_len) return uni_div(i, M.uni_inv_len);
    int lo = 0, hi = M.nl - 1;  // last start <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (M.start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Objects whose phi comes from a query kernel run ahead of the step kernel:
// a learned SDF, and a mesh answered by the raycast backend (its phi is a
// float pair, hi in nq_phi and lo in nq_phi_lo; a phi above R + 1 um marks a
// probe with no triangle within reach, whose surface-distance output is 0).
__device__ __forceinline__ bool phi_precomputed(const ObjDev& o, const ParamsDev& P) {
    return o.kind == TG_OBJ_NEURAL || (o.kind == TG_OBJ_MESH && P.depth_backend != 0);
}
__device__ __forceinline__ bool raycast_obj(const ObjDev& o, const ParamsDev& P) {
    return o.kind == TG_OBJ_MESH && P.depth_backend != 0;
}

// FP32 object-frame query point q^ = M x + t and scaled SDF s phi(q^).
// GRID: the object is known to be a plain SDF grid (a kernel form compiled
// for scenes whose objects are all grids: no dispatch on the kind).
template <bool GRID = false>
__device__ __forceinline__ float fast_query(const float* rec, const ObjDev& obj, float x0, float x1, float x2) {
    const float3 q = f3(fmaf(rec[0], x0, fmaf(rec[1], x1, fmaf(rec[2], x2, rec[18]))),
                        fmaf(rec[3], x0, fmaf(rec[4], x1, fmaf(rec[5], x2, rec[19]))),
                        fmaf(rec[6], x0, fmaf(rec[7], x1, fmaf(rec[8], x2, rec[20]))));
    return rec[38] * (GRID ? grid_phi_fast(obj, q) : sdf_phi_fast(obj, q));
}

// A taxel clear of the surface (or an inactive filler, R = 0): depth 0,
// contact off, zero force.  Stores its flag byte and surface distance (the
// zero clean depth and force/torque are stored with the noise state, after
// last step's values have been read there) and returns its shared-memory
// bits.
__device__ __forceinline__ uint8_t clear_taxel(const StepArgs& a, tidx g, float R, uint8_t flags, float phi) {
    __stcs(a.flags + g, (uint8_t)(flags & 2u));
    if (a.sensors & TG_SENSOR_DIST) __stcs(a.dist + g, R > 0.0f ? phi - R : 0.0f);
    return (uint8_t)(((flags & 2u) ? BIT_DEAD : 0u) | (R > 0.0f ? BIT_ACTIVE : 0u));
}

struct CleanReading {
    float d;
    float f[3], tq[3];
    // with probe-radius noise: the depth and force the noisy chain starts from
    float dn;
    float fn[3], tqn[3];
    uint8_t bits;
    uint8_t flags;   // the taxel's new flag byte
    float dist;      // surface distance phi - R
};

// A near-contact taxel at link-frame position (x0, x1, x2) with probe radius
// R and last step's flag byte: compensated query point and SDF (near-contact
// depths carry ~1e-14 relative error), depth, Schmitt decision on the
// compensated depth, force/torque, the new flag byte.  With probe-radius
// noise the noisy readout's radius max(0, R + eps) gives a second depth, its
// own Schmitt decision (flag bit 2) and a second force (same normal and
// velocities).  Pure: the caller stores the results (store_clean).
template <bool RADIUS, bool GRID = false>  // probe-radius noise on (rho > 0); GRID as in fast_query
__device__ __forceinline__ CleanReading refine_compute(const ParamsDev& P, const float* nq_phi, const float* nq_phi_lo,
                                                       const float* nq_grad, int64_t T, int64_t gid0,
                                                       const float* rec, const ObjDev& obj,
                                                       tidx g, float x0, float x1, float x2, float R,
                                                       uint8_t flags, uint32_t step) {
    // compensated query point (sums with df_add_abs's absolute bound, ~1e-15 m
    // for coordinates of a few centimetres)
    df qd[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        df acc = df{rec[18 + r], rec[21 + r]};
        acc = df_add_abs(acc, df_mul_f(df{rec[3 * r], rec[9 + 3 * r]}, x0));
        acc = df_add_abs(acc, df_mul_f(df{rec[3 * r + 1], rec[9 + 3 * r + 1]}, x1));
        acc = df_add_abs(acc, df_mul_f(df{rec[3 * r + 2], rec[9 + 3 * r + 2]}, x2));
        qd[r] = acc;
    }
    float3 go;
    const float scale = rec[38];
    df phid;
    if (!GRID && phi_precomputed(obj, P)) {
        // a learned SDF has no compensated form (its FP32 phi and gradient);
        // the raycast backend's phi is a compensated pair (its face normal)
        phid = raycast_obj(obj, P) ? df{nq_phi[g], nq_phi_lo[g]} : df_from(nq_phi[g]);
        go = f3(nq_grad[g], nq_grad[T + g], nq_grad[2 * T + g]);
    } else {
        const df3 qq{qd[0], qd[1], qd[2]};
        phid = df_mul_f(GRID ? grid_refine(obj, qq, &go) : sdf_refine(obj, qq, &go), scale);
    }
    const df dd = df_add_f(df_neg(phid), R);  // R - phi
    CleanReading out;
    out.d = dd.hi > 0.0f ? dd.hi : 0.0f;
    out.dist = -dd.hi;
    const df eta_on = df{P.eta_on_hi, P.eta_on_lo}, eta_off = df{P.eta_off_hi, P.eta_off_lo};
    const bool prev = flags & 1u;
    const bool y = df_gt(dd, eta_on) || (prev && df_gt(dd, eta_off));
    const bool dead = flags & 2u;
    bool yn = y && !dead;
    out.dn = out.d;
    if constexpr (RADIUS) {
        // eps = rho (2u - 1) in binary32 (2u - 1 is exact); R + eps exact as a pair
        const float u = u24(draw_rk(P.rk, (uint64_t)(gid0 + g), step, TAG_RADIUS).x);
        const float eps = P.rho * (2.0f * u - 1.0f);
        df Rn = df_add_f(df_from(R), eps);
        if (df_lt(Rn, df_from(0.0f))) Rn = df_from(0.0f);
        const df ddn = df_add(df_neg(phid), Rn);  // R~ - phi
        out.dn = ddn.hi > 0.0f ? ddn.hi : 0.0f;
        const bool prevn = flags & 4u;
        yn = (df_gt(ddn, eta_on) || (prevn && df_gt(ddn, eta_off))) && !dead;
    }
    out.flags = (uint8_t)((y ? 1u : 0u) | (flags & 2u) | (yn ? 4u : 0u));
#pragma unroll
    for (int c = 0; c < 3; ++c) { out.f[c] = 0.f; out.tq[c] = 0.f; out.fn[c] = 0.f; out.tqn[c] = 0.f; }
    const float d = out.d, dn = out.dn;
    if (d > 0.0f || (RADIUS && dn > 0.0f)) {
        const float3 mb = normalize_or(f3(rec[0] * go.x + rec[3] * go.y + rec[6] * go.z,
                                          rec[1] * go.x + rec[4] * go.y + rec[7] * go.z,
                                          rec[2] * go.x + rec[5] * go.y + rec[8] * go.z),
                                       f3(0.f, 0.f, 1.f));
        const float3 xv = f3(x0, x1, x2);
        const float3 V = f3(rec[24], rec[25], rec[26]), Wc = f3(rec[27], rec[28], rec[29]);
        const float3 Wl = f3(rec[30], rec[31], rec[32]), pLC = f3(rec[33], rec[34], rec[35]);
        const float3 vrel = V + cross(Wc, xv - pLC) - cross(Wl, xv);
        const float kk = rec[36], mu = rec[37];
        const float vns = dot(vrel, mb);
        const float3 vn = mb * vns;
        const float3 vt = vrel - vn;
        const float vtn = sqrtf(dot(vt, vt));
        const float spin = P.k_omega * dot(Wc - Wl, mb);
        // Eqs. 4-9 with the Coulomb clamp at depth dep
        auto force = [&](float dep, float* f, float* tq) {
            float s = dep;
            if (P.alpha != 1.0f) s = powf(dep, P.alpha);
            const float3 fnv = mb * (kk * s) + vn * (P.c * s);
            float sc = 1.0f;
            if (mu >= 0.0f && P.k_t * vtn > 0.0f) sc = fminf(1.0f, mu * sqrtf(dot(fnv, fnv)) / (P.k_t * vtn));
            const float3 ff = fnv - vt * (P.k_t * sc);
            const float3 tt = cross(xv, ff) - mb * spin;
            f[0] = ff.x; f[1] = ff.y; f[2] = ff.z;
            tq[0] = tt.x; tq[1] = tt.y; tq[2] = tt.z;
        };
        if (d > 0.0f) force(d, out.f, out.tq);
        if (RADIUS && dn > 0.0f) force(dn, out.fn, out.tqn);
    }
    out.bits = (uint8_t)((y ? BIT_CLEAN : 0u) | (yn ? BIT_NOISY : 0u) | (dead ? BIT_DEAD : 0u) | BIT_ACTIVE |
                         (RADIUS ? BIT_NEAR : 0u));
    return out;
}

// the flag byte and surface distance of a refined taxel (its clean depth and
// force/torque are stored with the noise state, see clear_taxel)
__device__ __forceinline__ void store_clean(const StepArgs& a, tidx g, const CleanReading& cr) {
    __stcs(a.flags + g, cr.flags);
    if (a.sensors & TG_SENSOR_DIST) __stcs(a.dist + g, cr.dist);
}

// The clean depth and force/torque outputs of taxel g, stored in the noise
// state phase: with prev_out the previous values there are the hysteresis
// state, read by that phase first.
__device__ __forceinline__ void store_clean_out(const StepArgs& a, tidx g, float d, const float* f) {
    const int64_t T = a.n_taxels;
    __stcs(a.depth_clean + g, d);
#pragma unroll
    for (int c = 0; c < 6; ++c) __stcs(a.ft_clean + c * T + g, f[c]);
}

template <bool RADIUS, bool GRID = false>
__device__ __forceinline__ CleanReading refine_taxel(const StepArgs& a, const float* rec, const ObjDev& obj,
                                                     tidx g, float x0, float x1, float x2, float R,
                                                     uint8_t flags, uint32_t step) {
    const CleanReading cr = refine_compute<RADIUS, GRID>(a.P, a.nq_phi, a.nq_phi_lo, a.nq_grad, a.n_taxels, a.gid0, rec,
                                                   obj, g, x0, x1, x2, R, flags, step);
    store_clean(a, g, cr);
    return cr;
}

// The noise state a taxel's step reads (hysteresis x_{t-1} and xi of the
// depth and six force/torque channels, the depth drift) and what the step
// leaves of it.  With prev_out, prev_d and pv hold last step's clean depth
// and force/torque, which the gain turns into x_{t-1}.
struct NoiseIn {
    float prev_d, xi_d, drift_d;
    float pv[6], xv[6];
};
struct NoiseOut {
    float prev_d, xi_d, drift_d;   // new state (stored where the group has it)
    float pv[6], xv[6];
    float xd;                      // noisy depth
    float hx[6];                   // force/torque after gain and hysteresis (crosstalk input)
};

// which state a parameter set reads and writes
__device__ __forceinline__ bool hyst_depth_on(const ParamsDev& P) { return P.depth.beta != 0.0f; }
__device__ __forceinline__ bool hyst_ft_on(const ParamsDev& P) { return P.ft.beta != 0.0f; }
__device__ __forceinline__ bool drift_depth_on(const ParamsDev& P) { return P.depth.sigma_rw != 0.0f; }
__device__ __forceinline__ bool drift_ft_on(const ParamsDev& P) { return P.ft.sigma_rw != 0.0f; }

// Noise state of one active taxel from its clean depth d and the depth and
// force/torque its noisy chain starts from (d_in, f_in: the clean ones, or
// those of the perturbed radius): gain, hysteresis (Eqs. 27, 29-30), depth
// base noise and dead override (Eqs. 25, 28).  Pure.
__device__ __forceinline__ NoiseOut noise_core(const ParamsDev& P, uint64_t gid, uint32_t ep, uint32_t step,
                                               uint8_t bits, float d_in, const float* f_in, const NoiseIn& s) {
    NoiseOut o;
    const bool hyst_d = hyst_depth_on(P), hyst_f = hyst_ft_on(P), walk_d = drift_depth_on(P);
    const bool dead = bits & BIT_DEAD;
    uint4 wep = make_uint4(0, 0, 0, 0);
    if (P.depth.gain_on | P.ft.gain_on) wep = draw_rk(P.rk, gid, ep, TAG_EPISODE);
    const float gain_d = P.depth.gain_on ? P.depth.gain_lo + P.depth.gain_span * u24(wep.y) : 1.0f;
    const float gain_f = P.ft.gain_on ? P.ft.gain_lo + P.ft.gain_span * u24(wep.z) : 1.0f;
    float xd = gain_d * d_in;
    // x_{t-1} = gain * last step's input: the same product as stored then
    const float prev_d = P.prev_out ? gain_d * s.prev_d : s.prev_d;
    o.prev_d = prev_d;
    o.xi_d = s.xi_d;
    if (hyst_d) {
        const float xi = P.depth.decay * s.xi_d + (xd - prev_d);
        o.xi_d = xi;
        o.prev_d = xd;
        xd = xd + P.depth.beta * xi;
    }
    if (hyst_f) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float x = gain_f * f_in[c];
            const float pv = P.prev_out ? gain_f * s.pv[c] : s.pv[c];
            const float xi = P.ft.decay * s.xv[c] + (x - pv);
            o.xv[c] = xi;
            o.pv[c] = x;
            o.hx[c] = x + P.ft.beta * xi;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            o.xv[c] = s.xv[c];
            o.pv[c] = s.pv[c];
            o.hx[c] = gain_f * f_in[c];
        }
    }
    o.drift_d = s.drift_d;
    if (P.depth.sigma_rw != 0.0f || P.depth.sigma_white != 0.0f) {
        uint4 w = draw_rk(P.rk, gid, step, TAG_SCALAR);
        float2 z = box_muller(w.x, w.y);
        float dr = 0.0f;
        if (walk_d) {
            dr = s.drift_d + P.depth.sigma_rw * z.x;
            o.drift_d = dr;
        }
        xd = xd + P.depth.bias + P.depth.sigma_white * z.y + dr;
    } else {
        xd += P.depth.bias;
    }
    xd = quantise(P.depth, xd);
    if (dead) xd = stuck_value(P, P.depth, gid, ep, 0);
    o.xd = xd;
    return o;
}

// Read delay (Appendix "Sensor Noise Model", base noise: the noisy readout is
// formed from y_{t - Delta_read}, with optional uniform jitter) of the env
// with global id env_gid at this step: delay + j, j uniform on {0..jitter}
// from the top 24 bits of Philox word 0 at (env id, step, TAG_JITTER), as an
// integer product.
__device__ __forceinline__ int read_delay(const ParamsDev& P, uint64_t env_gid, uint32_t step) {
    if (P.jitter <= 0) return P.delay;
    const uint32_t w = draw_rk(P.rk, env_gid, step, TAG_JITTER).x;
    return P.delay + (int)(((uint64_t)(w >> 8) * (uint64_t)(P.jitter + 1)) >> 24);
}

// The read delay's history ([ring_k][8][T]: slot, then channel 0 depth, 1-6
// force/torque, 7 the noisy contact bit): this step's noisy-chain input goes
// into slot step mod ring_k, and the input of `rd` steps earlier comes out
// of its slot into d_in, f_in and the returned bit (with rd = 0, the values
// just written).
__device__ __forceinline__ bool ring_step(const ParamsDev& P, float* ring, int64_t T, tidx g, uint32_t step,
                                          int rd, float& d_in, float* f_in, bool bit) {
    const uint32_t K = (uint32_t)P.ring_k;
    const uint32_t ws = step % K, rs = (ws + K - (uint32_t)rd) % K;
    float* w = ring + (size_t)ws * 8 * T + g;
    w[0] = d_in;
#pragma unroll
    for (int c = 0; c < 6; ++c) w[(1 + c) * T] = f_in[c];
    w[7 * T] = bit ? 1.0f : 0.0f;
    const float* r = ring + (size_t)rs * 8 * T + g;
    d_in = r[0];
#pragma unroll
    for (int c = 0; c < 6; ++c) f_in[c] = r[(1 + c) * T];
    return r[7 * T] != 0.0f;
}

// With a read delay: the delayed noisy-chain input replaces (d_in, f_in),
// the reported noisy contact (the delayed bit, then the dead override) goes
// into flag bit 3 and replaces BIT_NOISY in the returned bits.
__device__ __forceinline__ uint8_t delay_readout(const StepArgs& a, tidx g, uint32_t step, int rd, uint8_t bits,
                                                 float& d_in, float* f_in) {
    const bool yn = bits & BIT_NOISY;
    const bool rep = ring_step(a.P, a.ring, a.n_taxels, g, step, rd, d_in, f_in, yn) && !(bits & BIT_DEAD);
    __stcs(a.flags + g, (uint8_t)(((bits & BIT_CLEAN) ? 1u : 0u) | ((bits & BIT_DEAD) ? 2u : 0u) | (yn ? 4u : 0u) |
                                  (rep ? 8u : 0u)));
    return (uint8_t)((bits & ~BIT_NOISY) | (rep ? BIT_NOISY : 0u));
}

// Noise state of one active taxel after its clean reading (fc[.][i] and the
// clean depth in ag[0][i]), from and to the state arrays in HBM; stores the
// clean depth and force/torque outputs (with prev_out, after reading last
// step's values there as x_{t-1}).  The state
// loads do not depend on the geometry, and all of them are issued before
// the first store: the compiler cannot move a load above a store to a
// pointer that may alias it, and every such barrier would cost a further
// round trip to memory.
// (n0, n1, n2) is the taxel's probe normal, loaded by the caller (from HBM
// or from a staged copy in shared memory).
// The noise state taxel g's step reads (loads only; noise_apply uses it).
__device__ __forceinline__ NoiseIn noise_load(const StepArgs& a, tidx g) {
    const ParamsDev& P = a.P;
    const int64_t T = a.n_taxels;
    const bool hyst_d = hyst_depth_on(P), hyst_f = hyst_ft_on(P), walk_d = drift_depth_on(P);
    NoiseIn s;
    s.prev_d = s.xi_d = s.drift_d = 0.0f;
#pragma unroll
    for (int c = 0; c < 6; ++c) s.pv[c] = s.xv[c] = 0.0f;
    // x_{t-1}: kept in hyst_prev, or with prev_out last step's clean output
    const float* prev_d_src = P.prev_out ? a.depth_clean : a.hyst_prev;
    const float* prev_f_src = P.prev_out ? a.ft_clean : a.hyst_prev + T;
    if (hyst_d) {
        s.prev_d = __ldcs(prev_d_src + g);
        s.xi_d = __ldcs(a.hyst_xi + g);
    }
    if (hyst_f) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            s.pv[c] = __ldcs(prev_f_src + c * T + g);
            s.xv[c] = __ldcs(a.hyst_xi + (1 + c) * T + g);
        }
    }
    if (walk_d) s.drift_d = __ldcs(a.drift + g);
    return s;
}

// noise_state from state already loaded (noise_load), so that a thread can
// have several taxels' loads in flight before the first of them is used
template <bool RADIUS, class Smem>
__device__ __forceinline__ void noise_apply(const StepArgs& a, Smem& S, int i, tidx g, uint32_t ep, uint32_t step,
                                            uint8_t bits, float n0, float n1, float n2, const NoiseIn& s) {
    const ParamsDev& P = a.P;
    const int64_t T = a.n_taxels;
    const bool hyst_d = hyst_depth_on(P), hyst_f = hyst_ft_on(P), walk_d = drift_depth_on(P);
    const float d = S.dn[0][i];
    // the depth and force the noisy chain starts from: the clean ones, or with
    // probe-radius noise those of the perturbed radius (refined taxels; the
    // others are clear of it)
    float d_in = d, f_in[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) f_in[c] = S.fc[c][i];
    if constexpr (RADIUS) {
        const bool near = bits & BIT_NEAR;
        d_in = near ? S.dn[1][i] : 0.0f;
#pragma unroll
        for (int c = 0; c < 6; ++c) f_in[c] = near ? S.hx[c][i] : 0.0f;
    }
    if (P.ring_k > 1) {
        bits = delay_readout(a, g, step, S.rdelay, bits, d_in, f_in);
        S.bits[i] = bits;
    }
    const NoiseOut o = noise_core(P, (uint64_t)(a.gid0 + g), ep, step, bits, d_in, f_in, s);
    {
        float fc[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) fc[c] = S.fc[c][i];
        store_clean_out(a, g, d, fc);
    }
    if (hyst_d) {
        __stcs(a.hyst_xi + g, o.xi_d);
        if (!P.prev_out) __stcs(a.hyst_prev + g, o.prev_d);
    }
    if (hyst_f) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            __stcs(a.hyst_xi + (1 + c) * T + g, o.xv[c]);
            if (!P.prev_out) __stcs(a.hyst_prev + (1 + c) * T + g, o.pv[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) S.hx[c][i] = o.hx[c];
    if (walk_d) __stcs(a.drift + g, o.drift_d);
    __stcs(a.depth_noisy + g, o.xd);
    S.dn[1][i] = o.xd;
    S.dn[2][i] = n0; S.dn[3][i] = n1; S.dn[4][i] = n2;
}

template <bool RADIUS, class Smem>
__device__ __forceinline__ void noise_state(const StepArgs& a, Smem& S, int i, tidx g, uint32_t ep, uint32_t step,
                                            uint8_t bits, float n0, float n1, float n2) {
    const NoiseIn s = noise_load(a, g);
    noise_apply<RADIUS>(a, S, i, g, ep, step, bits, n0, n1, n2, s);
}

// Inactive filler: zero clean and noisy depth, clean force/torque and
// staged values.
template <class Smem>
__device__ __forceinline__ void noise_state_filler(const StepArgs& a, Smem& S, int i, tidx g) {
    const float zero[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    store_clean_out(a, g, 0.f, zero);
    __stcs(a.depth_noisy + g, 0.f);
#pragma unroll
    for (int c = 0; c < 6; ++c) S.hx[c][i] = 0.f;
#pragma unroll
    for (int c = 0; c < 5; ++c) S.dn[c][i] = 0.f;
}

// 3x3 crosstalk (Eq. 31) of the six force/torque channels at taxel i,
// lattice (r, cc) of a rows x cols lattice whose first taxel is `base` in
// hx ([6][kItemCap]): z = (1 - chi) hx_i + chi sum_k w_k hx_k, without
// branches: a neighbour off the lattice (no wrap) gets weight 0 and the
// taxel's own index, so every tap is a plain shared-memory load.
__device__ __forceinline__ void crosstalk(const ParamsDev& P, const float (*hx)[kItemCap], int i, int base, int r,
                                          int cc, int rows, int cols, bool wrap, float* z) {
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] = hx[c][i];
    if (P.chi == 0.0f) return;
    const bool vu = r > 0, vd = r + 1 < rows;
    int cl = cc - 1, cr = cc + 1;
    bool vl = true, vr = true;
    if (cl < 0) {
        if (wrap) cl += cols;
        else { vl = false; cl = cc; }
    }
    if (cr >= cols) {
        if (wrap) cr -= cols;
        else { vr = false; cr = cc; }
    }
    const int row_off[3] = {vu ? -cols : 0, 0, vd ? cols : 0};
    const float row_w[3] = {vu ? 1.f : 0.f, 1.f, vd ? 1.f : 0.f};
    const int col_idx[3] = {cl, cc, cr};
    const float col_w[3] = {vl ? 1.f : 0.f, 1.f, vr ? 1.f : 0.f};
    const int row0 = base + r * cols;
    float conv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int di = 0; di < 3; ++di) {
#pragma unroll
        for (int dj = 0; dj < 3; ++dj) {
            const float w = P.xt_w[di * 3 + dj] * (row_w[di] * col_w[dj]);
            const int nb = row0 + row_off[di] + col_idx[dj];
#pragma unroll
            for (int c = 0; c < 6; ++c) conv[c] = fmaf(w, hx[c][nb], conv[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] = (1.0f - P.chi) * z[c] + P.chi * conv[c];
}

// Noisy force/torque of an active taxel from its crosstalk output z: drift
// and white noise, quantisation, dead override (Eqs. 25, 28).  dr holds the
// drift state on entry and the new drift on return.  Pure.
__device__ __forceinline__ void noisy_core(const ParamsDev& P, uint64_t gid, uint32_t ep, uint32_t step, uint8_t bits,
                                           float* z, float* dr) {
    const NoiseDev& G = P.ft;
    if (G.sigma_rw != 0.0f || G.sigma_white != 0.0f) {
        float nrm[12];
        uint4 wa = draw_rk(P.rk, gid, step, TAG_FT_A);
        uint4 wb = draw_rk(P.rk, gid, step, TAG_FT_B);
        float2 p0 = box_muller(wa.x, wa.y), p1 = box_muller(wa.z, wa.w);
        float2 p2 = box_muller(wb.x, wb.y);
        nrm[0] = p0.x; nrm[1] = p0.y; nrm[2] = p1.x; nrm[3] = p1.y; nrm[4] = p2.x; nrm[5] = p2.y;
        if (G.sigma_white != 0.0f) {
            uint4 wc = draw_rk(P.rk, gid, step, TAG_FT_C);
            float2 p3 = box_muller(wb.z, wb.w), p4 = box_muller(wc.x, wc.y), p5 = box_muller(wc.z, wc.w);
            nrm[6] = p3.x; nrm[7] = p3.y; nrm[8] = p4.x; nrm[9] = p4.y; nrm[10] = p5.x; nrm[11] = p5.y;
        } else {
#pragma unroll
            for (int c = 6; c < 12; ++c) nrm[c] = 0.0f;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float d = 0.0f;
            if (G.sigma_rw != 0.0f) {
                d = dr[c] + G.sigma_rw * nrm[c];
                dr[c] = d;
            }
            z[c] = z[c] + G.bias + G.sigma_white * nrm[6 + c] + d;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) z[c] += G.bias;
    }
    if (G.quant > 0.0f) {
#pragma unroll
        for (int c = 0; c < 6; ++c) z[c] = G.quant * rintf(z[c] / G.quant);
    }
    if (bits & BIT_DEAD) {
        const float stuck = stuck_value(P, G, gid, ep, 1);
#pragma unroll
        for (int c = 0; c < 6; ++c) z[c] = stuck;
    }
}

// the force/torque drift state of taxel g (zeros when the drift is off)
__device__ __forceinline__ void noisy_drift_load(const StepArgs& a, tidx g, float* dr) {
    const int64_t T = a.n_taxels;
#pragma unroll
    for (int c = 0; c < 6; ++c) dr[c] = drift_ft_on(a.P) ? __ldcs(a.drift + (1 + c) * T + g) : 0.0f;
}

// noisy_ft of an active taxel from its drift state already loaded
template <class Smem, class Out>
__device__ __forceinline__ void noisy_ft_apply(const StepArgs& a, const Smem& S, Out out, int i, tidx g,
                                               uint32_t ep, uint32_t step, uint8_t bits, int base, int r, int cc,
                                               int rows, int cols, bool wrap, float* dr) {
    const ParamsDev& P = a.P;
    const int64_t T = a.n_taxels;
    float z[6];
    crosstalk(P, S.hx, i, base, r, cc, rows, cols, wrap, z);
    noisy_core(P, (uint64_t)(a.gid0 + g), ep, step, bits, z, dr);
    if (drift_ft_on(P)) {
#pragma unroll
        for (int c = 0; c < 6; ++c) __stcs(a.drift + (1 + c) * T + g, dr[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        __stcs(a.ft_noisy + c * T + g, z[c]);
        out[c][i] = z[c];
    }
}

// Noisy force/torque of taxel i at lattice (r, cc) of a rows x cols lattice
// whose first taxel is `base` in the hx arrays; writes ft_noisy and out[.][i].
template <class Smem, class Out>
__device__ __forceinline__ void noisy_ft(const StepArgs& a, const Smem& S, Out out, int i, tidx g, uint32_t ep,
                                         uint32_t step, uint8_t bits, int base, int r, int cc, int rows, int cols,
                                         bool wrap) {
    const int64_t T = a.n_taxels;
    if (!(bits & BIT_ACTIVE)) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            __stcs(a.ft_noisy + c * T + g, 0.f);
            out[c][i] = 0.f;
        }
        return;
    }
    float dr[6];
    noisy_drift_load(a, g, dr);
    noisy_ft_apply(a, S, out, i, g, ep, step, bits, base, r, cc, rows, cols, wrap, dr);
}

// One per-link quantity, summed over taxels [s0, s1) with compensated
// accumulation (link_sum, or link_sum_halves for the noisy force/torque:
// deterministic).  Quantities: 0-5 clean
// force/torque (out cols 0-5), 6-8 clean agg_force in ZYX order (cols 12-14,
// scaled 1e4), 9-11 noisy agg_force (cols 15-17), 12 clean count, 13 noisy
// count, 14-19 noisy force/torque (cols 6-11, read from `noisy`).
template <class Smem, class Noisy>
__device__ __forceinline__ void link_quantity(const StepArgs& a, const Smem& S, Noisy noisy, size_t rec, int s0, int s1,
                                              int qn) {
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
        sum = link_sum_halves(noisy[qn - 14], s0, s1);
    } else {
        // agg_force terms d n (clean or noisy depth), each a single rounded product
        const bool nz = qn >= 9;
        const int axis = nz ? 2 - (qn - 9) : 2 - (qn - 6);  // ZYX
        const float* d = S.dn[nz ? 1 : 0];
        const float* nv = S.dn[2 + axis];
        col = nz ? 15 + (qn - 9) : 12 + (qn - 6);
        scale = 1e4f;
        sum = link_sum_prod(d, nv, s0, s1);
    }
    a.link_out[rec * kLinkOut + col] = scale * sum;
}

}  // namespace tg
