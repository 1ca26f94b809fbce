// prox.cu -- geometry-aware proximity by rays (the ProximityTaxel reading in
// its ray form) and its noise chain.
//
// From each active probe centre, rays leave along the probe normal and on a
// cone around it; each ray is sphere-traced through the object's signed
// distance (step max(phi, 10 um), at most 192 samples).  When a sample falls
// inside, the crossing is bracketed by it and the last outside sample and
// refined by the Illinois variant of regula falsi, so the reported distance
// is the first surface crossing along the ray.  The reading is the mean over
// rays of hit (1 - t / range).  Noise (Eqs. 25-30): gain, hysteresis, bias,
// white noise and drift, quantisation, dead override.
// One CTA per work item, items in the object-sorted order of the step.
#include "step_common.cuh"

namespace tg {

constexpr int kProxItemLinks = 32;
constexpr float kMinStep = 1e-5f;
constexpr int kMaxMarch = 192;

// signed distance in world units along the ray q0 + t d (object frame, d
// already scaled by 1/s)
__device__ __forceinline__ float ray_field(const ObjDev& obj, float3 q0, float3 d, float t, float scale) {
    return scale * sdf_phi_fast(obj, q0 + d * t);
}

// The part [t0, t1] of [0, range] where the ray q0 + t d is inside a grid
// object's box (a grid has no surface outside it: the first crossing is
// searched in the box only); false when the ray misses the box within range.
// Other object kinds: [0, range].
__device__ __forceinline__ bool ray_box(const ObjDev& o, float3 q0, float3 d, float range, float* t0, float* t1) {
    float ta = 0.0f, tb = range;
    if (o.kind == TG_OBJ_GRID || o.kind == TG_OBJ_NEURAL) {
        const float q[3] = {q0.x, q0.y, q0.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (dd[a] == 0.0f) {
                if (q[a] < o.lo[a] || q[a] > o.hi[a]) return false;
            } else {
                float u = (o.lo[a] - q[a]) / dd[a], v = (o.hi[a] - q[a]) / dd[a];
                if (u > v) { const float w = u; u = v; v = w; }
                ta = fmaxf(ta, u);
                tb = fminf(tb, v);
            }
        }
    }
    *t0 = ta;
    *t1 = tb;
    return ta <= tb;
}

constexpr int kRefineIters = 24;
// idle lanes refill from the pool once at least this many are idle (or the
// whole warp is): a refill is ~200 instructions executed by the refilling
// lanes only, and refilling every iteration left most lanes of each warp
// masked off through it
constexpr int kRefillBatch = 16;

// The taxel of item-relative index i: its link (last start <= i).
__device__ __forceinline__ int link_of(const int* start, int nl, int i) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The rays of one item (pool, march, refine) into t_s.  Instantiated once for
// grid objects (the field is the inlined grid interpolation) and once for
// the other kinds (dispatch per sample), so the grid loop carries no calls.
template <bool GRID>
__device__ __forceinline__ void trace_item_rays(const StepArgs& a, const Item& it, int n, int nl,
                                                const float (*rec_s)[kLinkRec], const int* start_s,
                                                const ObjDev& obj_s, unsigned int* next_ray, float* t_s) {
    const ParamsDev& P = a.P;
    const int nr = P.prox_rays;
    const unsigned total = (unsigned)(n * nr);
    const float range = P.prox_range;
    const unsigned lane = threadIdx.x & 31u;
    // one ray per lane
    int rid = -1, mode = 0, cnt = 0, side = 0;  // mode 0 idle, 1 march, 2 refine
    bool exhausted = false;
    float ta = 0.f, fa = 0.f, tb = 0.f, fb = 0.f, scale = 1.f, tend = 0.f;
    float3 q0 = f3(0.f, 0.f, 0.f), d = f3(0.f, 0.f, 0.f);
    for (;;) {
        // refill idle lanes from the pool
        const bool want = mode == 0 && !exhausted;
        const unsigned need = __ballot_sync(0xffffffffu, want);
        const unsigned busy = __ballot_sync(0xffffffffu, mode != 0);
        if (need && (__popc(need) >= kRefillBatch || busy == 0u)) {
            const int leader = __ffs(need) - 1;
            unsigned base = 0;
            if ((int)lane == leader) base = atomicAdd(next_ray, (unsigned)__popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (want) {
                const unsigned r = base + (unsigned)__popc(need & ((1u << lane) - 1u));
                if (r >= total) {
                    exhausted = true;
                } else {
                    rid = (int)r;
                    const int i = rid / nr, k = rid - i * nr;
                    const int64_t g = it.taxel_begin + i;
                    const float R = a.R[g];
                    if (!(R > 0.0f)) {
                        t_s[rid] = -1.0f;  // filler: no rays
                    } else {
                        const float* rec = rec_s[link_of(start_s, nl, i)];
                        const float x0 = a.x[g], x1 = a.y[g], x2 = a.z[g];
                        const float3 nn = f3(a.nx[g], a.ny[g], a.nz[g]);
                        q0 = f3(fmaf(rec[0], x0, fmaf(rec[1], x1, fmaf(rec[2], x2, rec[18]))),
                                fmaf(rec[3], x0, fmaf(rec[4], x1, fmaf(rec[5], x2, rec[19]))),
                                fmaf(rec[6], x0, fmaf(rec[7], x1, fmaf(rec[8], x2, rec[20]))));
                        // the fan in the link frame: n, then the cone around n
                        float3 dl = nn;
                        if (k > 0) {
                            float3 u = cross(nn, f3(0.f, 0.f, 1.f));
                            if (dot(u, u) < 1e-12f) u = cross(nn, f3(1.f, 0.f, 0.f));
                            u = normalize_or(u, f3(1.f, 0.f, 0.f));
                            const float3 v = cross(nn, u);
                            dl = nn * P.prox_cos + (u * P.prox_az_cos[k] + v * P.prox_az_sin[k]) * P.prox_sin;
                        }
                        d = f3(rec[0] * dl.x + rec[1] * dl.y + rec[2] * dl.z, rec[3] * dl.x + rec[4] * dl.y + rec[5] * dl.z,
                               rec[6] * dl.x + rec[7] * dl.y + rec[8] * dl.z);
                        scale = rec[38];
                        float t0, t1;
                        if (!ray_box(obj_s, q0, d, range, &t0, &t1)) {
                            t_s[rid] = -1.0f;  // misses the object's box within the range
                        } else {
                            ta = t0;       // the first sample is the box entry (mode 1 with cnt = -1)
                            tend = t1;
                            fa = -1.0f;
                            cnt = -1;
                            mode = 1;
                        }
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, mode != 0 || !exhausted)) break;
        // the one field evaluation of this iteration
        float tq = 0.0f;
        bool eval = false;
        if (mode == 1) {
            tq = cnt < 0 ? ta : fminf(ta + fmaxf(fa, kMinStep), tend);
            eval = true;
        } else if (mode == 2) {
            if (cnt >= kRefineIters || !(tb - ta > 1e-7f)) {
                t_s[rid] = tb;
                mode = 0;
            } else {
                tq = (fa * tb - fb * ta) / (fa - fb);
                eval = true;
            }
        }
        // the marching and refining lanes evaluate the field together
        float fq = 0.0f;
        __syncwarp();
        if (eval) {
            if constexpr (GRID) fq = scale * grid_phi_fast(obj_s, q0 + d * tq);
            else fq = ray_field(obj_s, q0, d, tq, scale);
        }
        __syncwarp();
        if (mode == 1) {
            if (cnt < 0) {                   // the probe centre, or the box entry
                if (!(fq > 0.0f)) { t_s[rid] = tq; mode = 0; }
                else { fa = fq; cnt = 0; }
            } else if (!(fq > 0.0f)) {       // crossed: refine on [ta, tq]
                tb = tq; fb = fq; mode = 2; cnt = 0; side = 0;
            } else if (tq >= tend || ++cnt >= kMaxMarch) {
                t_s[rid] = -1.0f;            // no crossing within the range
                mode = 0;
            } else {
                ta = tq; fa = fq;
            }
        } else if (mode == 2 && eval) {
            if (fq > 0.0f) {
                ta = tq; fa = fq;
                if (side == -1) fb *= 0.5f;
                side = -1;
            } else {
                tb = tq; fb = fq;
                if (side == 1) fa *= 0.5f;
                side = 1;
            }
            ++cnt;
        }
    }
}

// Lanes take rays, not taxels: every lane owns one ray at a time and takes
// the next ray of the item's pool (a warp-aggregated atomic) once its ray has
// ended and enough lanes of the warp are idle, so the warp stays full while
// rays march for very different numbers of steps.  Marching and the Illinois refinement of the first crossing are
// one state machine with exactly one field evaluation per iteration, so the
// lanes of a warp stay converged on it:
//   march:  from the entry into the object's box (a grid has no surface
//           outside it), t' = min(t + max(f, 10 um), t_end) with t_end the
//           box exit or the range; f' = f(t'); f' <= 0 -> refine on [t, t'],
//           else if t' = t_end -> miss, else continue (at most 192 samples)
//   refine: t_c = (f_a t_b - f_b t_a) / (f_a - f_b), halving the retained
//           end's value after two moves on the same side (at most 24
//           samples, or until t_b - t_a <= 1e-7 m); the crossing is t_b.
// Per-ray distances go to shared memory; each taxel then sums its rays in
// ray order (deterministic) and runs the noise chain.
template <int NT>  // threads per CTA (128, 256 or 512: a launch shape the autotuner picks)
__global__ void __launch_bounds__(NT, 1024 / NT) prox_kernel(const StepArgs a) {
    extern __shared__ float t_s[];  // [n taxels][rays]: crossing distance or -1
    __shared__ float rec_s[kProxItemLinks][kLinkRec];
    __shared__ int start_s[kProxItemLinks + 1];
    __shared__ ObjDev obj_s;
    __shared__ unsigned int next_ray;
    const Item it = a.items_sorted ? a.items_sorted[blockIdx.x] : a.items[blockIdx.x];
    const int e = it.env, L = a.max_links, lb = it.link_begin, nl = it.link_end - it.link_begin, n = it.n_taxels;
    const ParamsDev& P = a.P;
    const uint32_t step = a.step_from_ctl ? a.ctl->step : a.step;
    for (int i = threadIdx.x; i < nl * kLinkRec; i += NT)
        rec_s[i / kLinkRec][i % kLinkRec] = a.link_rec[(size_t)(e * L + lb + i / kLinkRec) * kLinkRec + i % kLinkRec];
    if ((int)threadIdx.x <= nl) {
        const int base = a.lattice[e * L + lb].env_offset;
        start_s[threadIdx.x] = (int)threadIdx.x < nl ? a.lattice[e * L + lb + threadIdx.x].env_offset - base : n;
    }
    if (threadIdx.x == 0) {
        int oid = min(max(a.items_sorted ? it.pad : a.obj_id[e], 0), a.n_objects - 1);
        obj_s = a.objects[oid];
        next_ray = 0;
    }
    __syncthreads();
    if (obj_s.kind == TG_OBJ_GRID || obj_s.kind == TG_OBJ_NEURAL)
        trace_item_rays<true>(a, it, n, nl, rec_s, start_s, obj_s, &next_ray, t_s);
    else
        trace_item_rays<false>(a, it, n, nl, rec_s, start_s, obj_s, &next_ray, t_s);
    __syncthreads();
    const int nr = P.prox_rays;
    const float range = P.prox_range;
    const uint32_t ep = a.episode[e];
    const int64_t T = a.n_taxels;
    for (int i = threadIdx.x; i < n; i += NT) {
        const int64_t g = it.taxel_begin + i;
        const float R = a.R[g];
        if (!(R > 0.0f)) {
            a.prox_clean[g] = 0.0f;
            a.prox_noisy[g] = 0.0f;
            continue;
        }
        float reading = 0.0f;
        for (int k = 0; k < nr; ++k) {
            const float t = t_s[i * nr + k];
            if (t >= 0.0f) reading += 1.0f - t / range;
        }
        reading /= (float)nr;
        a.prox_clean[g] = reading;
        // noise chain of the proximity group
        const NoiseDev& G = P.prox;
        const uint64_t gid = (uint64_t)(a.gid0 + g);
        const bool dead = a.flags[g] & 2u;
        float x = reading;
        if (G.gain_on) x *= G.gain_lo + G.gain_span * u24(draw(P.seed, gid, ep, TAG_EPISODE).w);
        if (G.beta != 0.0f) x = hyst_update(G, x, a.hyst_prev + 7 * T + g, a.hyst_xi + 7 * T + g);
        if (G.sigma_rw != 0.0f || G.sigma_white != 0.0f) {
            const uint4 w = draw(P.seed, gid, step, TAG_SCALAR);
            const float2 z = box_muller(w.z, w.w);
            float dr = 0.0f;
            if (G.sigma_rw != 0.0f) {
                dr = a.drift[7 * T + g] + G.sigma_rw * z.x;
                a.drift[7 * T + g] = dr;
            }
            x = x + G.bias + G.sigma_white * z.y + dr;
        } else {
            x += G.bias;
        }
        x = quantise(G, x);
        if (dead) x = G.stuck_lo + G.stuck_span * u24(draw(P.seed, gid, ep, TAG_STUCK).z);
        a.prox_noisy[g] = x;
    }
}

template <int NT>
cudaError_t launch_prox_nt(const StepArgs& a, int n_items, size_t smem, cudaStream_t s) {
    const cudaError_t err = raise_smem_limit((const void*)prox_kernel<NT>, smem);
    if (err != cudaSuccess) return err;
    prox_kernel<NT><<<n_items, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prox(const StepArgs& a, int n_items, int threads, cudaStream_t s) {
    if (n_items == 0 || a.P.prox_rays < 1) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)kItemCap * (size_t)a.P.prox_rays;  // <= 64 KB (16 rays)
    switch (threads) {
    case 128: return launch_prox_nt<128>(a, n_items, smem, s);
    case 256: return launch_prox_nt<256>(a, n_items, smem, s);
    case 512: return launch_prox_nt<512>(a, n_items, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Elastomer markers: h = max(0, -phi) at every marker of the pad, then the
// dilation sum of Eqs. 20-21 over the neighbourhood, with the per-offset
// weights computed on the host; with shear anchors on, the shear of Eq. 19
// is added (one chunk of 256 tracked points at a time: anchor update, the
// contributing points compacted in point order into shared memory, then every
// marker sums their Gaussian-weighted drags).
// ---------------------------------------------------------------------------
template <int NT>  // threads per CTA (128, 256 or 512: a launch shape the autotuner picks)
__global__ void __launch_bounds__(NT) marker_kernel(const MarkerArgs m) {
    __shared__ float h_s[kMaxPadMarkers];
    __shared__ float ha_s[kMaxPadMarkers];
    __shared__ float ut_s[kMaxPadMarkers];   // shear, tangent
    __shared__ float ub_s[kMaxPadMarkers];   // shear, bitangent
    __shared__ float4 con_s[NT]; // contributing points of a chunk: z_t, z_b, drag_t, drag_b
    __shared__ int warp_cnt[NT / 32];
    __shared__ int anchored_s;
    __shared__ float rec[kLinkRec];
    __shared__ ObjDev obj_s;
    const int pad = blockIdx.x;  // e * P + p
    const int e = pad / m.pads_per_env;
    const int l = m.pad_link[pad];
    const int M = m.rows * m.cols;
    const int oid = min(max(m.obj_id[e], 0), m.n_objects - 1);
    if (threadIdx.x < kLinkRec) rec[threadIdx.x] = m.link_rec[(size_t)(e * m.max_links + l) * kLinkRec + threadIdx.x];
    if (threadIdx.x == 0) {
        obj_s = m.objects[oid];
        anchored_s = 0;
    }
    __syncthreads();
    const float* fr = m.pad_frame + (size_t)pad * 9;
    const float3 o = f3(fr[0], fr[1], fr[2]), nrm = f3(fr[3], fr[4], fr[5]), tu = f3(fr[6], fr[7], fr[8]);
    const float3 tv = cross(nrm, tu);
    const float half_a = 0.5f * m.rows * m.pitch, half_b = 0.5f * m.cols * m.pitch;
    for (int j = threadIdx.x; j < M; j += NT) {
        const int r = j / m.cols, c = j - r * m.cols;
        const float sa = (r - 0.5f * (m.rows - 1)) * m.pitch, sb = (c - 0.5f * (m.cols - 1)) * m.pitch;
        const float3 x = o + tu * sa + tv * sb;
        const float phi = fast_query(rec, obj_s, x.x, x.y, x.z);
        if (!isfinite(phi)) atomicAdd(m.err, 1u);
        const float h = phi < 0.0f ? -phi : 0.0f;
        h_s[j] = h;
        ha_s[j] = h > 0.0f ? powf(h, m.alpha) : 0.0f;
        ut_s[j] = 0.0f;
        ub_s[j] = 0.0f;
    }
    if (m.shear_n > 0) {
        float2* an = m.anchors + (size_t)pad * m.shear_n;
        // anchors taken on another object (or cleared by a reset) read as none and are rewritten
        const bool fresh = m.anchor_obj[pad] != oid;
        const int N = obj_s.pc_pts ? min(obj_s.pc_n, m.shear_n) : 0;
        const float s = rec[38], s2 = s * s;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int count = 0;
        for (int c0 = 0; c0 < N; c0 += NT) {
            const int i = c0 + threadIdx.x;
            bool contrib = false;
            float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < N) {
                const float4 p = __ldg(obj_s.pc_pts + i);
                // link frame x = s^2 M^T (p^ - t), then the pad's sensor frame
                const float dx = p.x - rec[18], dy = p.y - rec[19], dz = p.z - rec[20];
                const float3 xl = f3(s2 * (rec[0] * dx + rec[3] * dy + rec[6] * dz),
                                     s2 * (rec[1] * dx + rec[4] * dy + rec[7] * dz),
                                     s2 * (rec[2] * dx + rec[5] * dy + rec[8] * dz));
                const float3 r = xl - o;
                const float za = dot(r, tu), zb = dot(r, tv), zn = dot(r, nrm);
                // SDF of the elastomer box (centre -half_t along the normal)
                const float qa = fabsf(za) - half_a, qb = fabsf(zb) - half_b, qc = fabsf(zn + m.half_t) - m.half_t;
                const float oa = fmaxf(qa, 0.f), ob = fmaxf(qb, 0.f), oc = fmaxf(qc, 0.f);
                const float sdf = sqrtf(oa * oa + ob * ob + oc * oc) + fminf(fmaxf(qa, fmaxf(qb, qc)), 0.f);
                float2 ea = fresh ? make_float2(NAN, NAN) : an[i];
                bool anchored = !isnan(ea.x);
                bool write = fresh;
                if (!anchored && sdf < -m.eta_enter) {
                    ea = make_float2(za, zb);
                    anchored = write = true;
                } else if (anchored && sdf > m.eta_exit) {
                    ea = make_float2(NAN, NAN);
                    anchored = false;
                    write = true;
                }
                if (write) an[i] = ea;
                count += anchored;
                const float h = sdf < 0.0f ? -sdf : 0.0f;
                if (anchored && h > 0.0f) {
                    contrib = true;
                    cv = make_float4(za, zb, m.s_s * (za - ea.x) * h, m.s_s * (zb - ea.y) * h);
                }
            }
            // compaction in point order
            const unsigned bal = __ballot_sync(0xffffffffu, contrib);
            if (lane == 0) warp_cnt[warp] = __popc(bal);
            __syncthreads();
            int off = 0, K = 0;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
                off += w < warp ? warp_cnt[w] : 0;
                K += warp_cnt[w];
            }
            if (contrib) con_s[off + __popc(bal & ((1u << lane) - 1u))] = cv;
            __syncthreads();
            if (K > 0) {
                for (int j = threadIdx.x; j < M; j += NT) {
                    const int r = j / m.cols, c = j - r * m.cols;
                    const float sa = (r - 0.5f * (m.rows - 1)) * m.pitch, sb = (c - 0.5f * (m.cols - 1)) * m.pitch;
                    float ut = ut_s[j], ub = ub_s[j];
                    for (int k = 0; k < K; ++k) {
                        const float4 q = con_s[k];
                        const float da = sa - q.x, db = sb - q.y;
                        const float g = expf(-m.lambda_s * (da * da + db * db));
                        ut = fmaf(q.z, g, ut);
                        ub = fmaf(q.w, g, ub);
                    }
                    ut_s[j] = ut;
                    ub_s[j] = ub;
                }
            }
            __syncthreads();  // con_s and warp_cnt are reused by the next chunk
        }
        count = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && count) atomicAdd(&anchored_s, count);
    }
    __syncthreads();
    if (m.shear_n > 0 && threadIdx.x == 0) {
        m.n_anchored[pad] = anchored_s;
        m.anchor_obj[pad] = oid;
    }
    const int W = 2 * m.radius + 1;
    for (int j = threadIdx.x; j < M; j += NT) {
        const int r = j / m.cols, c = j - r * m.cols;
        float un = 0.f, ut = 0.f, uv = 0.f;
        for (int di = -m.radius; di <= m.radius; ++di) {
            const int ri = r + di;
            if (ri < 0 || ri >= m.rows) continue;
            for (int dj = -m.radius; dj <= m.radius; ++dj) {
                const int ci = c + dj;
                if (ci < 0 || ci >= m.cols) continue;
                const int i = ri * m.cols + ci;
                const float h = h_s[i];
                if (h == 0.0f) continue;
                const int w = (di + m.radius) * W + (dj + m.radius);
                // r_ij = x_j - x_i = -(di, dj) pitch in (tangent, bitangent)
                const float ht = h * m.w_tan[w];
                ut = fmaf(-di * m.pitch, ht, ut);
                uv = fmaf(-dj * m.pitch, ht, uv);
                un = fmaf(ha_s[i], m.w_norm[w], un);
            }
        }
        float* out = m.u + ((size_t)pad * M + j) * 3;
        out[0] = un;
        out[1] = ut + ut_s[j];
        out[2] = uv + ub_s[j];
    }
}

cudaError_t launch_markers(const MarkerArgs& m, int threads, cudaStream_t s) {
    const int n = m.n_envs * m.pads_per_env;
    if (n == 0) return cudaSuccess;
    switch (threads) {
    case 128: marker_kernel<128><<<n, 128, 0, s>>>(m); break;
    case 256: marker_kernel<256><<<n, 256, 0, s>>>(m); break;
    case 512: marker_kernel<512><<<n, 512, 0, s>>>(m); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

__global__ void shear_reset_kernel(int32_t* anchor_obj, int n_pads, int pads_per_env, const uint8_t* mask) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pads && (!mask || mask[i / pads_per_env])) anchor_obj[i] = -1;
}

cudaError_t launch_shear_reset(int32_t* anchor_obj, int n_envs, int pads_per_env, const uint8_t* mask,
                               cudaStream_t s) {
    const int n = n_envs * pads_per_env;
    if (n == 0) return cudaSuccess;
    shear_reset_kernel<<<(n + 255) / 256, 256, 0, s>>>(anchor_obj, n, pads_per_env, mask);
    return cudaGetLastError();
}

}  // namespace tg
