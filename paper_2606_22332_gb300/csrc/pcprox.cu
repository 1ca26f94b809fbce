// pcprox.cu -- the point-cloud ProximityTaxel (Appendix A "ProximityTaxel"):
// the env's object is tracked by surface points p_i (object frame, sorted
// into a uniform grid of cell size R/2 at upload); taxel j at q_j with normal
// a_j collects, from every point within its sensing sphere of radius R,
// P_ij = R - |p_i - q_j|, the point's velocity relative to the taxel's with
// the component along a_j removed (v_t), and reports in its link frame
//   f = k rho sum P a + ks rho sum P v_t,   tau = k rho sum P (p - q) x a,
// rho = density / max(N, 1), N the object's point count.
// One CTA per work item, one warp per taxel.  The lanes share the taxel's
// work: each takes one row of cells its sphere reaches (a row it misses, or
// whose x range within the sphere is empty, holds no points), a warp scan of
// the rows' point counts flattens the candidates, and the lanes stride over
// them 64 at a time (each finds its row by a binary search over the lanes),
// so that a warp's loads are consecutive points and its lanes stay busy
// however unevenly the points fall.  A warp reduction gives the sums.
// Everything is evaluated in the link frame: with the link record's
// M = R_C^T R_L / s and t (object frame scaled by 1/s), the link-frame offset
// of a point is s^2 M^T (p^ - q^), and the relative velocity of a point at
// link position x + d is V + W_C x (x + d - p_LC) - W_L x x.
#include "step_common.cuh"

namespace tg {

constexpr int kPcThreads = 256;
constexpr int kPcWarps = kPcThreads / 32;
constexpr int kPcItemLinks = 32;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int pc_link_of(const int* start, int nl, int i) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the lane whose row holds flattened candidate k: the last lane with
// excl <= k (excl, the rows' exclusive prefix, does not decrease over lanes)
__device__ __forceinline__ int pc_row_lane(int excl, int k) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int e = __shfl_sync(kFull, excl, lo + step);
        if (e <= k) lo += step;
    }
    return lo;
}

__global__ void __launch_bounds__(kPcThreads) pc_prox_kernel(const StepArgs a) {
    __shared__ float rec_s[kPcItemLinks][kLinkRec];
    __shared__ int start_s[kPcItemLinks + 1];
    __shared__ ObjDev obj_s;
    const Item it = a.items_sorted ? a.items_sorted[blockIdx.x] : a.items[blockIdx.x];
    const int e = it.env, L = a.max_links, lb = it.link_begin, nl = it.link_end - it.link_begin, n = it.n_taxels;
    const ParamsDev& P = a.P;
    for (int i = threadIdx.x; i < nl * kLinkRec; i += kPcThreads)
        rec_s[i / kLinkRec][i % kLinkRec] = a.link_rec[(size_t)(e * L + lb + i / kLinkRec) * kLinkRec + i % kLinkRec];
    if ((int)threadIdx.x <= nl) {
        const int base = a.lattice[e * L + lb].env_offset;
        start_s[threadIdx.x] = (int)threadIdx.x < nl ? a.lattice[e * L + lb + threadIdx.x].env_offset - base : n;
    }
    if (threadIdx.x == 0) obj_s = a.objects[min(max(a.obj_id[e], 0), a.n_objects - 1)];
    __syncthreads();
    const int64_t T = a.n_taxels;
    const float R = P.pc_radius;
    const float rho = P.pc_density / (float)max(obj_s.pc_n, 1);
    const float kr = P.pc_k * rho, ksr = P.pc_ks * rho;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < n; i += kPcWarps) {  // one warp per taxel (warp-uniform)
        const int64_t g = it.taxel_begin + i;
        float sp = 0.f, sv[3] = {0.f, 0.f, 0.f}, st[3] = {0.f, 0.f, 0.f};
        float3 nn = f3(0.f, 0.f, 0.f);
        if (a.R[g] > 0.0f && obj_s.pc_pts) {
            const float* rec = rec_s[pc_link_of(start_s, nl, i)];
            const float3 x = f3(a.x[g], a.y[g], a.z[g]);
            nn = f3(a.nx[g], a.ny[g], a.nz[g]);
            const float q[3] = {fmaf(rec[0], x.x, fmaf(rec[1], x.y, fmaf(rec[2], x.z, rec[18]))),
                                fmaf(rec[3], x.x, fmaf(rec[4], x.y, fmaf(rec[5], x.z, rec[19]))),
                                fmaf(rec[6], x.x, fmaf(rec[7], x.y, fmaf(rec[8], x.z, rec[20])))};
            const float s = rec[38], s2 = s * s;
            const float rh = R / s;  // the sphere in object-frame units
            const float3 V = f3(rec[24], rec[25], rec[26]), Wc = f3(rec[27], rec[28], rec[29]);
            const float3 Wl = f3(rec[30], rec[31], rec[32]), pLC = f3(rec[33], rec[34], rec[35]);
            const float3 vtax = cross(Wl, x);
            int c0[3], c1[3];
            bool empty = false;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const float lo = (q[ax] - rh - obj_s.pc_lo[ax]) * obj_s.pc_inv_h;
                const float hi = (q[ax] + rh - obj_s.pc_lo[ax]) * obj_s.pc_inv_h;
                if (hi < 0.0f || lo >= (float)obj_s.pc_dims[ax]) empty = true;  // the sphere misses the box
                c0[ax] = max((int)floorf(lo), 0);
                c1[ax] = min((int)floorf(hi), obj_s.pc_dims[ax] - 1);
            }
            // one point's contribution, if it lies in the sphere
            auto add = [&](const float4 p) {
                const float dx = p.x - q[0], dy = p.y - q[1], dz = p.z - q[2];
                if (!(dx * dx + dy * dy + dz * dz < rh * rh)) return;
                // link-frame offset s^2 M^T (p^ - q^)
                const float3 d = f3(s2 * (rec[0] * dx + rec[3] * dy + rec[6] * dz),
                                    s2 * (rec[1] * dx + rec[4] * dy + rec[7] * dz),
                                    s2 * (rec[2] * dx + rec[5] * dy + rec[8] * dz));
                const float dist = sqrtf(dot(d, d));
                if (!(dist < R)) return;
                const float Pw = R - dist;
                const float3 vr = V + cross(Wc, x + d - pLC) - vtax;
                const float3 vt = vr - nn * dot(vr, nn);
                const float3 tq = cross(d, nn);
                sp += Pw;
                sv[0] = fmaf(Pw, vt.x, sv[0]); sv[1] = fmaf(Pw, vt.y, sv[1]); sv[2] = fmaf(Pw, vt.z, sv[2]);
                st[0] = fmaf(Pw, tq.x, st[0]); st[1] = fmaf(Pw, tq.y, st[1]); st[2] = fmaf(Pw, tq.z, st[2]);
            };
            if (!empty) {
                const float h = 1.0f / obj_s.pc_inv_h;
                const int ny = c1[1] - c0[1] + 1, nrows = ny * (c1[2] - c0[2] + 1);
                for (int rb = 0; rb < nrows; rb += 32) {
                    // this lane's row of cells: its first point and point count
                    int p0 = 0, cnt = 0;
                    const int rr = rb + lane;
                    if (rr < nrows) {
                        const int cz = c0[2] + rr / ny, cy = c0[1] + rr % ny;
                        // distances from q to the slabs of the row's cells (0 inside)
                        const float z0 = obj_s.pc_lo[2] + cz * h, y0 = obj_s.pc_lo[1] + cy * h;
                        const float dzs = fmaxf(fmaxf(z0 - q[2], q[2] - (z0 + h)), 0.0f);
                        const float dys = fmaxf(fmaxf(y0 - q[1], q[1] - (y0 + h)), 0.0f);
                        // the sphere's x extent within this row
                        const float w2 = rh * rh - dys * dys - dzs * dzs;
                        if (w2 > 0.0f) {
                            const float w = sqrtf(w2) * 1.0001f;
                            const int x0 = max((int)floorf((q[0] - w - obj_s.pc_lo[0]) * obj_s.pc_inv_h), c0[0]);
                            const int x1 = min((int)floorf((q[0] + w - obj_s.pc_lo[0]) * obj_s.pc_inv_h), c1[0]);
                            if (x1 >= x0) {
                                const int row = (cz * obj_s.pc_dims[1] + cy) * obj_s.pc_dims[0];
                                p0 = __ldg(obj_s.pc_start + row + x0);
                                cnt = __ldg(obj_s.pc_start + row + x1 + 1) - p0;
                            }
                        }
                    }
                    // flatten the rows' candidates (inclusive warp scan of the counts)
                    int inc = cnt;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int t = __shfl_up_sync(kFull, inc, d);
                        if (lane >= d) inc += t;
                    }
                    const int total = __shfl_sync(kFull, inc, 31), excl = inc - cnt;
                    for (int k0 = 0; k0 < total; k0 += 64) {
                        const int ka = k0 + lane, kb = ka + 32;
                        const int la = pc_row_lane(excl, ka), lb2 = pc_row_lane(excl, kb);
                        const int ia = __shfl_sync(kFull, p0, la) + ka - __shfl_sync(kFull, excl, la);
                        const int ib = __shfl_sync(kFull, p0, lb2) + kb - __shfl_sync(kFull, excl, lb2);
                        float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
                        if (ka < total) pa = __ldg(obj_s.pc_pts + ia);
                        if (kb < total) pb = __ldg(obj_s.pc_pts + ib);
                        if (ka < total) add(pa);
                        if (kb < total) add(pb);
                    }
                }
            }
        }
        // the warp's sums
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sp += __shfl_xor_sync(kFull, sp, o);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sv[c] += __shfl_xor_sync(kFull, sv[c], o);
                st[c] += __shfl_xor_sync(kFull, st[c], o);
            }
        }
        if (lane < 6) {
            float v = kr * st[2];
            if (lane == 0) v = kr * sp * nn.x + ksr * sv[0];
            else if (lane == 1) v = kr * sp * nn.y + ksr * sv[1];
            else if (lane == 2) v = kr * sp * nn.z + ksr * sv[2];
            else if (lane == 3) v = kr * st[0];
            else if (lane == 4) v = kr * st[1];
            a.pc_ft[(int64_t)lane * T + g] = v;
        }
    }
}

cudaError_t launch_pc_prox(const StepArgs& a, int n_items, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    pc_prox_kernel<<<n_items, kPcThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tg
