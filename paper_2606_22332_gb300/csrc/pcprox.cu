// pcprox.cu -- the point-cloud ProximityTaxel (Appendix A "ProximityTaxel"):
// the env's object is tracked by surface points p_i (object frame, sorted
// into a uniform grid of cell size R/2 at upload); taxel j at q_j with normal
// a_j collects, from every point within its sensing sphere of radius R,
// P_ij = R - |p_i - q_j|, the point's velocity relative to the taxel's with
// the component along a_j removed (v_t), and reports in its link frame
//   f = k rho sum P a + ks rho sum P v_t,   tau = k rho sum P (p - q) x a,
// rho = density / max(N, 1), N the object's point count.
// One CTA per work item; a warp takes 32 consecutive taxels at a time.  Each
// lane sets one of them up (its object-frame centre and the box of cells its
// sphere reaches) in shared memory; the warp then serves the 32 in turn, its
// lanes sharing each taxel's work: a lane takes one row of cells of the box
// (a row the sphere misses, or whose x range within the sphere is empty,
// holds no points), a warp scan of the rows' point counts flattens the
// candidates, and the lanes take them 32 at a time: the rows that start in a
// window of 32 candidates form a bit mask (one warp OR), and a lane's row is
// the count of rows started before the window plus the mask's bits up to its
// own, so that a warp's loads are consecutive points and its lanes stay busy
// however unevenly the points fall.  A warp reduction gives the sums,
// and each lane turns its own taxel's sums into force and torque.
// Every term is linear in the point's link-frame offset d: with
// S0 = sum P and S1 = sum P d, the relative velocity of a point at x + d,
// V + W_C x (x + d - p_LC) - W_L x x, sums to S0 (V + W_C x (x - p_LC) -
// W_L x x) + W_C x S1, its tangential part follows by removing the normal
// component of that sum, and the torque is k rho S1 x a.  So a point costs
// its distance and four FMAs in the object frame: with the link record's
// M = R_C^T R_L / s and t (object frame scaled by 1/s), the link-frame
// offset is d = s^2 M^T (p^ - q^) and |d| = s |p^ - q^|, and S1 is
// s^2 M^T times the object-frame sum.
#include <climits>

#include "step_common.cuh"

namespace tg {

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

template <int NT>  // threads per CTA (128, 256 or 512: a launch shape the autotuner picks)
__global__ void __launch_bounds__(NT, 1024 / NT) pc_prox_kernel(const StepArgs a) {
    constexpr int kPcWarps = NT / 32;
    __shared__ float rec_s[kPcItemLinks][kLinkRec];
    __shared__ int start_s[kPcItemLinks + 1];
    __shared__ ObjDev obj_s;
    // per warp, the non-empty rows of cells in order: first candidate in the
    // flattened order and the offset from a candidate's flattened index to
    // its point index
    __shared__ int row_first_s[kPcWarps][32];
    __shared__ int row_base_s[kPcWarps][32];
    // per warp, the 32 taxels of its batch: object-frame centre and scale
    // (scale 0: no points to visit), the cell box, and the sums
    __shared__ float4 tq_s[kPcWarps][32];
    __shared__ int tc_s[kPcWarps][6][32];
    __shared__ float4 sum_s[kPcWarps][32];
    const Item it = a.items_sorted ? a.items_sorted[blockIdx.x] : a.items[blockIdx.x];
    const int e = it.env, L = a.max_links, lb = it.link_begin, nl = it.link_end - it.link_begin, n = it.n_taxels;
    const ParamsDev& P = a.P;
    for (int i = threadIdx.x; i < nl * kLinkRec; i += NT)
        rec_s[i / kLinkRec][i % kLinkRec] = a.link_rec[(size_t)(e * L + lb + i / kLinkRec) * kLinkRec + i % kLinkRec];
    if ((int)threadIdx.x <= nl) {
        const int base = a.lattice[e * L + lb].env_offset;
        start_s[threadIdx.x] = (int)threadIdx.x < nl ? a.lattice[e * L + lb + threadIdx.x].env_offset - base : n;
    }
    if (threadIdx.x == 0) obj_s = a.objects[min(max(a.items_sorted ? it.pad : a.obj_id[e], 0), a.n_objects - 1)];
    __syncthreads();
    const int64_t T = a.n_taxels;
    const float R = P.pc_radius;
    const float rho = P.pc_density / (float)max(obj_s.pc_n, 1);
    const float kr = P.pc_k * rho, ksr = P.pc_ks * rho;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* row_first = row_first_s[warp];
    int* row_base = row_base_s[warp];
    const unsigned lanes_upto = (2u << lane) - 1u;  // bits 0..lane
    for (int b = warp * 32; b < n; b += NT) {
        // this lane's taxel of the batch: set-up
        {
            const int i = b + lane;
            float4 tq = make_float4(0.f, 0.f, 0.f, 0.f);
            int c0[3] = {0, 0, 0}, c1[3] = {-1, -1, -1};
            if (i < n && a.R[it.taxel_begin + i] > 0.0f && obj_s.pc_pts) {
                const int64_t g = it.taxel_begin + i;
                const float* rec = rec_s[pc_link_of(start_s, nl, i)];
                const float3 x = f3(a.x[g], a.y[g], a.z[g]);
                tq = make_float4(fmaf(rec[0], x.x, fmaf(rec[1], x.y, fmaf(rec[2], x.z, rec[18]))),
                                 fmaf(rec[3], x.x, fmaf(rec[4], x.y, fmaf(rec[5], x.z, rec[19]))),
                                 fmaf(rec[6], x.x, fmaf(rec[7], x.y, fmaf(rec[8], x.z, rec[20]))), rec[38]);
                const float rh = R / tq.w;  // the sphere in object-frame units
                const float q[3] = {tq.x, tq.y, tq.z};
                bool empty = false;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const float lo = (q[ax] - rh - obj_s.pc_lo[ax]) * obj_s.pc_inv_h;
                    const float hi = (q[ax] + rh - obj_s.pc_lo[ax]) * obj_s.pc_inv_h;
                    if (hi < 0.0f || lo >= (float)obj_s.pc_dims[ax]) empty = true;  // the sphere misses the box
                    c0[ax] = max((int)floorf(lo), 0);
                    c1[ax] = min((int)floorf(hi), obj_s.pc_dims[ax] - 1);
                }
                if (empty) tq.w = 0.0f;
            }
            tq_s[warp][lane] = tq;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                tc_s[warp][ax][lane] = c0[ax];
                tc_s[warp][3 + ax][lane] = c1[ax];
            }
            __syncwarp();
        }
        const int nb = min(32, n - b);
        for (int t = 0; t < nb; ++t) {  // warp-uniform
            const float4 tq = tq_s[warp][t];
            float s0 = 0.f, s1[3] = {0.f, 0.f, 0.f};  // sum P, object-frame sum P (p^ - q^)
            if (tq.w > 0.0f) {
                const float q[3] = {tq.x, tq.y, tq.z};
                const float s = tq.w, rh = R / s, rh2 = rh * rh;
                const int c0[3] = {tc_s[warp][0][t], tc_s[warp][1][t], tc_s[warp][2][t]};
                const int c1[3] = {tc_s[warp][3][t], tc_s[warp][4][t], tc_s[warp][5][t]};
                // one point's contribution: P = R - s |p^ - q^|, 0 outside the sphere
                auto add = [&](const float4 p) {
                    const float dx = p.x - q[0], dy = p.y - q[1], dz = p.z - q[2];
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float dist = d2 * rsqrtf(fmaxf(d2, 1e-30f));
                    const float Pw = fmaxf(fmaf(-s, dist, R), 0.0f);
                    s0 += Pw;
                    s1[0] = fmaf(Pw, dx, s1[0]);
                    s1[1] = fmaf(Pw, dy, s1[1]);
                    s1[2] = fmaf(Pw, dz, s1[2]);
                };
                const float h = 1.0f / obj_s.pc_inv_h;
                const int ny = c1[1] - c0[1] + 1, nrows = ny * (c1[2] - c0[2] + 1);
                const float inv_ny = 1.0f / (float)ny;
                for (int rb = 0; rb < nrows; rb += 32) {
                    // this lane's row of cells: its first point and point count
                    int p0 = 0, cnt = 0;
                    const int rr = rb + lane;
                    if (rr < nrows) {
                        // rr / ny: (rr + 1/2) / ny is at least 1/(2 ny) from an integer
                        const int qz = (int)(((float)rr + 0.5f) * inv_ny);
                        const int cz = c0[2] + qz, cy = c0[1] + (rr - qz * ny);
                        // distances from q to the slabs of the row's cells (0 inside)
                        const float z0 = obj_s.pc_lo[2] + cz * h, y0 = obj_s.pc_lo[1] + cy * h;
                        const float dzs = fmaxf(fmaxf(z0 - q[2], q[2] - (z0 + h)), 0.0f);
                        const float dys = fmaxf(fmaxf(y0 - q[1], q[1] - (y0 + h)), 0.0f);
                        // the sphere's x extent within this row
                        const float w2 = rh2 - dys * dys - dzs * dzs;
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
                        const int v = __shfl_up_sync(kFull, inc, d);
                        if (lane >= d) inc += v;
                    }
                    const int total = __shfl_sync(kFull, inc, 31);
                    // the non-empty rows, compacted in order: lane c holds the c-th one's first
                    // candidate (first) and candidate-to-point offset (base)
                    const unsigned ne = __ballot_sync(kFull, cnt > 0);
                    const int nrow = __popc(ne);
                    __syncwarp();  // the previous chunk's readers are done with the table
                    if (cnt > 0) {
                        const int c = __popc(ne & (lanes_upto >> 1));
                        row_first[c] = inc - cnt;
                        row_base[c] = p0 - (inc - cnt);
                    }
                    __syncwarp();
                    const int first = lane < nrow ? row_first[lane] : INT_MAX;
                    const int base = lane < nrow ? row_base[lane] : 0;
                    // the point index of this lane's candidate in the window at k0
                    auto point_of = [&](int k0) {
                        // rows starting in the window, and rows started before it
                        const int pos = first - k0;
                        const unsigned wm = __reduce_or_sync(kFull, (pos >= 0 && pos < 32) ? 1u << pos : 0u);
                        const int before = __popc(__ballot_sync(kFull, first < k0));
                        const int row = before + __popc(wm & lanes_upto) - 1;  // >= 0: candidate k0 has a row
                        return __shfl_sync(kFull, base, row) + k0 + lane;
                    };
                    // two windows per pass: both loads in flight before either point's arithmetic
                    for (int k0 = 0; k0 < total; k0 += 64) {
                        const int ia = point_of(k0), ib = point_of(k0 + 32);
                        const bool ha = k0 + lane < total, hb = k0 + 32 + lane < total;
                        float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
                        if (ha) pa = __ldg(obj_s.pc_pts + ia);
                        if (hb) pb = __ldg(obj_s.pc_pts + ib);
                        if (ha) add(pa);
                        if (hb) add(pb);
                    }
                }
            }
            // the warp's sums, kept for the taxel's lane
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(kFull, s0, o);
#pragma unroll
                for (int c = 0; c < 3; ++c) s1[c] += __shfl_xor_sync(kFull, s1[c], o);
            }
            if (lane == t) sum_s[warp][t] = make_float4(s0, s1[0], s1[1], s1[2]);
        }
        __syncwarp();
        // this lane's taxel: link frame S1 = s^2 M^T (object-frame sum), sum P v_r, its
        // tangential part, force and torque (coalesced over the batch)
        const int i = b + lane;
        if (i < n) {
            const int64_t g = it.taxel_begin + i;
            float3 fo = f3(0.f, 0.f, 0.f), to = f3(0.f, 0.f, 0.f);
            const float4 sm = sum_s[warp][lane];
            if (tq_s[warp][lane].w > 0.0f) {
                const float* rec = rec_s[pc_link_of(start_s, nl, i)];
                const float3 x = f3(a.x[g], a.y[g], a.z[g]), nn = f3(a.nx[g], a.ny[g], a.nz[g]);
                const float s2 = rec[38] * rec[38];
                const float3 S1 = f3(s2 * (rec[0] * sm.y + rec[3] * sm.z + rec[6] * sm.w),
                                     s2 * (rec[1] * sm.y + rec[4] * sm.z + rec[7] * sm.w),
                                     s2 * (rec[2] * sm.y + rec[5] * sm.z + rec[8] * sm.w));
                const float3 V = f3(rec[24], rec[25], rec[26]), Wc = f3(rec[27], rec[28], rec[29]);
                const float3 Wl = f3(rec[30], rec[31], rec[32]), pLC = f3(rec[33], rec[34], rec[35]);
                const float3 svr = (V + cross(Wc, x - pLC) - cross(Wl, x)) * sm.x + cross(Wc, S1);
                const float3 svt = svr - nn * dot(svr, nn);
                fo = nn * (kr * sm.x) + svt * ksr;
                to = cross(S1, nn) * kr;
            }
            a.pc_ft[g] = fo.x;
            a.pc_ft[T + g] = fo.y;
            a.pc_ft[2 * T + g] = fo.z;
            a.pc_ft[3 * T + g] = to.x;
            a.pc_ft[4 * T + g] = to.y;
            a.pc_ft[5 * T + g] = to.z;
        }
        __syncwarp();  // the batch tables are rewritten by the next batch
    }
}

cudaError_t launch_pc_prox(const StepArgs& a, int n_items, int threads, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    switch (threads) {
    case 128: pc_prox_kernel<128><<<n_items, 128, 0, s>>>(a); break;
    case 256: pc_prox_kernel<256><<<n_items, 256, 0, s>>>(a); break;
    case 512: pc_prox_kernel<512><<<n_items, 512, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tg
