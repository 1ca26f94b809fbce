// pcprox.cu -- the point-cloud ProximityTaxel (Appendix A "ProximityTaxel"):
// the env's object is tracked by surface points p_i (object frame, sorted
// into a uniform grid of cell size R/2 at upload); taxel j at q_j with normal
// a_j collects, from every point within its sensing sphere of radius R,
// P_ij = R - |p_i - q_j|, the point's velocity relative to the taxel's with
// the component along a_j removed (v_t), and reports in its link frame
//   f = k rho sum P a + ks rho sum P v_t,   tau = k rho sum P (p - q) x a,
// rho = density / max(N, 1), N the object's point count.
// One CTA per work item, one thread per taxel; a taxel visits, row by row of
// cells, the x range of cells its sphere reaches in that row (rows it misses
// are skipped), four points' loads in flight at a time.  Everything is evaluated in the link frame: with the
// link record's M = R_C^T R_L / s and t (object frame scaled by 1/s), the
// link-frame offset of a point is s^2 M^T (p^ - q^), and the relative
// velocity of a point at link position x + d is V + W_C x (x + d - p_LC) -
// W_L x x.
#include "step_common.cuh"

namespace tg {

constexpr int kPcThreads = 256;
constexpr int kPcItemLinks = 32;

__device__ __forceinline__ int pc_link_of(const int* start, int nl, int i) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= i) lo = mid;
        else hi = mid - 1;
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
    for (int i = threadIdx.x; i < n; i += kPcThreads) {
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
            if (!empty) {
                const float h = 1.0f / obj_s.pc_inv_h;
                for (int cz = c0[2]; cz <= c1[2]; ++cz) {
                    // distance from q to the slab of cell layer cz (0 inside it)
                    const float z0 = obj_s.pc_lo[2] + cz * h;
                    const float dzs = fmaxf(fmaxf(z0 - q[2], q[2] - (z0 + h)), 0.0f);
                    for (int cy = c0[1]; cy <= c1[1]; ++cy) {
                        const float y0 = obj_s.pc_lo[1] + cy * h;
                        const float dys = fmaxf(fmaxf(y0 - q[1], q[1] - (y0 + h)), 0.0f);
                        // the sphere's x extent within this row of cells (skip the row if it misses)
                        const float w2 = rh * rh - dys * dys - dzs * dzs;
                        if (!(w2 > 0.0f)) continue;
                        const float w = sqrtf(w2) * 1.0001f;
                        const int x0 = max((int)floorf((q[0] - w - obj_s.pc_lo[0]) * obj_s.pc_inv_h), c0[0]);
                        const int x1 = min((int)floorf((q[0] + w - obj_s.pc_lo[0]) * obj_s.pc_inv_h), c1[0]);
                        if (x1 < x0) continue;
                        const int row = (cz * obj_s.pc_dims[1] + cy) * obj_s.pc_dims[0];
                        const int p0 = __ldg(obj_s.pc_start + row + x0), p1 = __ldg(obj_s.pc_start + row + x1 + 1);
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
                        // four points' loads in flight at a time (same order of the sums)
                        int k = p0;
                        for (; k + 3 < p1; k += 4) {
                            const float4 pa = __ldg(obj_s.pc_pts + k), pb = __ldg(obj_s.pc_pts + k + 1);
                            const float4 pc = __ldg(obj_s.pc_pts + k + 2), pd = __ldg(obj_s.pc_pts + k + 3);
                            add(pa); add(pb); add(pc); add(pd);
                        }
                        for (; k < p1; ++k) add(__ldg(obj_s.pc_pts + k));
                    }
                }
            }
        }
        const float kr = P.pc_k * rho, ksr = P.pc_ks * rho;
        a.pc_ft[g] = kr * sp * nn.x + ksr * sv[0];
        a.pc_ft[T + g] = kr * sp * nn.y + ksr * sv[1];
        a.pc_ft[2 * T + g] = kr * sp * nn.z + ksr * sv[2];
        a.pc_ft[3 * T + g] = kr * st[0];
        a.pc_ft[4 * T + g] = kr * st[1];
        a.pc_ft[5 * T + g] = kr * st[2];
    }
}

cudaError_t launch_pc_prox(const StepArgs& a, int n_items, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    pc_prox_kernel<<<n_items, kPcThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tg
