// raycast.cu -- the raycast contact-depth backend ("Two contact-depth
// backends"): a bounding volume hierarchy over a triangle mesh and, per
// probe, the deepest penetration over the triangles near it with the face
// normal of the triangle that gives it.
//
// The paper runs two tests per candidate triangle: a sphere-triangle
// closest-point test (penetration R - dist) and a ray-triangle test along the
// probe's sensing direction (penetration R - t).  A ray's hit lies on the
// triangle, so t is never below the triangle's distance and the ray test never
// gives the deeper value; the depth is R minus the distance to the nearest
// triangle within R, whichever tree is walked.  The query here is that nearest
// search: a stack walk visiting the nearer child first and pruning boxes no
// closer than the best triangle so far (or than R).
//
// Tree: median splits on the longest axis of the triangles' centroid box,
// leaves of at most 4 triangles, siblings stored next to each other.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "bvh.cuh"
#include "step_common.cuh"

namespace tg {

struct LowerBoundGrid {
    const float* lb;
    float lo[3], inv_h[3];
};

__global__ void raycast_depth_kernel(const BvhNode* __restrict__ nodes, const BvhTri* __restrict__ tris,
                                     const int32_t* __restrict__ face_id, const LowerBoundGrid lbg,
                                     const float* __restrict__ probes, const float* __restrict__ radius, int64_t n,
                                     float scale, float* depth, float* normal, int32_t* face) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float inv = 1.0f / scale;
    const float px = probes[3 * i] * inv, py = probes[3 * i + 1] * inv, pz = probes[3 * i + 2] * inv;
    const float R = radius[i], r = R * inv;
    float d = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;
    int f = -1;
    // probes no triangle can reach skip the walk (a non-finite probe walks and finds none)
    const bool reachable = !(isfinite(px) && isfinite(py) && isfinite(pz)) ||
                           bvh_lower_bound(lbg.lb, lbg.lo, lbg.inv_h, px, py, pz) < r;
    if (r > 0.0f && reachable) {
        float best;
        const int k = bvh_nearest(nodes, tris, px, py, pz, r * r, &best);
        if (k >= 0) {
            d = fmaxf(R - scale * sqrtf(best), 0.0f);
            if (d > 0.0f) {
                const float4 fn = tris[k].n;
                nx = fn.x; ny = fn.y; nz = fn.z;
                f = face_id[k];
            }
        }
    }
    depth[i] = d;
    if (normal) {
        normal[3 * i] = nx;
        normal[3 * i + 1] = ny;
        normal[3 * i + 2] = nz;
    }
    if (face) face[i] = f;
}

// Raycast backend inside the sensor step ("Two contact-depth backends"):
// for every taxel of an env whose object is a mesh, the distance from the
// probe centre to the nearest triangle within reach, with that triangle's
// normal (object frame).  The FP32 walk finds the nearest triangle within
// (R + 1 um) / s; every triangle within a guard of its distance is then
// re-evaluated in compensated arithmetic from the compensated probe centre,
// and the nearest wins (equal distances: the lowest original face index).
// The step kernel reads phi = s * distance as a float pair (depth R - phi)
// the way it reads a learned SDF's answer; a taxel with no triangle within
// reach gets phi = R + 1 m (clear).  One CTA per work item, in env order;
// items of other objects return at once.
constexpr int kRayStepThreads = 256;

// link of item taxel i: the last link start <= i
__device__ __forceinline__ int link_in(const int* start, int nl, int i) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kRayStepThreads)
    raycast_step_query_kernel(const StepArgs a, float* phi_hi, float* phi_lo, float* nrm) {
    __shared__ float rec_s[kItemMaxLinks][kLinkRec];
    __shared__ int start_s[kItemMaxLinks + 1];
    const Item it = a.items[blockIdx.x];
    const int e = it.env, L = a.max_links, lb = it.link_begin, nl = it.link_end - it.link_begin, n = it.n_taxels;
    const ObjDev* op = a.objects + min(max(a.obj_id[e], 0), a.n_objects - 1);
    if (op->kind != TG_OBJ_MESH || !op->bvh_nodes) return;  // the same for the whole CTA
    const BvhNode* nodes = static_cast<const BvhNode*>(op->bvh_nodes);
    const BvhTri* tris = static_cast<const BvhTri*>(op->bvh_tris);
    const int32_t* face = op->bvh_face;
    for (int v = threadIdx.x; v < nl * kLinkRec; v += blockDim.x)
        (&rec_s[0][0])[v] = a.link_rec[(size_t)(e * L + lb) * kLinkRec + v];
    if ((int)threadIdx.x <= nl) {
        const int base = a.lattice[e * L + lb].env_offset;
        start_s[threadIdx.x] = (int)threadIdx.x < nl ? a.lattice[e * L + lb + threadIdx.x].env_offset - base : n;
    }
    __syncthreads();
    const int64_t T = a.n_taxels;
    // pass 1: taxels whose lower-bound cell is out of reach are clear (no
    // triangle within R); the others are listed for the tree walk, so that
    // the walks run on whole warps
    __shared__ int16_t queue_s[kItemCap];
    __shared__ int nq_s;
    if (threadIdx.x == 0) nq_s = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t g = it.taxel_begin + i;
        const float R = a.R[g];
        if (!(R > 0.0f)) continue;
        const float* rec = rec_s[link_in(start_s, nl, i)];
        const float x0 = a.x[g], x1 = a.y[g], x2 = a.z[g];
        const float q[3] = {fmaf(rec[0], x0, fmaf(rec[1], x1, fmaf(rec[2], x2, rec[18]))),
                            fmaf(rec[3], x0, fmaf(rec[4], x1, fmaf(rec[5], x2, rec[19]))),
                            fmaf(rec[6], x0, fmaf(rec[7], x1, fmaf(rec[8], x2, rec[20])))};
        if (!(isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]))) {
            // a non-finite pose: phi is NaN, which the step kernel counts
            // (TG_ERR_NUMERIC) and reads as clear
            phi_hi[g] = __int_as_float(0x7fc00000);
            phi_lo[g] = 0.0f;
            nrm[g] = nrm[T + g] = nrm[2 * T + g] = 0.0f;
            continue;
        }
        const float reach = (R + 1e-6f) / rec[38];
        if (bvh_lower_bound(op->bvh_lb, op->bvh_lb_lo, op->bvh_lb_inv_h, q[0], q[1], q[2]) >= reach) {
            phi_hi[g] = R + 1.0f;
            phi_lo[g] = 0.0f;
            nrm[g] = nrm[T + g] = nrm[2 * T + g] = 0.0f;
        } else {
            queue_s[atomicAdd(&nq_s, 1)] = (int16_t)i;
        }
    }
    __syncthreads();
    // pass 2: the listed taxels, one per thread
    const int nq = nq_s;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
        const int i = queue_s[k];
        const int64_t g = it.taxel_begin + i;
        const float R = a.R[g];
        const float* rec = rec_s[link_in(start_s, nl, i)];
        const float x0 = a.x[g], x1 = a.y[g], x2 = a.z[g];
        const float qx = fmaf(rec[0], x0, fmaf(rec[1], x1, fmaf(rec[2], x2, rec[18])));
        const float qy = fmaf(rec[3], x0, fmaf(rec[4], x1, fmaf(rec[5], x2, rec[19])));
        const float qz = fmaf(rec[6], x0, fmaf(rec[7], x1, fmaf(rec[8], x2, rec[20])));
        const float s = rec[38];
        const float reach = (R + 1e-6f) / s;
        float best;
        const int k0 = bvh_nearest(nodes, tris, qx, qy, qz, reach * reach, &best);
        if (k0 < 0) {
            phi_hi[g] = R + 1.0f;
            phi_lo[g] = 0.0f;
            nrm[g] = nrm[T + g] = nrm[2 * T + g] = 0.0f;
            continue;
        }
        // the compensated probe centre, as the step's refinement forms it
        df qd[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            df acc = df{rec[18 + r], rec[21 + r]};
            acc = df_add(acc, df_mul_f(df{rec[3 * r], rec[9 + 3 * r]}, x0));
            acc = df_add(acc, df_mul_f(df{rec[3 * r + 1], rec[9 + 3 * r + 1]}, x1));
            acc = df_add(acc, df_mul_f(df{rec[3 * r + 2], rec[9 + 3 * r + 2]}, x2));
            qd[r] = acc;
        }
        const V3<dfn> pd{dfn{qd[0]}, dfn{qd[1]}, dfn{qd[2]}};
        const float lim = sqrtf(best) + 1e-6f / s;
        df bd = df_from(INFINITY);
        int bk = k0, bf = 0x7fffffff;
        bvh_within(nodes, tris, qx, qy, qz, lim * lim, [&](int kk) {
            const BvhTri& t = tris[kk];
            const V3<dfn> A{mk(t.a.x), mk(t.a.y), mk(t.a.z)}, B{mk(t.b.x), mk(t.b.y), mk(t.b.z)},
                C{mk(t.c.x), mk(t.c.y), mk(t.c.z)};
            V3<dfn> cp;
            int reg;
            const dfn d2 = closest_point_tri<dfn>(pd, A, B, C, &cp, &reg);
            const int fid = face[kk];
            if (df_lt(d2.v, bd) || (!df_lt(bd, d2.v) && fid < bf)) {
                bd = d2.v;
                bk = kk;
                bf = fid;
            }
        });
        const df phi = df_mul_f(df_sqrt(bd), s);
        phi_hi[g] = phi.hi;
        phi_lo[g] = phi.lo;
        const float4 fn = tris[bk].n;
        nrm[g] = fn.x;
        nrm[T + g] = fn.y;
        nrm[2 * T + g] = fn.z;
    }
}

cudaError_t launch_raycast_step_query(const StepArgs& a, int n_items, float* phi_hi, float* phi_lo, float* normal,
                                      cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    raycast_step_query_kernel<<<n_items, kRayStepThreads, 0, s>>>(a, phi_hi, phi_lo, normal);
    return cudaGetLastError();
}

const char* upload_mesh_bvh(const float* verts, int nv, const int32_t* faces, int nf, ObjDev* t,
                            std::vector<void*>* bufs) {
    std::vector<BvhNode> nodes;
    std::vector<BvhTri> tris;
    std::vector<int32_t> fid;
    if (const char* m = bvh_build(verts, nv, faces, nf, nodes, tris, fid)) return m;
    // the lower-bound grid over the mesh's box (a flat axis gets a 1 nm extent)
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = nodes[0].lo[a];
        hi[a] = std::max(nodes[0].hi[a], lo[a] + 1e-9f);
    }
    std::vector<float> lbg((size_t)kBvhLbCells * kBvhLbCells * kBvhLbCells);
    bvh_lower_bounds(nodes, tris, lo, hi, lbg.data(),
                     (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    float* dl = nullptr;
    BvhNode* dn = nullptr;
    BvhTri* dt = nullptr;
    int32_t* df_ = nullptr;
    cudaError_t e = cudaMalloc(&dn, sizeof(BvhNode) * nodes.size());
    if (dn) bufs->push_back(dn);
    if (e == cudaSuccess) e = cudaMalloc(&dt, sizeof(BvhTri) * tris.size());
    if (dt) bufs->push_back(dt);
    if (e == cudaSuccess) e = cudaMalloc(&df_, sizeof(int32_t) * fid.size());
    if (df_) bufs->push_back(df_);
    if (e == cudaSuccess) e = cudaMemcpy(dn, nodes.data(), sizeof(BvhNode) * nodes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dt, tris.data(), sizeof(BvhTri) * tris.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(df_, fid.data(), sizeof(int32_t) * fid.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(float) * lbg.size());
    if (dl) bufs->push_back(dl);
    if (e == cudaSuccess) e = cudaMemcpy(dl, lbg.data(), sizeof(float) * lbg.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return "mesh tree upload failed";
    t->bvh_nodes = dn;
    t->bvh_tris = dt;
    t->bvh_face = df_;
    t->bvh_lb = dl;
    for (int a = 0; a < 3; ++a) {
        t->bvh_lb_lo[a] = lo[a];
        t->bvh_lb_inv_h[a] = (float)kBvhLbCells / (hi[a] - lo[a]);
    }
    return nullptr;
}

}  // namespace tg

using namespace tg;

namespace {

thread_local std::string g_bvh_error;

tg_status bfail(tg_status st, const std::string& m) {
    g_bvh_error = m;
    return st;
}

bool b_is_dev(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct tg_mesh_bvh {
    BvhNode* nodes = nullptr;
    BvhTri* tris = nullptr;
    int32_t* face_id = nullptr;
    float* lb = nullptr;  // the distance lower-bound grid
    float lb_lo[3] = {0, 0, 0}, lb_inv_h[3] = {0, 0, 0};
    int32_t n_nodes = 0, n_tris = 0;
};

extern "C" {

tg_status tg_mesh_bvh_create(const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                             tg_mesh_bvh** out) {
    if (!verts || !faces || !out || n_verts < 3 || n_faces < 1)
        return bfail(TG_ERR_INVALID_ARG, "verts, faces and out with n_verts >= 3, n_faces >= 1 are required");
    *out = nullptr;
    std::vector<BvhNode> nodes;
    std::vector<BvhTri> tris;
    std::vector<int32_t> fid;
    if (const char* m = bvh_build(verts, n_verts, faces, n_faces, nodes, tris, fid))
        return bfail(TG_ERR_INVALID_ARG, m);
    tg_mesh_bvh* b = new tg_mesh_bvh();
    b->n_nodes = (int32_t)nodes.size();
    b->n_tris = n_faces;
    float hi[3];
    for (int a = 0; a < 3; ++a) {
        b->lb_lo[a] = nodes[0].lo[a];
        hi[a] = std::max(nodes[0].hi[a], b->lb_lo[a] + 1e-9f);
        b->lb_inv_h[a] = (float)kBvhLbCells / (hi[a] - b->lb_lo[a]);
    }
    std::vector<float> lbg((size_t)kBvhLbCells * kBvhLbCells * kBvhLbCells);
    bvh_lower_bounds(nodes, tris, b->lb_lo, hi, lbg.data(),
                     (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    cudaError_t e = cudaMalloc(&b->nodes, sizeof(BvhNode) * nodes.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->lb, sizeof(float) * lbg.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->lb, lbg.data(), sizeof(float) * lbg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->tris, sizeof(BvhTri) * tris.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->face_id, sizeof(int32_t) * fid.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->nodes, nodes.data(), sizeof(BvhNode) * nodes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tris, tris.data(), sizeof(BvhTri) * tris.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->face_id, fid.data(), sizeof(int32_t) * fid.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        tg_mesh_bvh_destroy(b);
        return bfail(e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA,
                     std::string("tree upload: ") + cudaGetErrorString(e));
    }
    *out = b;
    return TG_OK;
}

void tg_mesh_bvh_destroy(tg_mesh_bvh* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->nodes) cudaFree(b->nodes);
    if (b->tris) cudaFree(b->tris);
    if (b->face_id) cudaFree(b->face_id);
    if (b->lb) cudaFree(b->lb);
    delete b;
}

tg_status tg_raycast_depth(const tg_mesh_bvh* b, const float* probes, const float* radius, int64_t n, double scale,
                           float* depth, float* normal, int32_t* face, tg_stream stream) {
    if (!b || n < 0 || !(scale > 0.0) || !std::isfinite(scale))
        return bfail(TG_ERR_INVALID_ARG, "tree, n >= 0 and a finite scale > 0 are required");
    if (n == 0) return TG_OK;
    if (!probes || !radius || !depth || !b_is_dev(probes) || !b_is_dev(radius) || !b_is_dev(depth) ||
        (normal && !b_is_dev(normal)) || (face && !b_is_dev(face)))
        return bfail(TG_ERR_INVALID_ARG, "probes, radius, depth (and normal, face) must be device buffers");
    const unsigned blocks = (unsigned)((n + 127) / 128);
    LowerBoundGrid lbg{b->lb, {b->lb_lo[0], b->lb_lo[1], b->lb_lo[2]}, {b->lb_inv_h[0], b->lb_inv_h[1], b->lb_inv_h[2]}};
    raycast_depth_kernel<<<blocks, 128, 0, (cudaStream_t)stream>>>(b->nodes, b->tris, b->face_id, lbg, probes, radius,
                                                                   n, (float)scale, depth, normal, face);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(TG_ERR_CUDA, std::string("raycast launch: ") + cudaGetErrorString(e));
    return TG_OK;
}

const char* tg_mesh_bvh_last_error(void) { return g_bvh_error.c_str(); }

}  // extern "C"
