// bvh.cuh -- the raycast backend's bounding volume hierarchy over a
// triangle mesh: layout, the host build, the FP32 nearest-triangle walk and
// the walk that visits every triangle within a radius.  __host__ __device__
// so that the library's own walk can be checked on the host.
//
// Tree: median splits on the longest axis of the triangles' centroid box,
// leaves of at most 4 triangles, siblings stored next to each other.
#pragma once
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

namespace tg {

struct BvhNode {
    float lo[3];
    int32_t first;   // leaf: first triangle; inner node: left child (the right child is first + 1)
    float hi[3];
    int32_t count;   // leaf: triangles (> 0); inner node: 0
};

struct BvhTri {
    float4 a, b, c;  // vertices (w unused)
    float4 n;        // unit face normal in winding order (w unused)
};

constexpr int kBvhLeaf = 4;
constexpr int kBvhStack = 64;
constexpr int kBvhLbCells = 64;  // cells per axis of the distance lower-bound grid

__host__ __device__ inline float bvh_box_d2(const BvhNode& nd, float px, float py, float pz) {
    const float dx = fmaxf(fmaxf(nd.lo[0] - px, px - nd.hi[0]), 0.0f);
    const float dy = fmaxf(fmaxf(nd.lo[1] - py, py - nd.hi[1]), 0.0f);
    const float dz = fmaxf(fmaxf(nd.lo[2] - pz, pz - nd.hi[2]), 0.0f);
    return dx * dx + dy * dy + dz * dz;
}

// squared distance from p to triangle abc (Voronoi regions of the vertices,
// edges and face; vertices taken relative to p)
__host__ __device__ inline float bvh_tri_d2(const BvhTri& t, float px, float py, float pz) {
    const float ax = t.a.x - px, ay = t.a.y - py, az = t.a.z - pz;
    const float bx = t.b.x - px, by = t.b.y - py, bz = t.b.z - pz;
    const float cx = t.c.x - px, cy = t.c.y - py, cz = t.c.z - pz;
    const float abx = bx - ax, aby = by - ay, abz = bz - az;
    const float acx = cx - ax, acy = cy - ay, acz = cz - az;
    // ap = p - a = -a (p is the origin)
    const float d1 = -(abx * ax + aby * ay + abz * az), d2 = -(acx * ax + acy * ay + acz * az);
    float qx, qy, qz;  // closest point relative to p
    if (d1 <= 0.0f && d2 <= 0.0f) {
        qx = ax; qy = ay; qz = az;
    } else {
        const float d3 = -(abx * bx + aby * by + abz * bz), d4 = -(acx * bx + acy * by + acz * bz);
        if (d3 >= 0.0f && d4 <= d3) {
            qx = bx; qy = by; qz = bz;
        } else {
            const float vc = d1 * d4 - d3 * d2;
            const float d5 = -(abx * cx + aby * cy + abz * cz), d6 = -(acx * cx + acy * cy + acz * cz);
            const float vb = d5 * d2 - d1 * d6;
            const float va = d3 * d6 - d5 * d4;
            if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
                const float v = d1 / (d1 - d3);
                qx = ax + v * abx; qy = ay + v * aby; qz = az + v * abz;
            } else if (d6 >= 0.0f && d5 <= d6) {
                qx = cx; qy = cy; qz = cz;
            } else if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
                const float w = d2 / (d2 - d6);
                qx = ax + w * acx; qy = ay + w * acy; qz = az + w * acz;
            } else if (va <= 0.0f && (d4 - d3) >= 0.0f && (d5 - d6) >= 0.0f) {
                const float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
                qx = bx + w * (cx - bx); qy = by + w * (cy - by); qz = bz + w * (cz - bz);
            } else {
                const float den = 1.0f / (va + vb + vc);
                const float v = vb * den, w = vc * den;
                qx = ax + abx * v + acx * w; qy = ay + aby * v + acy * w; qz = az + abz * v + acz * w;
            }
        }
    }
    return qx * qx + qy * qy + qz * qz;
}

// nearest triangle to p with squared distance below r2 (-1 if none); *best_d2 its squared distance
__host__ __device__ inline int bvh_nearest(const BvhNode* nodes, const BvhTri* tris, float px, float py, float pz,
                                           float r2, float* best_d2) {
    float best = r2;
    int bi = -1;
    int stack[kBvhStack];
    float stack_d[kBvhStack];
    int sp = 0;
    if (!(bvh_box_d2(nodes[0], px, py, pz) < best)) {
        *best_d2 = best;
        return -1;
    }
    int node = 0;
    for (;;) {
        const BvhNode& nd = nodes[node];
        bool descend = false;
        if (nd.count > 0) {
            for (int k = nd.first; k < nd.first + nd.count; ++k) {
                const float d2 = bvh_tri_d2(tris[k], px, py, pz);
                if (d2 < best) {
                    best = d2;
                    bi = k;
                }
            }
        } else {
            const int l = nd.first, r = nd.first + 1;
            const float dl = bvh_box_d2(nodes[l], px, py, pz), dr = bvh_box_d2(nodes[r], px, py, pz);
            const int nearc = dl <= dr ? l : r, farc = dl <= dr ? r : l;
            const float dn = fminf(dl, dr), df = fmaxf(dl, dr);
            if (dn < best) {
                if (df < best && sp < kBvhStack) {
                    stack[sp] = farc;
                    stack_d[sp] = df;
                    ++sp;
                }
                node = nearc;
                descend = true;
            }
        }
        if (descend) continue;
        // next pending subtree still closer than the best triangle
        bool found = false;
        while (sp > 0) {
            --sp;
            if (stack_d[sp] < best) {
                node = stack[sp];
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    *best_d2 = best;
    return bi;
}

// host tree build; returns an error message or null
inline const char* bvh_build(const float* V, int nv, const int32_t* F, int nf, std::vector<BvhNode>& nodes,
                             std::vector<BvhTri>& tris, std::vector<int32_t>& face_id) {
    if (nf < 1 || nv < 3) return "the mesh needs at least one triangle";
    std::vector<float> cen((size_t)3 * nf);
    std::vector<BvhTri> all((size_t)nf);
    for (int f = 0; f < nf; ++f) {
        float p[3][3];
        for (int k = 0; k < 3; ++k) {
            const int v = F[3 * f + k];
            if (v < 0 || v >= nv) return "face index out of range";
            for (int a = 0; a < 3; ++a) {
                p[k][a] = V[3 * v + a];
                if (!std::isfinite(p[k][a])) return "vertices must be finite";
            }
        }
        const double e1[3] = {(double)p[1][0] - p[0][0], (double)p[1][1] - p[0][1], (double)p[1][2] - p[0][2]};
        const double e2[3] = {(double)p[2][0] - p[0][0], (double)p[2][1] - p[0][1], (double)p[2][2] - p[0][2]};
        double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double l = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int a = 0; a < 3; ++a) nn[a] = l > 0.0 ? nn[a] / l : 0.0;
        all[f].a = make_float4(p[0][0], p[0][1], p[0][2], 0.f);
        all[f].b = make_float4(p[1][0], p[1][1], p[1][2], 0.f);
        all[f].c = make_float4(p[2][0], p[2][1], p[2][2], 0.f);
        all[f].n = make_float4((float)nn[0], (float)nn[1], (float)nn[2], 0.f);
        for (int a = 0; a < 3; ++a) cen[3 * f + a] = (p[0][a] + p[1][a] + p[2][a]) / 3.0f;
    }
    std::vector<int32_t> idx((size_t)nf);
    for (int f = 0; f < nf; ++f) idx[f] = f;
    nodes.clear();
    nodes.reserve((size_t)2 * nf);
    nodes.push_back(BvhNode{});
    struct Job { int node, begin, end, depth; };
    std::vector<Job> jobs{{0, 0, nf, 0}};
    while (!jobs.empty()) {
        const Job j = jobs.back();
        jobs.pop_back();
        if (j.depth > kBvhStack - 4) return "the tree is too deep";
        BvhNode nd{};
        float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = INFINITY;
            nd.hi[a] = -INFINITY;
        }
        for (int k = j.begin; k < j.end; ++k) {
            const BvhTri& t = all[idx[k]];
            const float xs[3][3] = {{t.a.x, t.a.y, t.a.z}, {t.b.x, t.b.y, t.b.z}, {t.c.x, t.c.y, t.c.z}};
            for (int v = 0; v < 3; ++v)
                for (int a = 0; a < 3; ++a) {
                    nd.lo[a] = std::min(nd.lo[a], xs[v][a]);
                    nd.hi[a] = std::max(nd.hi[a], xs[v][a]);
                }
            for (int a = 0; a < 3; ++a) {
                clo[a] = std::min(clo[a], cen[3 * idx[k] + a]);
                chi[a] = std::max(chi[a], cen[3 * idx[k] + a]);
            }
        }
        if (j.end - j.begin <= kBvhLeaf) {
            nd.first = j.begin;
            nd.count = j.end - j.begin;
            nodes[j.node] = nd;
            continue;
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
        const int mid = (j.begin + j.end) / 2;
        std::nth_element(idx.begin() + j.begin, idx.begin() + mid, idx.begin() + j.end,
                         [&](int x, int y) { return cen[3 * x + axis] < cen[3 * y + axis]; });
        const int left = (int)nodes.size();
        nodes.push_back(BvhNode{});
        nodes.push_back(BvhNode{});
        nd.first = left;
        nd.count = 0;
        nodes[j.node] = nd;
        jobs.push_back({left + 1, mid, j.end, j.depth + 1});
        jobs.push_back({left, j.begin, mid, j.depth + 1});
    }
    tris.resize((size_t)nf);
    face_id.resize((size_t)nf);
    for (int k = 0; k < nf; ++k) {
        tris[k] = all[idx[k]];
        face_id[k] = idx[k];
    }
    return nullptr;
}

// Every triangle whose FP32 squared distance to p is below r2, in tree
// order: visit(k) for each.
template <class Visit>
__host__ __device__ inline void bvh_within(const BvhNode* nodes, const BvhTri* tris, float px, float py, float pz,
                                           float r2, Visit visit) {
    int stack[kBvhStack];
    int sp = 0;
    if (!(bvh_box_d2(nodes[0], px, py, pz) < r2)) return;
    stack[sp++] = 0;
    while (sp > 0) {
        const BvhNode& nd = nodes[stack[--sp]];
        if (nd.count > 0) {
            for (int k = nd.first; k < nd.first + nd.count; ++k)
                if (bvh_tri_d2(tris[k], px, py, pz) < r2) visit(k);
        } else {
            for (int c = 0; c < 2; ++c)
                if (bvh_box_d2(nodes[nd.first + c], px, py, pz) < r2 && sp < kBvhStack) stack[sp++] = nd.first + c;
        }
    }
}

#ifdef __CUDACC__
// The lower bound (from the grid below) on the distance from p to the mesh:
// the cell of p's projection onto the grid's box.  A NaN coordinate lands in
// cell 0 (the caller handles non-finite points first).
__device__ __forceinline__ float bvh_lower_bound(const float* lb, const float lo[3], const float inv_h[3], float px,
                                                 float py, float pz) {
    const float p[3] = {px, py, pz};
    int c[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float u = (p[ax] - lo[ax]) * inv_h[ax];
        c[ax] = min(max((int)floorf(fminf(fmaxf(u, 0.0f), (float)kBvhLbCells)), 0), kBvhLbCells - 1);
    }
    return lb[(c[2] * kBvhLbCells + c[1]) * kBvhLbCells + c[0]];
}
#endif

// Lower bound on the distance from any point of each cell of a
// kBvhLbCells^3 grid over the box [lo, hi] to the mesh: the FP32 distance
// from the cell centre to the nearest triangle, less the cell's half
// diagonal and a relative margin of 1e-6 of the box (covering the FP32
// distance's rounding), floored at 0.  For a point p outside the box, the
// cell of its projection onto the box bounds the distance of p too (the
// projection onto a convex set holding the mesh moves no point farther from
// it).  Cells are filled by `threads` host threads.
inline void bvh_lower_bounds(const std::vector<BvhNode>& nodes, const std::vector<BvhTri>& tris, const float lo[3],
                             const float hi[3], float* out, int threads) {
    const int n = kBvhLbCells;
    double h[3], ext2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        h[a] = ((double)hi[a] - (double)lo[a]) / n;
        ext2 += ((double)hi[a] - lo[a]) * ((double)hi[a] - lo[a]);
    }
    const double half_diag = 0.5 * std::sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    const double margin = 1e-6 * std::sqrt(ext2);
    auto work = [&](int t) {
        for (int c = t; c < n * n * n; c += threads) {
            const int i = c % n, j = (c / n) % n, k = c / (n * n);
            const float px = (float)(lo[0] + (i + 0.5) * h[0]), py = (float)(lo[1] + (j + 0.5) * h[1]),
                        pz = (float)(lo[2] + (k + 0.5) * h[2]);
            float best;
            bvh_nearest(nodes.data(), tris.data(), px, py, pz, INFINITY, &best);
            const double lb = std::sqrt((double)best) - half_diag - margin;
            out[c] = lb > 0.0 ? std::nextafter((float)lb, 0.0f) : 0.0f;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
}

}  // namespace tg
