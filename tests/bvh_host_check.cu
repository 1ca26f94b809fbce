// Host-side check of the raycast backend's tree: builds trees over random
// triangle soups with the library's own build, walks them with the library's
// own query (host-compiled, no GPU call) and compares every nearest distance
// with brute force over all triangles.  Prints "ok <checks>" or the first
// mismatch.
#include "bvh.cuh"

#include <cstdio>
#include <random>

int main() {
    std::mt19937 rng(7);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    long checks = 0;
    for (int trial = 0; trial < 24; ++trial) {
        const int nf = 1 + (trial * 53) % 2500;
        std::vector<float> V;
        std::vector<int32_t> F;
        for (int f = 0; f < nf; ++f) {
            const float cx = 0.05f * U(rng), cy = 0.05f * U(rng), cz = 0.05f * U(rng);
            for (int k = 0; k < 3; ++k) {
                V.push_back(cx + 0.004f * U(rng));
                V.push_back(cy + 0.004f * U(rng));
                V.push_back(cz + 0.004f * U(rng));
                F.push_back(3 * f + k);
            }
        }
        std::vector<tg::BvhNode> nodes;
        std::vector<tg::BvhTri> tris;
        std::vector<int32_t> fid;
        if (const char* m = tg::bvh_build(V.data(), (int)V.size() / 3, F.data(), nf, nodes, tris, fid)) {
            std::printf("build failed: %s\n", m);
            return 1;
        }
        std::vector<int> seen(nf, 0);
        for (int k = 0; k < nf; ++k) seen[fid[k]]++;
        for (int f = 0; f < nf; ++f)
            if (seen[f] != 1) {
                std::printf("face %d appears %d times\n", f, seen[f]);
                return 1;
            }
        for (int q = 0; q < 300; ++q) {
            const float px = 0.06f * U(rng), py = 0.06f * U(rng), pz = 0.06f * U(rng);
            const float r = 0.02f * (U(rng) + 1.0f);
            float best;
            const int k = tg::bvh_nearest(nodes.data(), tris.data(), px, py, pz, r * r, &best);
            float bb = r * r;
            int bk = -1;
            for (int t = 0; t < nf; ++t) {
                const float d2 = tg::bvh_tri_d2(tris[t], px, py, pz);
                if (d2 < bb) {
                    bb = d2;
                    bk = t;
                }
            }
            ++checks;
            if ((k < 0) != (bk < 0) || (k >= 0 && best != bb)) {
                std::printf("mismatch: trial %d query %d tree %d %.9g brute %d %.9g\n", trial, q, k, best, bk, bb);
                return 1;
            }
        }
    }
    std::printf("ok %ld\n", checks);
    return 0;
}
