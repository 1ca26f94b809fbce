// mesh.cu -- exact signed distance to a closed triangle mesh at many points:
// the grid bake (points = grid nodes) and arbitrary point queries, with the
// kernel of mesh_kernel.cuh.
#include "mesh_kernel.cuh"

namespace tg {

static cudaError_t run(const float* tri, const float* tri_n, int nf, const MeshSrc& src, float* phi, float* grad,
                       void* grid, int fp16, cudaStream_t s) {
    if (src.n == 0) return cudaSuccess;
    const int64_t blocks = (src.n + kMeshThreads - 1) / kMeshThreads;
    mesh_sdf_kernel<kMeshThreads><<<(unsigned)blocks, kMeshThreads, 0, s>>>(tri, tri_n, nf, src, phi, grad, grid, fp16);
    return cudaGetLastError();
}

cudaError_t launch_mesh_sdf_points(const float* tri, const float* tri_n, int n_faces, const float* points, int64_t n,
                                   float* phi, float* grad, cudaStream_t s) {
    MeshSrc src{};
    src.points = points;
    src.n = n;
    src.mode = 0;
    return run(tri, tri_n, n_faces, src, phi, grad, nullptr, 0, s);
}

cudaError_t launch_mesh_bake(const float* tri, const float* tri_n, int n_faces, const int dims[3], const float lo[3],
                             const float hi[3], int fp16, void* out, cudaStream_t s) {
    MeshSrc src{};
    src.mode = 1;
    src.n = (int64_t)dims[0] * dims[1] * dims[2];
    for (int a = 0; a < 3; ++a) {
        src.dims[a] = dims[a];
        const double h = ((double)hi[a] - (double)lo[a]) / (double)(dims[a] - 1);
        src.lo_hi[a] = lo[a];
        src.lo_lo[a] = 0.0f;
        src.h_hi[a] = (float)h;
        src.h_lo[a] = (float)(h - (double)(float)h);
    }
    return run(tri, tri_n, n_faces, src, nullptr, nullptr, out, fp16, s);
}

}  // namespace tg
