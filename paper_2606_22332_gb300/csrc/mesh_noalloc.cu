// mesh_noalloc.cu -- exact mesh signed distance at points without any device
// allocation, for callers that cannot call cudaMalloc: an application whose
// own allocator owns all of the GPU's memory (a framework with a fixed
// memory budget that forbids allocations from outside it), or code on a path
// where cudaMalloc's implicit device-wide synchronisation is not acceptable
// (a control loop with a latency budget).
//
// tg_mesh_sdf copies the mesh into a triangle list it allocates per call.
// This variant builds that triangle list on the GPU in a file-scope
// device array instead, sized for kNoAllocMaxFaces faces (12 floats per face:
// three vertices and the unit normal; 3 MiB) plus one 256-byte block whose
// first word counts the call's invalid faces.  Every GPU that loads this
// library holds the array until the process exits.  All calls share it:
// each call clears the counter and overwrites the faces it uses, and reads
// nothing left by an earlier call, but calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it and must be
// serialised by the caller.
#include <algorithm>
#include <mutex>

#include "mesh_kernel.cuh"

namespace tg {

constexpr int kNoAllocMaxFaces = TG_NOALLOC_MAX_FACES;
constexpr int kNoAllocMaxDevices = 64;

constexpr size_t kNoAllocFlag = (size_t)kNoAllocMaxFaces * 12;   // float index of the invalid-face counter
static __device__ __align__(256) float g_noalloc_tri[kNoAllocFlag + 64];

// device address of g_noalloc_tri per device, resolved once per device
static float* g_noalloc_ptr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

static cudaError_t noalloc_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_tri);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// triangle list (vertices, then unit normals after kNoAllocMaxFaces * 9
// floats) from the indexed mesh.  A face with an index outside [0, nv) (read
// as a zero vertex, never out of bounds), with two equal indices, or with a
// zero FP32 cross product (zero area) is counted in *bad; the query's
// results are then set to NaN.
__global__ void gather_triangles_kernel(const float* verts, int nv, const int32_t* faces, int nf, float* tri,
                                        float* tri_n, unsigned int* bad) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    float p[3][3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int vi = faces[3 * f + k];
        ok = ok && vi >= 0 && vi < nv;
#pragma unroll
        for (int a = 0; a < 3; ++a) p[k][a] = (vi >= 0 && vi < nv) ? verts[3 * vi + a] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) tri[(size_t)f * 9 + 3 * k + a] = p[k][a];
    const float3 u = f3(p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]);
    const float3 w = f3(p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]);
    // each product rounded on its own (no fused multiply-add), so that two
    // equal edges give exactly zero
    const float3 cr = f3(__fsub_rn(__fmul_rn(u.y, w.z), __fmul_rn(u.z, w.y)),
                         __fsub_rn(__fmul_rn(u.z, w.x), __fmul_rn(u.x, w.z)),
                         __fsub_rn(__fmul_rn(u.x, w.y), __fmul_rn(u.y, w.x)));
    const int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    if (!ok || i0 == i1 || i1 == i2 || i0 == i2 || !(dot(cr, cr) > 0.0f)) atomicAdd(bad, 1u);
    const float3 nrm = normalize_or(cr, f3(0.f, 0.f, 1.f));
    tri_n[(size_t)f * 3] = nrm.x;
    tri_n[(size_t)f * 3 + 1] = nrm.y;
    tri_n[(size_t)f * 3 + 2] = nrm.z;
}

// every distance (and gradient) NaN when the mesh had an invalid face
__global__ void poison_kernel(const unsigned int* bad, int64_t n, float* phi, float* grad) {
    if (*bad == 0u) return;
    const float nan = __int_as_float(0x7fc00000);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        phi[i] = nan;
        if (grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = nan;
    }
}

static bool on_device(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_mesh_sdf_noalloc(const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                                         const float* points, int64_t n, float* phi, float* grad, tg_stream stream) {
    if (n_faces < 1 || n_faces > kNoAllocMaxFaces || n_verts < 3 || n < 0) return TG_ERR_INVALID_ARG;
    if (!verts || !faces || (n > 0 && (!points || !phi))) return TG_ERR_INVALID_ARG;
    if (!on_device(verts) || !on_device(faces)) return TG_ERR_INVALID_ARG;
    if (n > 0 && (!on_device(points) || !on_device(phi) || (grad && !on_device(grad)))) return TG_ERR_INVALID_ARG;
    float* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return TG_ERR_CUDA;
    float* tri = scratch;
    float* tri_n = scratch + (size_t)kNoAllocMaxFaces * 9;
    unsigned int* bad = reinterpret_cast<unsigned int*>(scratch + kNoAllocFlag);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(bad, 0, sizeof(unsigned int), st) != cudaSuccess) return TG_ERR_CUDA;
    gather_triangles_kernel<<<(n_faces + 127) / 128, 128, 0, st>>>(verts, n_verts, faces, n_faces, tri, tri_n, bad);
    if (cudaGetLastError() != cudaSuccess) return TG_ERR_CUDA;
    if (launch_mesh_sdf_points(tri, tri_n, n_faces, points, n, phi, grad, st) != cudaSuccess) return TG_ERR_CUDA;
    if (n > 0) {
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
        poison_kernel<<<(unsigned)blocks, 256, 0, st>>>(bad, n, phi, grad);
        if (cudaGetLastError() != cudaSuccess) return TG_ERR_CUDA;
    }
    return TG_OK;
}
