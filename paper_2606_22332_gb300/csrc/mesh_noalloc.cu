// mesh_noalloc.cu -- exact mesh signed distance at points without any device
// allocation, for callers that cannot call cudaMalloc: code running inside
// a CUDA-graph capture that must not allocate, inside another framework's
// memory budget that forbids outside allocations, or on a path where an
// allocation's implicit synchronisation is not acceptable.
//
// tg_mesh_sdf copies the mesh into a triangle list it allocates per call.
// This variant builds that triangle list on the GPU in a file-scope
// device array instead, sized for kNoAllocMaxFaces faces (12 floats per face:
// three vertices and the unit normal; 3 MiB).  Every GPU that loads this
// library holds the array until the process exits.  All calls share it:
// each call overwrites the faces it uses and reads nothing left by an earlier
// call, but calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "mesh_kernel.cuh"

namespace tg {

constexpr int kNoAllocMaxFaces = TG_NOALLOC_MAX_FACES;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_tri[(size_t)kNoAllocMaxFaces * 12];

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
// floats) from the indexed mesh; an out-of-range index yields a NaN triangle
// instead of an out-of-bounds read.
__global__ void gather_triangles_kernel(const float* verts, int nv, const int32_t* faces, int nf, float* tri,
                                        float* tri_n) {
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
    const float nan = __int_as_float(0x7fc00000);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) tri[(size_t)f * 9 + 3 * k + a] = ok ? p[k][a] : nan;
    const float3 u = f3(p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]);
    const float3 w = f3(p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]);
    const float3 nrm = normalize_or(cross(u, w), f3(0.f, 0.f, 1.f));
    tri_n[(size_t)f * 3] = nrm.x;
    tri_n[(size_t)f * 3 + 1] = nrm.y;
    tri_n[(size_t)f * 3 + 2] = nrm.z;
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
    cudaStream_t st = (cudaStream_t)stream;
    gather_triangles_kernel<<<(n_faces + 127) / 128, 128, 0, st>>>(verts, n_verts, faces, n_faces, tri, tri_n);
    if (cudaGetLastError() != cudaSuccess) return TG_ERR_CUDA;
    if (launch_mesh_sdf_points(tri, tri_n, n_faces, points, n, phi, grad, st) != cudaSuccess) return TG_ERR_CUDA;
    return TG_OK;
}
