// nsdf_api.cu -- host side of the learned-SDF entry points declared in
// include/tg.h: parameter ownership, evaluation, the training loop
// (minibatch sampling, forward/backward, Adam) and the error probe.
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

using namespace tg;

namespace {

constexpr int kWeights = TG_NSDF_WEIGHTS;
constexpr int64_t kEntries = TG_NSDF_TABLE_ENTRIES;

thread_local std::string g_nsdf_error;

bool is_dev(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct tg_nsdf {
    NsdfNet net{};
    float* g_w = nullptr;       // [6208]
    float* g_table = nullptr;   // [16][2^16][2]
    float* g_part = nullptr;    // [ctas][6208]
    float* loss_part = nullptr; // [ctas]
    uint32_t* idx = nullptr;    // [batch]
    int64_t cap = 0;            // points the scratch holds
    unsigned* err = nullptr;    // inference CTAs stopped on an MMA wait timeout
};

namespace tg {

ObjDev nsdf_objdev(const NsdfNet& n) {
    ObjDev o{};
    o.kind = TG_OBJ_NEURAL;
    for (int a = 0; a < 3; ++a) {
        o.nlo[a] = n.lo[a];
        o.nhi[a] = n.hi[a];
        o.ninv_ext[a] = (float)(1.0 / ((double)n.hi[a] - (double)n.lo[a]));
    }
    o.ntable = n.table;
    o.nweights = n.weights;
    return o;
}

const NsdfNet* nsdf_net(const tg_nsdf* h) { return h ? &h->net : nullptr; }

}  // namespace tg

namespace {

tg_status nfail(tg_status st, const std::string& m) {
    g_nsdf_error = m;
    return st;
}

tg_status ncuda(cudaError_t e, const char* what) {
    return nfail(e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define NCK(call)                                  \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) return ncuda(_e, #call); \
    } while (0)

tg_status ensure_scratch(tg_nsdf* h, int64_t n) {
    if (n <= h->cap) return TG_OK;
    cudaFree(h->g_part);
    cudaFree(h->loss_part);
    cudaFree(h->idx);
    h->g_part = nullptr;
    h->loss_part = nullptr;
    h->idx = nullptr;
    h->cap = 0;
    const int ctas = nsdf_train_ctas(n);
    NCK(cudaMalloc(&h->g_part, sizeof(float) * (size_t)ctas * kWeights));
    NCK(cudaMalloc(&h->loss_part, sizeof(float) * (size_t)ctas));
    NCK(cudaMalloc(&h->idx, sizeof(uint32_t) * (size_t)n));
    h->cap = n;
    return TG_OK;
}

__global__ void scale_kernel(float* x, int64_t n, float s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= s;
}

__global__ void probe_err_kernel(const float* a, const float* b, int64_t n, double* out) {
    // out[0] = max |a - b| (mm), out[1] = sum |a - b| (mm); one CTA
    __shared__ double smax[256], ssum[256];
    double mx = 0.0, sm = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = fabs((double)a[i] - (double)b[i]) * 1e3;
        mx = d > mx ? d : mx;
        sm += d;
    }
    smax[threadIdx.x] = mx;
    ssum[threadIdx.x] = sm;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
            ssum[threadIdx.x] += ssum[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = smax[0];
        out[1] = ssum[0];
    }
}

}  // namespace

tg_status tg_nsdf_create(const float lo[3], const float hi[3], uint64_t seed, tg_nsdf** out) {
    if (!lo || !hi || !out) return nfail(TG_ERR_INVALID_ARG, "lo, hi and out are required");
    for (int a = 0; a < 3; ++a)
        if (!(lo[a] < hi[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a]))
            return nfail(TG_ERR_INVALID_ARG, "the box needs finite lo < hi on every axis");
    tg_nsdf* h = new tg_nsdf();
    for (int a = 0; a < 3; ++a) {
        h->net.lo[a] = lo[a];
        h->net.hi[a] = hi[a];
    }
    cudaError_t e = nsdf_alloc(&h->net);
    if (e == cudaSuccess) e = cudaMalloc(&h->g_w, sizeof(float) * kWeights);
    if (e == cudaSuccess) e = cudaMalloc(&h->g_table, sizeof(float) * 2 * (size_t)kEntries);
    if (e == cudaSuccess) e = cudaMalloc(&h->err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = nsdf_init(&h->net, seed, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        tg_nsdf_destroy(h);
        return ncuda(e, "tg_nsdf_create");
    }
    *out = h;
    return TG_OK;
}

void tg_nsdf_destroy(tg_nsdf* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    nsdf_free(&h->net);
    cudaFree(h->g_w);
    cudaFree(h->g_table);
    cudaFree(h->g_part);
    cudaFree(h->loss_part);
    cudaFree(h->idx);
    cudaFree(h->err);
    delete h;
}

tg_status tg_nsdf_set_params(tg_nsdf* h, const uint16_t* table, const uint16_t* weights) {
    if (!h || !table || !weights) return nfail(TG_ERR_INVALID_ARG, "net, table and weights are required");
    NCK(cudaMemcpy(h->net.table, table, sizeof(uint32_t) * (size_t)kEntries, cudaMemcpyDefault));
    NCK(cudaMemcpy(h->net.weights, weights, sizeof(uint16_t) * kWeights, cudaMemcpyDefault));
    NCK(nsdf_sync_masters(&h->net, 0));
    NCK(cudaDeviceSynchronize());
    return TG_OK;
}

tg_status tg_nsdf_get_params(tg_nsdf* h, uint16_t* table, uint16_t* weights) {
    if (!h) return nfail(TG_ERR_INVALID_ARG, "net is NULL");
    NCK(cudaDeviceSynchronize());
    if (table) NCK(cudaMemcpy(table, h->net.table, sizeof(uint32_t) * (size_t)kEntries, cudaMemcpyDefault));
    if (weights) NCK(cudaMemcpy(weights, h->net.weights, sizeof(uint16_t) * kWeights, cudaMemcpyDefault));
    return TG_OK;
}

tg_status tg_nsdf_eval(tg_nsdf* h, const float* points, int64_t n, float* phi, float* grad, tg_stream stream) {
    if (!h || n < 0 || (n > 0 && (!points || !phi))) return nfail(TG_ERR_INVALID_ARG, "net, points and phi are required");
    if (n > 0 && (!is_dev(points) || !is_dev(phi) || (grad && !is_dev(grad))))
        return nfail(TG_ERR_INVALID_ARG, "points, phi and grad must be device buffers");
    NCK(launch_nsdf_eval(nsdf_objdev(h->net), points, n, phi, grad, h->err, (cudaStream_t)stream));
    return TG_OK;
}

tg_status tg_nsdf_loss_grad(tg_nsdf* h, const float* points, const float* labels_mm, int64_t n, double* loss,
                            float* g_weights, float* g_table, tg_stream stream) {
    if (!h || n < 1 || !points || !labels_mm) return nfail(TG_ERR_INVALID_ARG, "net, points, labels and n >= 1 required");
    if (!is_dev(points) || !is_dev(labels_mm) || (g_weights && !is_dev(g_weights)) || (g_table && !is_dev(g_table)))
        return nfail(TG_ERR_INVALID_ARG, "points, labels and gradient buffers must be device buffers");
    if (tg_status st = ensure_scratch(h, n)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    NCK(cudaMemsetAsync(h->g_table, 0, sizeof(float) * 2 * (size_t)kEntries, s));
    NCK(launch_nsdf_train_step(nsdf_objdev(h->net), points, labels_mm, nullptr, n, h->g_part, h->g_w, h->g_table,
                               h->loss_part, s));
    const float inv = (float)(1.0 / (double)n);
    scale_kernel<<<(kWeights + 255) / 256, 256, 0, s>>>(h->g_w, kWeights, inv);
    scale_kernel<<<(unsigned)((2 * kEntries + 255) / 256), 256, 0, s>>>(h->g_table, 2 * kEntries, inv);
    NCK(cudaGetLastError());
    if (g_weights) NCK(cudaMemcpyAsync(g_weights, h->g_w, sizeof(float) * kWeights, cudaMemcpyDeviceToDevice, s));
    if (g_table)
        NCK(cudaMemcpyAsync(g_table, h->g_table, sizeof(float) * 2 * (size_t)kEntries, cudaMemcpyDeviceToDevice, s));
    const int ctas = nsdf_train_ctas(n);
    std::vector<float> lp(ctas);
    NCK(cudaMemcpyAsync(lp.data(), h->loss_part, sizeof(float) * ctas, cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
    double sum = 0.0;
    for (float v : lp) sum += v;
    if (loss) *loss = sum / (double)n;
    return TG_OK;
}

tg_status tg_nsdf_train(tg_nsdf* h, const float* points, const float* labels_mm, int64_t n, int32_t steps,
                        int32_t batch, double lr0, double lr_final, uint64_t seed, float* losses, tg_stream stream) {
    if (!h || n < 1 || !points || !labels_mm || steps < 0 || batch < 1 || !(lr0 > 0.0) || !(lr_final > 0.0))
        return nfail(TG_ERR_INVALID_ARG, "net, points, labels, n >= 1, batch >= 1 and positive rates are required");
    if (n > 0xffffffffLL) return nfail(TG_ERR_INVALID_ARG, "at most 2^32 - 1 labelled points");
    if (!is_dev(points) || !is_dev(labels_mm)) return nfail(TG_ERR_INVALID_ARG, "points and labels must be device buffers");
    if (tg_status st = ensure_scratch(h, batch)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int ctas = nsdf_train_ctas(batch);
    std::vector<float> lp(ctas);
    for (int32_t t = 0; t < steps; ++t) {
        const double lr = lr0 * std::pow(lr_final / lr0, (double)t / (double)(steps > 1 ? steps - 1 : 1));
        NCK(launch_nsdf_sample(seed, (uint32_t)t, n, batch, h->idx, s));
        NCK(cudaMemsetAsync(h->g_table, 0, sizeof(float) * 2 * (size_t)kEntries, s));
        NCK(launch_nsdf_train_step(nsdf_objdev(h->net), points, labels_mm, h->idx, batch, h->g_part, h->g_w,
                                   h->g_table, h->loss_part, s));
        NCK(launch_nsdf_adam(&h->net, h->g_w, h->g_table, (float)lr, (float)(1.0 / batch), s));
        if (losses) {
            NCK(cudaMemcpyAsync(lp.data(), h->loss_part, sizeof(float) * ctas, cudaMemcpyDeviceToHost, s));
            NCK(cudaStreamSynchronize(s));
            double sum = 0.0;
            for (float v : lp) sum += v;
            losses[t] = (float)(sum / batch);
        }
    }
    return TG_OK;
}

tg_status tg_nsdf_probe(tg_nsdf* h, const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                        const float* points, int64_t n, double* max_err_mm, double* mean_err_mm, tg_stream stream) {
    if (!h || n < 1 || !points || !is_dev(points)) return nfail(TG_ERR_INVALID_ARG, "net and device points are required");
    cudaStream_t s = (cudaStream_t)stream;
    float *phi_n = nullptr, *phi_m = nullptr;
    double* stats = nullptr;
    NCK(cudaMallocAsync(&phi_n, sizeof(float) * n, s));
    NCK(cudaMallocAsync(&phi_m, sizeof(float) * n, s));
    NCK(cudaMallocAsync(&stats, sizeof(double) * 2, s));
    tg_status st = tg_mesh_sdf(verts, n_verts, faces, n_faces, points, n, phi_m, nullptr, stream);
    if (st == TG_OK) st = tg_nsdf_eval(h, points, n, phi_n, nullptr, stream);
    double out[2] = {0.0, 0.0};
    unsigned timeouts = 0;
    if (st == TG_OK) {
        probe_err_kernel<<<1, 256, 0, s>>>(phi_n, phi_m, n, stats);
        cudaError_t e = cudaMemcpyAsync(out, stats, sizeof(out), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&timeouts, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = ncuda(e, "probe");
        else if (timeouts) {
            cudaMemset(h->err, 0, sizeof(unsigned));
            st = nfail(TG_ERR_TIMEOUT, "a tensor-core MMA of the network's evaluation did not complete in time");
        }
    }
    cudaFreeAsync(phi_n, s);
    cudaFreeAsync(phi_m, s);
    cudaFreeAsync(stats, s);
    if (st != TG_OK) return st;
    if (max_err_mm) *max_err_mm = out[0];
    if (mean_err_mm) *mean_err_mm = out[1] / (double)n;
    return TG_OK;
}

const char* tg_nsdf_last_error(void) { return g_nsdf_error.c_str(); }
