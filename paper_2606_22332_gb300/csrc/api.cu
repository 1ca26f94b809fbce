// api.cu -- host side of the C-ABI declared in include/tg.h: argument
// validation, scene layout (CSR work items, link lattices), device
// allocation, staging of host inputs, launches, reads and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace tg {

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> mark;  // (kernel, device) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& m = mark[{func, dev}];
    if (bytes <= m) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) m = bytes;
    return e;
}

}  // namespace tg

using namespace tg;

struct ObjInfo {
    int32_t kind = 0;
    double err_mm = NAN;
};

struct tg_scene {
    int E = 0, L = 0;
    int64_t T = 0;
    uint32_t sensors = 0;
    int64_t gid0 = 0;
    int env_gid0 = 0;
    tg_params params{};
    ParamsDev P{};
    std::vector<Item> items_h;
    int n_items = 0;
    // device: geometry and layout
    float *x = nullptr, *y = nullptr, *z = nullptr, *nx = nullptr, *ny = nullptr, *nz = nullptr, *R = nullptr;
    Item* items = nullptr;
    LinkLattice* lattice = nullptr;
    // objects
    ObjDev* objects = nullptr;
    int n_objects = 0;
    std::vector<void*> obj_bufs;
    // state
    uint8_t* flags = nullptr;
    float *hyst_prev = nullptr, *hyst_xi = nullptr, *drift = nullptr;
    uint32_t* episode = nullptr;
    // outputs
    float *depth_clean = nullptr, *depth_noisy = nullptr, *dist = nullptr;
    float *ft_clean = nullptr, *ft_noisy = nullptr, *link_out = nullptr;
    int32_t* link_count = nullptr;
    unsigned* err = nullptr;
    float* link_rec = nullptr;
    float* ring = nullptr;            // [ring_k][8][T] read-delay history (read delay on)
    // staging of host inputs: two sets, filled in turn on the copy stream so
    // that a step's host-to-device copies overlap the previous step's kernels
    // (set k is refilled once the kernels of the step that read it are done)
    float *s_link_pose[2] = {}, *s_link_vel[2] = {}, *s_obj_pose[2] = {}, *s_obj_vel[2] = {};
    float* s_env_params[2] = {};
    int32_t* s_obj_id[2] = {};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t staged_ev[2] = {nullptr, nullptr}, used_ev[2] = {nullptr, nullptr};
    // the work-item order kernel runs on aux_stream beside the pose kernel
    // (it reads only the step's object ids): fork_ev / join_ev bracket it
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool used_rec[2] = {false, false};
    int next_set = 0;
    uint8_t* s_mask = nullptr;
    uint8_t* s_contact = nullptr;
    Item* items_sorted = nullptr;     // per-step object-sorted copy of the items
    // proximity and markers
    float *prox_clean = nullptr, *prox_noisy = nullptr;
    float* pc_ft = nullptr;            // [6][T] point-cloud proximity (sensor on)
    MarkerArgs markers{};
    int32_t* pad_link = nullptr;
    float* pad_frame = nullptr;
    float* marker_u = nullptr;
    float2* anchors = nullptr;         // shear anchors [E][P][shear_points]
    int32_t* anchor_obj = nullptr;     // [E][P]
    int32_t* n_anchored = nullptr;     // [E][P]

    // objects as uploaded; learned-SDF query scratch
    std::vector<ObjInfo> obj_info;
    bool any_neural = false;
    float* nq_phi = nullptr;          // [T]
    float* nq_grad = nullptr;         // [3][T]
    float* nq_phi_lo = nullptr;       // [T] (raycast backend)
    bool any_raycast = false;         // a mesh object answered by the raycast backend
    bool all_grid = false;            // every object is a plain SDF grid
    // schedule (tg_set_schedule / tg_autotune) and step control
    int schedule = TG_SCHED_GRID;     // step kernel schedule (tg_schedule)
    int sorted = 1;                   // object-sorted item order (several objects)
    // threads per CTA of the sensor kernels (tg_sensor_kernel order: proximity,
    // point-cloud proximity, markers)
    int sensor_threads[3] = {256, 256, 256};
    int resident_ctas[kStepShapes] = {0, 0};  // step kernel CTAs resident on the device at once, per shape
    int sms = 0;                      // streaming multiprocessors (pipelined schedules: one CTA each)
    ItemMeta* metas = nullptr;        // [n_items] static item layout (pipelined schedules)
    SlotRec* slots = nullptr;         // [n_items] this step's order records (pipelined schedules)
    StepCtl* ctl = nullptr;
    // captured step (tg_graph_*)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphNode_t graph_ev_node[3] = {nullptr, nullptr, nullptr};  // timing events of the replay
    cudaEvent_t graph_ev[3] = {nullptr, nullptr, nullptr};

    std::string last_error;
    // kernel timing (tg_profile_*)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<cudaEvent_t> ev_pending;   // triples: before pose, after pose, after step
};

namespace {

thread_local std::string g_create_error;

tg_status fail(tg_scene* s, tg_status st, const std::string& msg) {
    if (s) s->last_error = msg;
    else g_create_error = msg;
    return st;
}

tg_status cuda_fail(tg_scene* s, cudaError_t e, const char* what) {
    return fail(s, e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(scene, call)                                                 \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return cuda_fail((scene), _e, #call);    \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

bool finite(double v) { return std::isfinite(v); }

NoiseDev make_group(const tg_noise_group& g, double dt) {
    NoiseDev n{};
    n.gain_lo = (float)g.gain_lo;
    n.gain_span = (float)(g.gain_hi - g.gain_lo);
    n.gain_on = !(g.gain_lo == 1.0 && g.gain_hi == 1.0);
    n.beta = (float)g.beta;
    n.decay = g.tau > 0.0 ? (float)std::exp(-dt / g.tau) : 0.0f;
    n.bias = (float)g.bias;
    n.sigma_white = (float)g.sigma_white;
    n.sigma_rw = (float)g.sigma_rw;
    n.quant = (float)g.quant;
    n.stuck_lo = (float)g.stuck_lo;
    n.stuck_span = (float)(g.stuck_hi - g.stuck_lo);
    return n;
}

const char* check_group(const tg_noise_group& g) {
    const double v[] = {g.gain_lo, g.gain_hi, g.beta, g.tau, g.bias, g.sigma_white, g.sigma_rw, g.quant,
                        g.stuck_lo, g.stuck_hi};
    for (double x : v)
        if (!finite(x)) return "non-finite noise parameter";
    if (g.gain_hi < g.gain_lo || g.stuck_hi < g.stuck_lo) return "noise range with hi < lo";
    if (g.beta != 0.0 && !(g.tau > 0.0)) return "hysteresis needs tau > 0";
    if (g.sigma_white < 0 || g.sigma_rw < 0 || g.quant < 0) return "negative noise sigma or quantisation step";
    return nullptr;
}

const char* make_params(const tg_params& p, ParamsDev* out) {
    const double v[] = {p.k, p.c, p.alpha, p.k_t, p.k_omega, p.mu, p.eta_on, p.eta_off, p.dt, p.p_dead, p.chi, p.xt_sigma};
    for (double x : v)
        if (!finite(x)) return "non-finite parameter";
    if (p.eta_off > p.eta_on) return "eta_off must not exceed eta_on";
    if (!(p.dt > 0.0)) return "dt must be positive";
    if (p.p_dead < 0.0 || p.p_dead > 1.0) return "p_dead outside [0, 1]";
    if (!(p.alpha > 0.0)) return "alpha must be positive";
    if (p.chi != 0.0 && !(p.xt_sigma > 0.0)) return "crosstalk needs xt_sigma > 0";
    if (!finite(p.probe_radius_noise) || p.probe_radius_noise < 0.0 || p.probe_radius_noise > 5e-4)
        return "probe_radius_noise must be in [0, 5e-4] m";
    if (p.prox_rays < 0 || p.prox_rays > 16 || !finite(p.prox_range) || !finite(p.prox_cone))
        return "prox_rays must be in 0..16 with finite range and cone";
    if (p.dr_on) {
        const double* b[3] = {p.dr_mu, p.dr_k, p.dr_scale};
        for (int i = 0; i < 3; ++i)
            if (!finite(b[i][0]) || !finite(b[i][1]) || b[i][0] > b[i][1])
                return "domain randomisation bounds must be finite with lo <= hi";
        if (!(p.dr_scale[0] > 0.0)) return "domain randomisation scale must be positive";
        if (p.dr_k[0] < 0.0) return "domain randomisation k must be non-negative";
    }
    for (const tg_noise_group* g : {&p.depth, &p.ft, &p.prox})
        if (const char* m = check_group(*g)) return m;
    ParamsDev d{};
    d.k = (float)p.k;
    d.c = (float)p.c;
    d.alpha = (float)p.alpha;
    d.k_t = (float)p.k_t;
    d.k_omega = (float)p.k_omega;
    d.mu = (float)p.mu;
    d.eta_on_hi = (float)p.eta_on;
    d.eta_on_lo = (float)(p.eta_on - (double)d.eta_on_hi);
    d.eta_off_hi = (float)p.eta_off;
    d.eta_off_lo = (float)(p.eta_off - (double)d.eta_off_hi);
    d.dead_threshold24 = (uint32_t)std::nearbyint(p.p_dead * 16777216.0);
    d.chi = (float)p.chi;
    double w[9], sum = 0.0;
    for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
            double s = p.xt_sigma > 0.0 ? p.xt_sigma : 1.0;
            w[(di + 1) * 3 + dj + 1] = std::exp(-(double)(di * di + dj * dj) / (2.0 * s * s));
            sum += w[(di + 1) * 3 + dj + 1];
        }
    for (int i = 0; i < 9; ++i) d.xt_w[i] = (float)(w[i] / sum);
    d.seed = p.seed;
    d.rho = (float)p.probe_radius_noise;
    d.pc_radius = (float)p.pc_radius;
    d.pc_k = (float)p.pc_k;
    d.pc_ks = (float)p.pc_ks;
    d.pc_density = (float)p.pc_density;
    if (p.read_delay < 0 || p.read_jitter < 0 || p.read_jitter > 255 || p.read_delay + p.read_jitter > 63)
        return "read_delay >= 0 and read_jitter in 0..255 with read_delay + read_jitter <= 63";
    d.delay = p.read_delay;
    d.jitter = p.read_jitter;
    d.ring_k = p.read_delay + p.read_jitter + 1;
    if (p.depth_backend != 0 && p.depth_backend != 1) return "depth_backend must be 0 (sdf) or 1 (raycast)";
    if (p.depth_backend == 1 && p.probe_radius_noise > 0.0)
        return "probe-radius noise is not supported with the raycast depth backend";
    d.depth_backend = p.depth_backend;
    d.prev_out = (p.probe_radius_noise == 0.0 && d.ring_k == 1) ? 1 : 0;
    for (uint32_t r = 0; r < 10; ++r) {
        d.rk[2 * r] = (uint32_t)p.seed + r * 0x9E3779B9u;
        d.rk[2 * r + 1] = (uint32_t)(p.seed >> 32) + r * 0xBB67AE85u;
    }
    d.depth = make_group(p.depth, p.dt);
    d.ft = make_group(p.ft, p.dt);
    d.prox = make_group(p.prox, p.dt);
    d.prox_rays = p.prox_rays;
    d.prox_range = (float)p.prox_range;
    d.prox_cos = (float)std::cos(p.prox_cone);
    d.prox_sin = (float)std::sin(p.prox_cone);
    for (int k = 0; k < 16; ++k) {
        const double az = (k >= 1 && p.prox_rays > 1) ? 2.0 * 3.14159265358979323846 * (k - 1) / (p.prox_rays - 1) : 0.0;
        d.prox_az_cos[k] = (float)std::cos(az);
        d.prox_az_sin[k] = (float)std::sin(az);
    }
    d.dr_on = p.dr_on ? 1 : 0;
    const double* b[3] = {p.dr_mu, p.dr_k, p.dr_scale};
    for (int i = 0; i < 3; ++i) {
        d.dr_lo[i] = (float)b[i][0];
        d.dr_hi[i] = (float)b[i][1];
    }
    *out = d;
    return nullptr;
}

// the step kernel of a schedule: pipelined, persistent, and its CTA shape
bool sched_pipe(int sc) { return sc >= TG_SCHED_PIPE_1024 && sc <= TG_SCHED_PIPE_512; }
bool sched_persistent(int sc) { return sc == TG_SCHED_PERSISTENT || sc == TG_SCHED_PERSISTENT_384; }
int sched_shape(int sc) { return (sc == TG_SCHED_GRID_384 || sc == TG_SCHED_PERSISTENT_384) ? 1 : 0; }

StepArgs step_args(tg_scene* s) {
    StepArgs a{};
    a.x = s->x; a.y = s->y; a.z = s->z; a.nx = s->nx; a.ny = s->ny; a.nz = s->nz; a.R = s->R;
    a.items = s->items;
    a.lattice = s->lattice;
    a.objects = s->objects;
    a.n_objects = s->n_objects;
    a.n_envs = s->E;
    a.max_links = s->L;
    a.n_taxels = s->T;
    a.gid0 = s->gid0;
    a.sensors = s->sensors;
    a.P = s->P;
    a.link_rec = s->link_rec;
    a.flags = s->flags;
    a.hyst_prev = s->hyst_prev;
    a.hyst_xi = s->hyst_xi;
    a.drift = s->drift;
    a.episode = s->episode;
    a.ring = s->ring;
    a.env_gid0 = s->env_gid0;
    a.depth_clean = s->depth_clean;
    a.depth_noisy = s->depth_noisy;
    a.dist = s->dist;
    a.ft_clean = s->ft_clean;
    a.ft_noisy = s->ft_noisy;
    a.link_out = s->link_out;
    a.link_count = s->link_count;
    a.err = s->err;
    a.prox_clean = s->prox_clean;
    a.pc_ft = s->pc_ft;
    a.prox_noisy = s->prox_noisy;
    a.ctl = s->ctl;
    a.n_items = s->n_items;
    a.persistent = sched_persistent(s->schedule) ? 1 : 0;
    a.shape = sched_shape(s->schedule);
    a.resident_ctas = s->resident_ctas[a.shape];
    a.metas = s->metas;
    a.slots = s->slots;
    a.sms = s->sms;
    a.nq_phi = s->nq_phi;
    a.nq_grad = s->nq_grad;
    a.nq_phi_lo = s->nq_phi_lo;
    a.any_neural = s->any_neural ? 1 : 0;
    a.all_grid = s->all_grid ? 1 : 0;
    return a;
}

// device copy of a host-or-device input: returns the pointer the kernels read
template <class T>
cudaError_t stage(const T* src, T* staging, size_t count, cudaStream_t st, const T** out) {
    if (is_device_ptr(src)) {
        *out = src;
        return cudaSuccess;
    }
    *out = staging;
    return cudaMemcpyAsync(staging, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
}

void free_objects(tg_scene* s) {
    for (void* p : s->obj_bufs) dfree(p);
    s->obj_bufs.clear();
    dfree(s->objects);
    s->objects = nullptr;
    s->n_objects = 0;
}

// host copy of a host-or-device array
template <class T>
bool host_copy(const T* src, size_t count, std::vector<T>* out) {
    out->resize(count);
    if (count == 0) return true;
    return cudaMemcpy(out->data(), src, count * sizeof(T), cudaMemcpyDefault) == cudaSuccess;
}

// triangles [nf][9] and unit outward normals [nf][3] from an indexed mesh
const char* build_triangles(const float* verts, int nv, const int32_t* faces, int nf, std::vector<float>* tri,
                            std::vector<float>* tri_n) {
    if (nv < 3 || nf < 1 || !verts || !faces) return "mesh needs >= 3 vertices and >= 1 face";
    std::vector<float> V;
    std::vector<int32_t> F;
    if (!host_copy(verts, (size_t)nv * 3, &V) || !host_copy(faces, (size_t)nf * 3, &F)) return "mesh copy failed";
    tri->resize((size_t)nf * 9);
    tri_n->resize((size_t)nf * 3);
    for (int f = 0; f < nf; ++f) {
        double p[3][3];
        for (int k = 0; k < 3; ++k) {
            int vi = F[3 * f + k];
            if (vi < 0 || vi >= nv) return "face index out of range";
            for (int a = 0; a < 3; ++a) {
                p[k][a] = V[3 * vi + a];
                (*tri)[(size_t)f * 9 + 3 * k + a] = V[3 * vi + a];
            }
        }
        double u[3], w[3], n[3];
        for (int a = 0; a < 3; ++a) { u[a] = p[1][a] - p[0][a]; w[a] = p[2][a] - p[0][a]; }
        n[0] = u[1] * w[2] - u[2] * w[1];
        n[1] = u[2] * w[0] - u[0] * w[2];
        n[2] = u[0] * w[1] - u[1] * w[0];
        double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0)) return "degenerate (zero-area) face";
        for (int a = 0; a < 3; ++a) (*tri_n)[(size_t)f * 3 + a] = (float)(n[a] / nn);
    }
    return nullptr;
}

}  // namespace

extern "C" {

int32_t tg_max_link_taxels(void) { return kItemCap; }

tg_status tg_create_scene(const tg_scene_desc* d, tg_scene** out) {
    if (!out) return fail(nullptr, TG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(nullptr, TG_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_envs < 1 || d->max_links < 1 || d->max_links > kMaxLinks)
        return fail(nullptr, TG_ERR_INVALID_ARG, "n_envs must be >= 1 and max_links in 1..255");
    if (!d->taxel_offsets || !d->link_rows || !d->link_cols)
        return fail(nullptr, TG_ERR_INVALID_ARG, "taxel_offsets, link_rows and link_cols are required");
    const int E = d->n_envs, L = d->max_links;
    if (d->taxel_offsets[0] != 0) return fail(nullptr, TG_ERR_INVALID_ARG, "taxel_offsets[0] must be 0");
    for (int e = 0; e < E; ++e)
        if (d->taxel_offsets[e + 1] < d->taxel_offsets[e])
            return fail(nullptr, TG_ERR_INVALID_ARG, "taxel_offsets must be non-decreasing");
    const int64_t T = d->taxel_offsets[E];
    if (T >= kMaxSceneTaxels - 64) return fail(nullptr, TG_ERR_INVALID_ARG, "a scene holds fewer than 2^31 taxels");
    if (T > 0 && (!d->x || !d->y || !d->z || !d->nx || !d->ny || !d->nz || !d->R))
        return fail(nullptr, TG_ERR_INVALID_ARG, "taxel geometry pointers are required");
    ParamsDev P;
    if (const char* m = make_params(d->params, &P)) return fail(nullptr, TG_ERR_INVALID_ARG, m);
    if ((d->sensors & TG_SENSOR_PROX) && (d->params.prox_rays < 1 || !(d->params.prox_range > 0.0)))
        return fail(nullptr, TG_ERR_INVALID_ARG, "TG_SENSOR_PROX needs prox_rays in 1..16 and prox_range > 0");
    if ((d->sensors & TG_SENSOR_PCPROX) &&
        (!(d->params.pc_radius > 0.0) || d->params.pc_radius > 0.1 || !std::isfinite(d->params.pc_k) ||
         !std::isfinite(d->params.pc_ks) || !(d->params.pc_density >= 0.0) || !std::isfinite(d->params.pc_density)))
        return fail(nullptr, TG_ERR_INVALID_ARG,
                    "TG_SENSOR_PCPROX needs pc_radius in (0, 0.1] m, finite pc_k and pc_ks, pc_density >= 0");
    const tg_pad_desc& pd = d->pads;
    if (d->sensors & TG_SENSOR_MARKERS) {
        if (pd.pads_per_env < 1 || pd.rows < 1 || pd.cols < 1 || pd.rows * pd.cols > kMaxPadMarkers ||
            pd.radius < 0 || pd.radius > kMaxPadRadius || !(pd.pitch > 0.0) || !pd.pad_link || !pd.pad_frame ||
            !(pd.lambda_d > 0.0) || !(pd.eps > 0.0) || !std::isfinite(pd.s_d) || !std::isfinite(pd.alpha) || !std::isfinite(pd.c))
            return fail(nullptr, TG_ERR_INVALID_ARG,
                        "TG_SENSOR_MARKERS needs pads_per_env >= 1, rows*cols <= 1024, radius <= 4, pitch, "
                        "lambda_d, eps > 0 and the pad_link / pad_frame arrays");
        if (pd.shear_points < 0 || pd.shear_points > 65536 ||
            (pd.shear_points > 0 && (!std::isfinite(pd.s_s) || !(pd.lambda_s >= 0.0) || !std::isfinite(pd.lambda_s) ||
                                     !(pd.eta_enter >= 0.0) || !(pd.eta_exit >= 0.0) || !std::isfinite(pd.eta_enter) ||
                                     !std::isfinite(pd.eta_exit) || !(pd.thickness > 0.0) || !std::isfinite(pd.thickness))))
            return fail(nullptr, TG_ERR_INVALID_ARG,
                        "shear anchors need shear_points in 0..65536, finite s_s, lambda_s >= 0, eta_enter and "
                        "eta_exit >= 0, thickness > 0");
        for (int i = 0; i < d->n_envs * pd.pads_per_env; ++i) {
            const int l = pd.pad_link[i];
            const int e = i / pd.pads_per_env;
            if (l < 0 || l >= d->max_links || d->link_rows[e * d->max_links + l] == 0)
                return fail(nullptr, TG_ERR_INVALID_ARG, "pad_link must name a present link of the env");
        }
    }

    // lattice table and work items
    std::vector<LinkLattice> lat((size_t)E * L);
    std::vector<Item> items;
    for (int e = 0; e < E; ++e) {
        int64_t acc = 0;
        for (int l = 0; l < L; ++l) {
            const int r = d->link_rows[e * L + l], c = d->link_cols[e * L + l];
            if (r < 0 || c < 0 || (r == 0) != (c == 0) || r > 65535 || c > 65535)
                return fail(nullptr, TG_ERR_INVALID_ARG, "link rows/cols must be both zero or both positive");
            const int64_t nl = (int64_t)r * c;
            if (nl > kItemCap)
                return fail(nullptr, TG_ERR_INVALID_ARG,
                            "a link lattice holds more taxels than tg_max_link_taxels()");
            LinkLattice& t = lat[(size_t)e * L + l];
            t.env_offset = (int32_t)acc;
            t.rows = (uint16_t)r;
            t.cols = (uint16_t)c;
            t.wrap = d->link_wrap ? (d->link_wrap[e * L + l] ? 1 : 0) : 0;
            t.present = nl > 0;
            acc += nl;
        }
        if (acc != d->taxel_offsets[e + 1] - d->taxel_offsets[e])
            return fail(nullptr, TG_ERR_INVALID_ARG, "sum of rows*cols over an env's links must equal its taxel count");
        // pack consecutive link slots into items of <= kItemCap taxels and <= 32 links
        int l = 0;
        while (l < L) {
            Item it{};
            it.env = e;
            it.link_begin = (int16_t)l;
            it.taxel_begin = d->taxel_offsets[e] + lat[(size_t)e * L + l].env_offset;
            int n = 0, k = 0;
            while (l < L && k < kItemMaxLinksHost) {
                const int nl = lat[(size_t)e * L + l].rows * lat[(size_t)e * L + l].cols;
                if (n + nl > kItemCap) break;
                n += nl;
                ++l;
                ++k;
            }
            it.link_end = (int16_t)l;
            it.n_taxels = n;
            if (n > 0) items.push_back(it);
        }
    }

    tg_scene* s = new tg_scene();
    s->E = E;
    s->L = L;
    s->T = T;
    s->sensors = d->sensors;
    s->gid0 = d->taxel_gid0;
    s->env_gid0 = d->env_gid0;
    s->params = d->params;
    s->P = P;
    s->items_h = items;
    s->n_items = (int)items.size();

    auto bail = [&](cudaError_t e, const char* what) {
        tg_status st = cuda_fail(nullptr, e, what);
        tg_destroy_scene(s);
        return st;
    };
#define CKC(call)                                   \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) return bail(_e, #call); \
    } while (0)

    const size_t EL = (size_t)E * L;
    // per-taxel arrays the pipelined step kernel bulk-copies carry 16 bytes
    // of slack: a copy runs to the 16-byte boundary at or past an item's end
    const size_t Tp = (size_t)T + 16;
    CKC(dalloc(&s->x, Tp)); CKC(dalloc(&s->y, Tp)); CKC(dalloc(&s->z, Tp));
    CKC(dalloc(&s->nx, Tp)); CKC(dalloc(&s->ny, Tp)); CKC(dalloc(&s->nz, Tp)); CKC(dalloc(&s->R, Tp));
    const float* src[7] = {d->x, d->y, d->z, d->nx, d->ny, d->nz, d->R};
    float* dst[7] = {s->x, s->y, s->z, s->nx, s->ny, s->nz, s->R};
    for (int i = 0; i < 7; ++i)
        if (T > 0) CKC(cudaMemcpy(dst[i], src[i], (size_t)T * sizeof(float), cudaMemcpyDefault));
    CKC(dalloc(&s->items, items.size()));
    if (!items.empty()) CKC(cudaMemcpy(s->items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice));
    CKC(dalloc(&s->lattice, EL));
    CKC(cudaMemcpy(s->lattice, lat.data(), EL * sizeof(LinkLattice), cudaMemcpyHostToDevice));
    CKC(dalloc(&s->flags, Tp));
    CKC(dalloc(&s->hyst_prev, (size_t)8 * T + 16));
    CKC(dalloc(&s->hyst_xi, (size_t)8 * T + 16));
    CKC(dalloc(&s->drift, (size_t)8 * T + 16));
    CKC(dalloc(&s->episode, E));
    if (P.ring_k > 1) {
        const size_t nr = (size_t)P.ring_k * 8 * T + 16;
        CKC(dalloc(&s->ring, nr));
        CKC(cudaMemset(s->ring, 0, nr * sizeof(float)));
    }
    CKC(dalloc(&s->depth_clean, T));
    CKC(dalloc(&s->depth_noisy, T));
    CKC(dalloc(&s->dist, (d->sensors & TG_SENSOR_DIST) ? T : 1));
    CKC(dalloc(&s->ft_clean, (size_t)6 * T));
    CKC(dalloc(&s->ft_noisy, (size_t)6 * T));
    CKC(dalloc(&s->link_out, EL * kLinkOut));
    CKC(dalloc(&s->link_count, EL * 2));
    CKC(dalloc(&s->err, 4));
    CKC(dalloc(&s->link_rec, EL * kLinkRec));
    for (int k = 0; k < 2; ++k) {
        CKC(dalloc(&s->s_link_pose[k], EL * 7));
        CKC(dalloc(&s->s_link_vel[k], EL * 6));
        CKC(dalloc(&s->s_obj_pose[k], (size_t)E * 7));
        CKC(dalloc(&s->s_obj_vel[k], (size_t)E * 6));
        CKC(dalloc(&s->s_env_params[k], (size_t)E * 3));
        CKC(dalloc(&s->s_obj_id[k], E));
        CKC(cudaEventCreateWithFlags(&s->staged_ev[k], cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&s->used_ev[k], cudaEventDisableTiming));
    }
    CKC(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&s->aux_stream, cudaStreamNonBlocking));
    CKC(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming));
    CKC(dalloc(&s->s_mask, E));
    CKC(dalloc(&s->s_contact, T));
    CKC(dalloc(&s->items_sorted, items.size()));
    {
        // static layout of every item for the pipelined schedules
        std::vector<ItemMeta> metas(items.size());
        for (size_t q = 0; q < items.size(); ++q) {
            const Item& it = items[q];
            ItemMeta& m = metas[q];
            std::memset(&m, 0, sizeof(m));
            m.nl = it.link_end - it.link_begin;
            const LinkLattice* ll = &lat[(size_t)it.env * L + it.link_begin];
            const int base = ll[0].env_offset;
            bool uni = true;
            for (int k = 0; k < m.nl; ++k) {
                m.start[k] = ll[k].env_offset - base;
                m.rows[k] = ll[k].rows;
                m.cols[k] = ll[k].cols;
                m.wrap[k] = ll[k].wrap;
                const int cnt = (k + 1 < m.nl ? ll[k + 1].env_offset - base : it.n_taxels) - m.start[k];
                uni = uni && ll[k].rows == ll[0].rows && ll[k].cols == ll[0].cols && ll[k].wrap == ll[0].wrap &&
                      cnt == ll[0].rows * ll[0].cols;
            }
            m.start[m.nl] = it.n_taxels;
            const int len = ll[0].rows * ll[0].cols;
            uni = uni && len > 0;
            // the same rule and the same FP32 reciprocals as the step kernel's prologue
            m.uni_len = uni ? len : 0;
            m.uni_rows = ll[0].rows;
            m.uni_cols = ll[0].cols;
            m.uni_wrap = ll[0].wrap;
            m.uni_inv_len = uni ? 1.0f / (float)len : 0.0f;
            m.uni_inv_cols = uni ? 1.0f / (float)ll[0].cols : 0.0f;
        }
        CKC(dalloc(&s->metas, metas.size()));
        if (!metas.empty())
            CKC(cudaMemcpy(s->metas, metas.data(), metas.size() * sizeof(ItemMeta), cudaMemcpyHostToDevice));
        CKC(dalloc(&s->slots, items.size()));
    }
    CKC(dalloc(&s->ctl, 1));
    CKC(cudaMemset(s->ctl, 0, sizeof(StepCtl)));
    CKC(configure_step_kernels());
    CKC(configure_pipe_kernels());
    {
        int dev = 0;
        CKC(cudaGetDevice(&dev));
        CKC(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev));
    }
    for (int k = 0; k < kStepShapes; ++k) {
        s->resident_ctas[k] = step_kernel_resident_ctas(k);
        if (s->resident_ctas[k] <= 0) return bail(cudaErrorInvalidConfiguration, "step kernel occupancy");
    }
    if (d->sensors & TG_SENSOR_PROX) {
        CKC(dalloc(&s->prox_clean, T));
        CKC(dalloc(&s->prox_noisy, T));
        CKC(cudaMemset(s->prox_clean, 0, (size_t)T * sizeof(float)));
        CKC(cudaMemset(s->prox_noisy, 0, (size_t)T * sizeof(float)));
    }
    if (d->sensors & TG_SENSOR_PCPROX) {
        CKC(dalloc(&s->pc_ft, (size_t)6 * std::max<int64_t>(T, 1)));
        CKC(cudaMemset(s->pc_ft, 0, (size_t)6 * std::max<int64_t>(T, 1) * sizeof(float)));
    }
    if (d->sensors & TG_SENSOR_MARKERS) {
        const size_t EP = (size_t)E * pd.pads_per_env, M = (size_t)pd.rows * pd.cols;
        CKC(dalloc(&s->pad_link, EP));
        CKC(dalloc(&s->pad_frame, EP * 9));
        CKC(dalloc(&s->marker_u, EP * M * 3));
        CKC(cudaMemcpy(s->pad_link, pd.pad_link, EP * sizeof(int32_t), cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(s->pad_frame, pd.pad_frame, EP * 9 * sizeof(float), cudaMemcpyHostToDevice));
        CKC(cudaMemset(s->marker_u, 0, EP * M * 3 * sizeof(float)));
        MarkerArgs& m = s->markers;
        m.n_envs = E;
        m.max_links = L;
        m.pads_per_env = pd.pads_per_env;
        m.rows = pd.rows;
        m.cols = pd.cols;
        m.radius = pd.radius;
        m.pitch = (float)pd.pitch;
        m.alpha = (float)pd.alpha;
        m.pad_link = s->pad_link;
        m.pad_frame = s->pad_frame;
        m.link_rec = s->link_rec;
        m.u = s->marker_u;
        m.err = s->err;
        if (pd.shear_points > 0) {
            CKC(dalloc(&s->anchors, EP * (size_t)pd.shear_points));
            CKC(dalloc(&s->anchor_obj, EP));
            CKC(dalloc(&s->n_anchored, EP));
            CKC(cudaMemset(s->anchor_obj, 0xff, EP * sizeof(int32_t)));  // -1: no anchors
            CKC(cudaMemset(s->n_anchored, 0, EP * sizeof(int32_t)));
            m.shear_n = pd.shear_points;
            m.s_s = (float)pd.s_s;
            m.lambda_s = (float)pd.lambda_s;
            m.eta_enter = (float)pd.eta_enter;
            m.eta_exit = (float)pd.eta_exit;
            m.half_t = (float)(0.5 * pd.thickness);
            m.anchors = s->anchors;
            m.anchor_obj = s->anchor_obj;
            m.n_anchored = s->n_anchored;
        }
        // per-offset weights: w_norm = s_d g(r), w_tan = s_d (c g / g_bar + (1 - c) rho / rho_bar)
        const double gbar = std::exp(-0.5) / std::sqrt(2.0 * pd.lambda_d), rbar = 1.0 / (2.0 * pd.eps);
        const int W = 2 * pd.radius + 1;
        for (int di = -pd.radius; di <= pd.radius; ++di)
            for (int dj = -pd.radius; dj <= pd.radius; ++dj) {
                const double r2 = (di * di + dj * dj) * pd.pitch * pd.pitch;
                const double g = std::exp(-pd.lambda_d * r2), rho = 1.0 / (r2 + pd.eps * pd.eps);
                const int w = (di + pd.radius) * W + (dj + pd.radius);
                m.w_norm[w] = (float)(pd.s_d * g);
                m.w_tan[w] = (float)(pd.s_d * (pd.c * g / gbar + (1.0 - pd.c) * rho / rbar));
            }
    }

    CKC(cudaMemset(s->link_out, 0, EL * kLinkOut * sizeof(float)));
    CKC(cudaMemset(s->link_count, 0, EL * 2 * sizeof(int32_t)));
    CKC(cudaMemset(s->err, 0, 4 * sizeof(unsigned)));
    CKC(cudaMemset(s->link_rec, 0, EL * kLinkRec * sizeof(float)));
    CKC(cudaMemset(s->hyst_prev, 0, (size_t)8 * T * sizeof(float)));
    CKC(cudaMemset(s->hyst_xi, 0, (size_t)8 * T * sizeof(float)));
    CKC(cudaMemset(s->drift, 0, (size_t)8 * T * sizeof(float)));
    CKC(cudaMemset(s->episode, 0, (size_t)E * sizeof(uint32_t)));
    CKC(cudaMemset(s->depth_clean, 0, (size_t)T * sizeof(float)));
    CKC(cudaMemset(s->depth_noisy, 0, (size_t)T * sizeof(float)));
    CKC(cudaMemset(s->ft_clean, 0, (size_t)6 * T * sizeof(float)));
    CKC(cudaMemset(s->ft_noisy, 0, (size_t)6 * T * sizeof(float)));
    CKC(launch_reset(step_args(s), s->n_items, nullptr, 0u, s->episode, 0));
    CKC(cudaDeviceSynchronize());
#undef CKC
    *out = s;
    return TG_OK;
}

void tg_destroy_scene(tg_scene* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->aux_stream) cudaStreamDestroy(s->aux_stream);
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    if (s->join_ev) cudaEventDestroy(s->join_ev);
    for (int k = 0; k < 2; ++k) {
        if (s->staged_ev[k]) cudaEventDestroy(s->staged_ev[k]);
        if (s->used_ev[k]) cudaEventDestroy(s->used_ev[k]);
        for (void* p : {(void*)s->s_link_pose[k], (void*)s->s_link_vel[k], (void*)s->s_obj_pose[k],
                        (void*)s->s_obj_vel[k], (void*)s->s_env_params[k], (void*)s->s_obj_id[k]})
            dfree(p);
    }
    for (cudaEvent_t e : s->graph_ev)
        if (e) cudaEventDestroy(e);
    free_objects(s);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : s->ev_pending) cudaEventDestroy(e);
    void* ptrs[] = {s->x, s->y, s->z, s->nx, s->ny, s->nz, s->R, s->items, s->lattice, s->flags, s->hyst_prev,
                    s->hyst_xi, s->drift, s->episode, s->depth_clean, s->depth_noisy, s->dist, s->ft_clean,
                    s->ft_noisy, s->link_out, s->link_count, s->err, s->link_rec, s->s_mask, s->s_contact,
                    s->items_sorted, s->metas, s->slots, s->prox_clean, s->prox_noisy, s->pad_link, s->pad_frame,
                    s->marker_u, s->ctl, s->nq_phi, s->nq_grad, s->nq_phi_lo, s->pc_ft, s->anchors, s->anchor_obj,
                    s->ring,
                    s->n_anchored};
    for (void* p : ptrs) dfree(p);
    delete s;
}

// An object's tracked points sorted into a uniform grid of cell size h over
// their box (counting sort on the host), uploaded as float4 points and cell
// start offsets; returns an error message or null.
static const char* load_cloud(const tg_object_desc& o, double h, ObjDev& t, std::vector<void*>& bufs) {
    const int64_t n = o.n_cloud;
    std::vector<float> pts((size_t)n * 3);
    if (cudaMemcpy(pts.data(), o.cloud, pts.size() * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        return "cloud copy failed";
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            const double v = pts[3 * i + a];
            if (!std::isfinite(v)) return "cloud points must be finite";
            lo[a] = std::min(lo[a], v);
            hi[a] = std::max(hi[a], v);
        }
    int dims[3];
    size_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        dims[a] = (int)std::floor((hi[a] - lo[a]) / h) + 1;
        cells *= (size_t)dims[a];
    }
    if (cells > ((size_t)1 << 22)) return "cloud box over 2^22 cells of pc_radius / 2";
    const float inv_h = (float)(1.0 / h);
    auto cell_of = [&](int64_t i) {
        int c[3];
        for (int a = 0; a < 3; ++a)
            c[a] = std::min(std::max((int)std::floor((pts[3 * i + a] - (float)lo[a]) * inv_h), 0), dims[a] - 1);
        return ((size_t)c[2] * dims[1] + c[1]) * dims[0] + c[0];
    };
    std::vector<int32_t> start(cells + 1, 0);
    for (int64_t i = 0; i < n; ++i) ++start[cell_of(i) + 1];
    for (size_t c = 0; c < cells; ++c) start[c + 1] += start[c];
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    std::vector<float4> sorted((size_t)n);
    for (int64_t i = 0; i < n; ++i) sorted[fill[cell_of(i)]++] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], 0.f);
    float4* dp = nullptr;
    int32_t* ds = nullptr;
    cudaError_t e1 = dalloc(&dp, (size_t)n), e2 = dalloc(&ds, cells + 1);
    if (dp) bufs.push_back(dp);
    if (ds) bufs.push_back(ds);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return "cloud alloc failed";
    if (cudaMemcpy(dp, sorted.data(), sizeof(float4) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ds, start.data(), sizeof(int32_t) * (cells + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        return "cloud upload failed";
    t.pc_pts = dp;
    t.pc_start = ds;
    for (int a = 0; a < 3; ++a) {
        t.pc_dims[a] = dims[a];
        t.pc_lo[a] = (float)lo[a];
    }
    t.pc_inv_h = inv_h;
    t.pc_n = (int32_t)n;
    return nullptr;
}

tg_status tg_upload_objects(tg_scene* s, const tg_object_desc* objs, int32_t n) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (!objs || n < 1) return fail(s, TG_ERR_INVALID_ARG, "need at least one object");
    std::vector<ObjDev> table(n);
    std::vector<void*> bufs;
    auto cleanup = [&]() {
        for (void* p : bufs) dfree(p);
    };
    std::vector<ObjInfo> info(n);
    for (int i = 0; i < n; ++i) info[i].kind = objs[i].kind;
    bool any_neural = false, any_raycast = false;
    // a grid (or a neural object's fallback grid): cell-major device copy
    auto load_grid = [&](const tg_object_desc& o, ObjDev& t) -> tg_status {
        size_t cnt = 1;
        for (int a = 0; a < 3; ++a) {
            if (o.dims[a] < 2 || !(o.hi[a] > o.lo[a]) || !std::isfinite(o.lo[a]) || !std::isfinite(o.hi[a]))
                return fail(s, TG_ERR_INVALID_ARG, "grid needs dims >= 2 and lo < hi on every axis");
            cnt *= (size_t)o.dims[a];
            t.dims[a] = o.dims[a];
            t.lo[a] = o.lo[a];
            t.hi[a] = o.hi[a];
            const double h = ((double)o.hi[a] - (double)o.lo[a]) / (double)(o.dims[a] - 1);
            const double ih = 1.0 / h;
            t.h[a] = (float)h;
            t.inv_h_hi[a] = (float)ih;
            t.inv_h_lo[a] = (float)(ih - (double)t.inv_h_hi[a]);
        }
        if (!o.values) return fail(s, TG_ERR_INVALID_ARG, "grid values are NULL");
        const size_t esz = o.fp16 ? 2 : 4;
        const size_t bytes = cnt * esz;
        const size_t ncell = (size_t)(o.dims[0] - 1) * (o.dims[1] - 1) * (o.dims[2] - 1);
        void *dv = nullptr, *dc = nullptr;
        cudaError_t e = cudaMalloc(&dv, bytes);
        if (e != cudaSuccess) return cuda_fail(s, e, "grid alloc");
        e = cudaMalloc(&dc, ncell * 8 * esz);
        if (e != cudaSuccess) {
            cudaFree(dv);
            return cuda_fail(s, e, "grid cell alloc");
        }
        bufs.push_back(dc);
        e = cudaMemcpy(dv, o.values, bytes, cudaMemcpyDefault);
        if (e == cudaSuccess) e = launch_build_cells(dv, o.dims, o.fp16 ? 1 : 0, dc, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(dv);  // queries read the cell-major copy only
        if (e != cudaSuccess) return cuda_fail(s, e, "grid copy");
        t.fp16 = o.fp16 ? 1 : 0;
        t.cells = dc;
        return TG_OK;
    };
    for (int i = 0; i < n; ++i) {
        const tg_object_desc& o = objs[i];
        ObjDev& t = table[i];
        t = ObjDev{};
        t.kind = o.kind;
        switch (o.kind) {
        case TG_OBJ_SPHERE:
            if (!(o.radius >= 0.0f) || !std::isfinite(o.radius)) { cleanup(); return fail(s, TG_ERR_INVALID_ARG, "sphere radius must be >= 0"); }
            t.radius = o.radius;
            break;
        case TG_OBJ_BOX:
            for (int a = 0; a < 3; ++a) {
                if (!(o.half[a] >= 0.0f) || !std::isfinite(o.half[a])) { cleanup(); return fail(s, TG_ERR_INVALID_ARG, "box half extents must be >= 0"); }
                t.half[a] = o.half[a];
            }
            break;
        case TG_OBJ_PLANE: break;
        case TG_OBJ_MESH: {
            std::vector<float> tri, trin;
            if (const char* m = build_triangles(o.verts, o.n_verts, o.faces, o.n_faces, &tri, &trin)) {
                cleanup();
                return fail(s, TG_ERR_INVALID_ARG, m);
            }
            float *dt = nullptr, *dn = nullptr;
            cudaError_t e1 = dalloc(&dt, tri.size()), e2 = dalloc(&dn, trin.size());
            if (dt) bufs.push_back(dt);
            if (dn) bufs.push_back(dn);
            if (e1 != cudaSuccess || e2 != cudaSuccess) { cleanup(); return cuda_fail(s, e1 != cudaSuccess ? e1 : e2, "mesh alloc"); }
            cudaMemcpy(dt, tri.data(), tri.size() * sizeof(float), cudaMemcpyHostToDevice);
            cudaMemcpy(dn, trin.data(), trin.size() * sizeof(float), cudaMemcpyHostToDevice);
            t.n_verts = o.n_verts;
            t.n_faces = o.n_faces;
            t.tri = dt;
            t.tri_n = dn;
            if (s->P.depth_backend == 1) {
                std::vector<float> hv;
                std::vector<int32_t> hf;
                if (!host_copy(o.verts, (size_t)o.n_verts * 3, &hv) || !host_copy(o.faces, (size_t)o.n_faces * 3, &hf)) {
                    cleanup();
                    return fail(s, TG_ERR_INVALID_ARG, "mesh copy failed");
                }
                if (const char* m = upload_mesh_bvh(hv.data(), o.n_verts, hf.data(), o.n_faces, &t, &bufs)) {
                    cleanup();
                    return fail(s, TG_ERR_INVALID_ARG, m);
                }
                any_raycast = true;
            }
            break;
        }
        case TG_OBJ_GRID:
            if (tg_status st = load_grid(o, t)) { cleanup(); return st; }
            break;
        case TG_OBJ_NEURAL: {
            if (!o.nsdf) { cleanup(); return fail(s, TG_ERR_INVALID_ARG, "neural object without a network"); }
            if (tg_status st = load_grid(o, t)) { cleanup(); return st; }  // the fallback
            const NsdfNet* net = nsdf_net(o.nsdf);
            const double smax = s->params.dr_on ? s->params.dr_scale[1] : 1.0;
            const double err = o.nsdf_err_mm;
            const bool use = err >= 0.0 && err * smax <= s->params.nsdf_max_err_mm;
            info[i].kind = use ? TG_OBJ_NEURAL : TG_OBJ_GRID;
            info[i].err_mm = err;
            if (!use) { t.kind = TG_OBJ_GRID; break; }
            uint32_t* tab = nullptr;
            uint16_t* w = nullptr;
            cudaError_t e1 = dalloc(&tab, (size_t)TG_NSDF_TABLE_ENTRIES), e2 = dalloc(&w, (size_t)TG_NSDF_WEIGHTS);
            if (tab) bufs.push_back(tab);
            if (w) bufs.push_back(w);
            if (e1 != cudaSuccess || e2 != cudaSuccess) { cleanup(); return cuda_fail(s, e1 != cudaSuccess ? e1 : e2, "network alloc"); }
            cudaError_t e = cudaDeviceSynchronize();  // the network may still be training on a stream
            if (e == cudaSuccess) e = cudaMemcpy(tab, net->table, sizeof(uint32_t) * TG_NSDF_TABLE_ENTRIES, cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(w, net->weights, sizeof(uint16_t) * TG_NSDF_WEIGHTS, cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) { cleanup(); return cuda_fail(s, e, "network copy"); }
            const ObjDev nd = nsdf_objdev(*net);
            for (int a = 0; a < 3; ++a) {
                t.nlo[a] = nd.nlo[a];
                t.nhi[a] = nd.nhi[a];
                t.ninv_ext[a] = nd.ninv_ext[a];
            }
            t.ntable = tab;
            t.nweights = w;
            any_neural = true;
            break;
        }
        default:
            cleanup();
            return fail(s, TG_ERR_INVALID_ARG, "unknown object kind");
        }
        if (o.n_cloud < 0 || o.n_cloud > (1 << 24) || (o.n_cloud > 0 && !o.cloud)) {
            cleanup();
            return fail(s, TG_ERR_INVALID_ARG, "n_cloud must be in 0..2^24 with a cloud");
        }
        if (s->markers.shear_n > 0 && o.n_cloud > s->markers.shear_n) {
            cleanup();
            return fail(s, TG_ERR_INVALID_ARG, "an object's n_cloud exceeds the pads' shear_points");
        }
        const bool pcprox = s->sensors & TG_SENSOR_PCPROX;
        if ((pcprox || s->markers.shear_n > 0) && o.n_cloud > 0) {
            // the cell grid serves the point-cloud proximity; the shear pass reads the points alone
            if (const char* m = load_cloud(o, pcprox ? 0.5 * s->params.pc_radius : 1e3, t, bufs)) {
                cleanup();
                return fail(s, TG_ERR_INVALID_ARG, m);
            }
        }
    }
    ObjDev* dtab = nullptr;
    cudaError_t e = dalloc(&dtab, (size_t)n);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(s, e, "object table alloc"); }
    cudaMemcpy(dtab, table.data(), sizeof(ObjDev) * n, cudaMemcpyHostToDevice);
    CK(s, cudaDeviceSynchronize());  // old objects may still be read by queued steps
    if ((any_neural || any_raycast) && !s->nq_phi) {
        cudaError_t ea = dalloc(&s->nq_phi, (size_t)std::max<int64_t>(s->T, 1));
        if (ea == cudaSuccess) ea = dalloc(&s->nq_grad, (size_t)3 * std::max<int64_t>(s->T, 1));
        if (ea != cudaSuccess) {
            dfree(dtab);
            cleanup();
            return cuda_fail(s, ea, "query scratch");
        }
    }
    if (any_raycast && !s->nq_phi_lo) {
        cudaError_t ea = dalloc(&s->nq_phi_lo, (size_t)std::max<int64_t>(s->T, 1));
        if (ea != cudaSuccess) {
            dfree(dtab);
            cleanup();
            return cuda_fail(s, ea, "query scratch");
        }
    }
    free_objects(s);
    s->objects = dtab;
    s->n_objects = n;
    s->obj_bufs = bufs;
    s->obj_info = info;
    s->any_neural = any_neural;
    s->any_raycast = any_raycast;
    s->all_grid = n > 0;
    for (int i = 0; i < n; ++i) s->all_grid = s->all_grid && objs[i].kind == TG_OBJ_GRID;
    return TG_OK;
}

tg_status tg_object_info(const tg_scene* s, int32_t i, int32_t* kind_used, double* nsdf_err_mm) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (i < 0 || i >= (int32_t)s->obj_info.size()) return TG_ERR_INVALID_ARG;
    if (kind_used) *kind_used = s->obj_info[i].kind;
    if (nsdf_err_mm) *nsdf_err_mm = s->obj_info[i].err_mm;
    return TG_OK;
}

tg_status tg_reset_envs(tg_scene* s, const uint8_t* env_mask, uint32_t episode, tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t* m = nullptr;
    if (env_mask) CK(s, stage(env_mask, s->s_mask, (size_t)s->E, st, &m));
    CK(s, launch_reset(step_args(s), s->n_items, m, episode, s->episode, st));
    if (s->anchor_obj) CK(s, launch_shear_reset(s->anchor_obj, s->E, s->markers.pads_per_env, m, st));
    return TG_OK;
}

namespace {

const char* check_inputs(const tg_scene* s, const tg_step_inputs* in) {
    if (!in || !in->link_pose || !in->link_vel || !in->obj_pose || !in->obj_vel || !in->obj_id)
        return "step inputs: link_pose, link_vel, obj_pose, obj_vel, obj_id are required";
    if (!std::isfinite(in->pose_dt)) return "pose_dt must be finite";
    if (s->P.dr_on && in->env_params) return "env_params must be NULL when domain randomisation is on";
    return nullptr;
}

// Every launch of one sensor step, in order, on `st`.  graph: the kernels
// take step and pose_dt from the device step control (and no profiling
// events are recorded), so the sequence can be captured and replayed.
tg_status enqueue_step(tg_scene* s, const tg_step_inputs* in, cudaStream_t st, bool graph) {
    const size_t EL = (size_t)s->E * s->L;
    PoseArgs pa{};
    // host inputs: outside a capture, copied on the copy stream into the
    // staging set the step before last used, then `st` waits for them
    const bool host_in = !(is_device_ptr(in->link_pose) && is_device_ptr(in->link_vel) &&
                           is_device_ptr(in->obj_pose) && is_device_ptr(in->obj_vel) &&
                           is_device_ptr(in->obj_id) && (!in->env_params || is_device_ptr(in->env_params)));
    const bool async_copy = host_in && !graph;
    const int b = async_copy ? s->next_set : 0;
    cudaStream_t cs = async_copy ? s->copy_stream : st;
    if (async_copy) {
        s->next_set ^= 1;
        if (s->used_rec[b]) CK(s, cudaStreamWaitEvent(cs, s->used_ev[b], 0));
    }
    CK(s, stage(in->link_pose, s->s_link_pose[b], EL * 7, cs, &pa.link_pose));
    CK(s, stage(in->link_vel, s->s_link_vel[b], EL * 6, cs, &pa.link_vel));
    CK(s, stage(in->obj_pose, s->s_obj_pose[b], (size_t)s->E * 7, cs, &pa.obj_pose));
    CK(s, stage(in->obj_vel, s->s_obj_vel[b], (size_t)s->E * 6, cs, &pa.obj_vel));
    pa.env_params = nullptr;
    if (in->env_params) CK(s, stage(in->env_params, s->s_env_params[b], (size_t)s->E * 3, cs, &pa.env_params));
    const int32_t* oid = nullptr;
    CK(s, stage(in->obj_id, s->s_obj_id[b], (size_t)s->E, cs, &oid));
    if (async_copy) {
        CK(s, cudaEventRecord(s->staged_ev[b], cs));
        CK(s, cudaStreamWaitEvent(st, s->staged_ev[b], 0));
    }
    pa.n_envs = s->E;
    pa.max_links = s->L;
    pa.lattice = s->lattice;
    pa.def_mu = (float)s->params.mu;
    pa.def_k = (float)s->params.k;
    pa.tau_hi = (float)in->pose_dt;
    pa.tau_lo = (float)(in->pose_dt - (double)pa.tau_hi);
    pa.link_rec = s->link_rec;
    pa.dr_on = s->P.dr_on;
    for (int i = 0; i < 3; ++i) {
        pa.dr_lo[i] = s->P.dr_lo[i];
        pa.dr_hi[i] = s->P.dr_hi[i];
    }
    pa.seed = s->P.seed;
    pa.env_gid0 = s->env_gid0;
    pa.step = in->step;
    pa.ctl = graph ? s->ctl : nullptr;
    // (in a capture the three events become event-record nodes that every
    // replay re-targets to fresh events, see tg_graph_launch)
    const bool prof = s->profiling;
    auto record = [&](cudaEvent_t e) {
        return graph ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
    };
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (prof) {
        for (int i = 0; i < 3; ++i) {
            if (s->ev_pool.empty()) {
                CK(s, cudaEventCreate(&ev[i]));
            } else {
                ev[i] = s->ev_pool.back();
                s->ev_pool.pop_back();
            }
            s->ev_pending.push_back(ev[i]);
        }
        CK(s, record(ev[0]));
    }
    StepArgs a = step_args(s);
    a.obj_id = oid;
    a.step = in->step;
    a.step_from_ctl = graph ? 1 : 0;
    a.items_sorted = nullptr;
    const bool pipe = sched_pipe(s->schedule);
    const bool sort = s->sorted && s->n_objects > 1 && s->n_objects <= 12288;
    // The order of the work items depends on the step's object ids only, so
    // its kernel (one CTA) runs on the auxiliary stream beside the pose
    // kernel and `st` waits for it before the first kernel that reads it.
    // (Under capture the event pair becomes a fork and a join of the graph.)
    const bool order = pipe || sort;
    if (order) {
        CK(s, cudaEventRecord(s->fork_ev, st));
        CK(s, cudaStreamWaitEvent(s->aux_stream, s->fork_ev, 0));
    }
    CK(s, launch_pose(pa, st));
    if (pipe) {
        CK(s, launch_slot_records(s->items, s->n_items, oid, s->n_objects, s->episode, sort ? 1 : 0, s->slots,
                                  s->aux_stream));
    } else if (sort) {
        CK(s, launch_order_items(s->items, s->n_items, oid, s->n_objects, s->items_sorted, s->aux_stream));
        a.items_sorted = s->items_sorted;
    }
    if (order) {
        CK(s, cudaEventRecord(s->join_ev, s->aux_stream));
        CK(s, cudaStreamWaitEvent(st, s->join_ev, 0));
    }
    if (prof) CK(s, record(ev[1]));
    if (s->any_neural) CK(s, launch_nsdf_step_query(a, s->n_items, s->nq_phi, s->nq_grad, st));
    if (s->any_raycast) CK(s, launch_raycast_step_query(a, s->n_items, s->nq_phi, s->nq_phi_lo, s->nq_grad, st));
    if (pipe) CK(s, launch_step_pipe(a, s->n_items, kPipeThreads[s->schedule - TG_SCHED_PIPE_1024], st));
    else CK(s, launch_step(a, s->n_items, st));
    if (prof) CK(s, record(ev[2]));
    if (s->sensors & TG_SENSOR_PROX) CK(s, launch_prox(a, s->n_items, s->sensor_threads[0], st));
    if (s->sensors & TG_SENSOR_PCPROX) CK(s, launch_pc_prox(a, s->n_items, s->sensor_threads[1], st));
    if (s->sensors & TG_SENSOR_MARKERS) {
        MarkerArgs m = s->markers;
        m.obj_id = oid;
        m.objects = s->objects;
        m.n_objects = s->n_objects;
        CK(s, launch_markers(m, s->sensor_threads[2], st));
    }
    if (graph) CK(s, launch_advance_ctl(s->ctl, st));
    if (async_copy) {  // the step's kernels are the last readers of staging set b
        CK(s, cudaEventRecord(s->used_ev[b], st));
        s->used_rec[b] = true;
    }
    return TG_OK;
}

StepCtl make_ctl(uint32_t step, double tau0, double dtau) {
    StepCtl c{};
    c.step = step;
    c.replay = 0;
    c.tau0_hi = (float)tau0;
    c.tau0_lo = (float)(tau0 - (double)c.tau0_hi);
    c.dtau_hi = (float)dtau;
    c.dtau_lo = (float)(dtau - (double)c.dtau_hi);
    return c;
}

void release_graph(tg_scene* s) {
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->graph_exec = nullptr;
    s->graph = nullptr;
    for (int k = 0; k < 3; ++k) {
        if (s->graph_ev[k]) s->ev_pool.push_back(s->graph_ev[k]);
        s->graph_ev[k] = nullptr;
        s->graph_ev_node[k] = nullptr;
    }
}

// the event-record nodes of a captured step, in the order of s->graph_ev
cudaError_t find_event_nodes(tg_scene* s) {
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(s->graph, nullptr, &n);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(n);
    e = cudaGraphGetNodes(s->graph, nodes.data(), &n);
    if (e != cudaSuccess) return e;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if ((e = cudaGraphNodeGetType(nd, &t)) != cudaSuccess) return e;
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        if ((e = cudaGraphEventRecordNodeGetEvent(nd, &ev)) != cudaSuccess) return e;
        for (int k = 0; k < 3; ++k)
            if (ev == s->graph_ev[k]) s->graph_ev_node[k] = nd;
    }
    for (int k = 0; k < 3; ++k)
        if (!s->graph_ev_node[k]) return cudaErrorInvalidValue;
    return cudaSuccess;
}

}  // namespace

tg_status tg_step_sensors(tg_scene* s, const tg_step_inputs* in, tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (const char* m = check_inputs(s, in)) return fail(s, TG_ERR_INVALID_ARG, m);
    if (s->n_objects < 1) return fail(s, TG_ERR_STATE, "tg_upload_objects must come before tg_step_sensors");
    // object indices passed in host memory are checked here, before anything
    // runs (device-resident indices are clamped by the kernels)
    if (!is_device_ptr(in->obj_id))
        for (int e = 0; e < s->E; ++e)
            if (in->obj_id[e] < 0 || in->obj_id[e] >= s->n_objects)
                return fail(s, TG_ERR_INVALID_ARG, "obj_id[" + std::to_string(e) + "] = " +
                                                       std::to_string(in->obj_id[e]) + " is not an uploaded object");
    return enqueue_step(s, in, (cudaStream_t)stream, false);
}

tg_status tg_graph_capture(tg_scene* s, const tg_step_inputs* in, double pose_dt_per_step, tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (const char* m = check_inputs(s, in)) return fail(s, TG_ERR_INVALID_ARG, m);
    if (!std::isfinite(pose_dt_per_step)) return fail(s, TG_ERR_INVALID_ARG, "pose_dt_per_step must be finite");
    if (s->n_objects < 1) return fail(s, TG_ERR_STATE, "tg_upload_objects must come before tg_graph_capture");
    const void* ptrs[] = {in->link_pose, in->link_vel, in->obj_pose, in->obj_vel, in->obj_id, in->env_params};
    for (const void* p : ptrs)
        if (p && !is_device_ptr(p))
            return fail(s, TG_ERR_INVALID_ARG, "a captured step reads its inputs in place: device pointers only");
    release_graph(s);
    if (!s->cap_stream) CK(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
    cudaStream_t st = (cudaStream_t)stream;
    CK(s, launch_set_ctl(s->ctl, make_ctl(in->step, in->pose_dt, pose_dt_per_step), st));
    CK(s, cudaStreamSynchronize(st));
    CK(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    const size_t pending = s->ev_pending.size();
    const tg_status r = enqueue_step(s, in, s->cap_stream, true);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s->cap_stream, &g);
    if (s->ev_pending.size() == pending + 3) {
        // the capture's timing events belong to the graph, not to a step
        for (int k = 0; k < 3; ++k) s->graph_ev[k] = s->ev_pending[pending + k];
        s->ev_pending.resize(pending);
    }
    if (r != TG_OK) {
        if (g) cudaGraphDestroy(g);
        release_graph(s);
        return r;
    }
    if (ec != cudaSuccess) {
        release_graph(s);
        return cuda_fail(s, ec, "graph capture");
    }
    s->graph = g;
    if (s->graph_ev[0]) {
        const cudaError_t en = find_event_nodes(s);
        if (en != cudaSuccess) {
            release_graph(s);
            return cuda_fail(s, en, "graph timing nodes");
        }
    }
    const cudaError_t ei = cudaGraphInstantiate(&s->graph_exec, g, 0);
    if (ei != cudaSuccess) {
        release_graph(s);
        return cuda_fail(s, ei, "graph instantiate");
    }
    return TG_OK;
}

tg_status tg_graph_launch(tg_scene* s, int32_t n_steps, tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (!s->graph_exec) return fail(s, TG_ERR_STATE, "no captured step: call tg_graph_capture first");
    if (n_steps < 0) return fail(s, TG_ERR_INVALID_ARG, "n_steps must be >= 0");
    for (int32_t i = 0; i < n_steps; ++i) {
        if (s->profiling && s->graph_ev_node[0]) {
            // this replay records into its own events (earlier replays keep theirs)
            for (int k = 0; k < 3; ++k) {
                cudaEvent_t ev = nullptr;
                if (s->ev_pool.empty()) {
                    CK(s, cudaEventCreate(&ev));
                } else {
                    ev = s->ev_pool.back();
                    s->ev_pool.pop_back();
                }
                s->ev_pending.push_back(ev);
                CK(s, cudaGraphExecEventRecordNodeSetEvent(s->graph_exec, s->graph_ev_node[k], ev));
            }
        }
        CK(s, cudaGraphLaunch(s->graph_exec, (cudaStream_t)stream));
    }
    return TG_OK;
}

tg_status tg_graph_seek(tg_scene* s, uint32_t step, double pose_dt, double pose_dt_per_step, tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (!std::isfinite(pose_dt) || !std::isfinite(pose_dt_per_step))
        return fail(s, TG_ERR_INVALID_ARG, "pose_dt and pose_dt_per_step must be finite");
    CK(s, launch_set_ctl(s->ctl, make_ctl(step, pose_dt, pose_dt_per_step), (cudaStream_t)stream));
    return TG_OK;
}

tg_status tg_graph_release(tg_scene* s) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    CK(s, cudaDeviceSynchronize());
    release_graph(s);
    return TG_OK;
}

tg_status tg_set_schedule(tg_scene* s, int32_t schedule, int32_t sorted) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (s->graph_exec) return fail(s, TG_ERR_STATE, "release the captured step before changing the schedule");
    if (schedule < 0 || schedule >= TG_SCHED_COUNT) return fail(s, TG_ERR_INVALID_ARG, "unknown schedule");
    s->schedule = schedule;
    s->sorted = sorted != 0;
    return TG_OK;
}

tg_status tg_get_schedule(const tg_scene* s, int32_t* schedule, int32_t* sorted) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (schedule) *schedule = s->schedule;
    if (sorted) *sorted = s->sorted;
    return TG_OK;
}

namespace {
bool sensor_threads_ok(int32_t t) { return t == 128 || t == 256 || t == 512; }
// the sensor kernels a scene runs (tg_sensor_kernel order)
bool sensor_kernel_on(const tg_scene* s, int k) {
    if (k == 0) return (s->sensors & TG_SENSOR_PROX) && s->P.prox_rays > 0;
    if (k == 1) return (s->sensors & TG_SENSOR_PCPROX) != 0;
    return (s->sensors & TG_SENSOR_MARKERS) != 0;
}
int step_threads(int schedule) {
    return sched_pipe(schedule) ? kPipeThreads[schedule - TG_SCHED_PIPE_1024] : kStepShapeThreads[sched_shape(schedule)];
}
}  // namespace

tg_status tg_set_sensor_threads(tg_scene* s, int32_t kernel, int32_t threads) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (s->graph_exec) return fail(s, TG_ERR_STATE, "release the captured step before changing a launch shape");
    if (kernel < 0 || kernel >= TG_SENSOR_KERNEL_COUNT) return fail(s, TG_ERR_INVALID_ARG, "unknown sensor kernel");
    if (!sensor_threads_ok(threads)) return fail(s, TG_ERR_INVALID_ARG, "threads must be 128, 256 or 512");
    s->sensor_threads[kernel] = threads;
    return TG_OK;
}

tg_status tg_get_sensor_threads(const tg_scene* s, int32_t kernel, int32_t* threads) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (kernel < 0 || kernel >= TG_SENSOR_KERNEL_COUNT) return fail(nullptr, TG_ERR_INVALID_ARG, "unknown sensor kernel");
    if (threads) *threads = s->sensor_threads[kernel];
    return TG_OK;
}

tg_status tg_autotune(tg_scene* s, const tg_step_inputs* in, int32_t steps, tg_tune_report* report,
                      tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (const char* m = check_inputs(s, in)) return fail(s, TG_ERR_INVALID_ARG, m);
    if (s->n_objects < 1) return fail(s, TG_ERR_STATE, "tg_upload_objects must come before tg_autotune");
    if (steps < 1 || steps > 1000) return fail(s, TG_ERR_INVALID_ARG, "steps must be in 1..1000");
    if (s->graph_exec) return fail(s, TG_ERR_STATE, "release the captured step before tuning");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t T = (size_t)s->T, E = (size_t)s->E;
    // the noise state is put back afterwards: trials are not steps of the run
    uint8_t* keep = nullptr;
    const size_t RB = s->ring ? (size_t)s->P.ring_k * 8 * T * 4 : 0;
    // the shear anchors are state of the markers' trials too
    const size_t EP = s->anchors ? (size_t)s->E * s->markers.pads_per_env : 0;
    const size_t AB = EP * (size_t)s->markers.shear_n * 8;
    // (and the clean depth and force/torque outputs, which with prev_out are
    // the hysteresis x_{t-1})
    const size_t bytes = T + 3 * 8 * T * 4 + 7 * T * 4 + E * 4 + RB + AB + 2 * EP * 4;
    CK(s, cudaMalloc(&keep, bytes));
    auto save = [&](bool back) {
        struct { void* p; size_t n; } part[] = {{s->flags, T}, {s->hyst_prev, 8 * T * 4}, {s->hyst_xi, 8 * T * 4},
                                                 {s->drift, 8 * T * 4}, {s->depth_clean, T * 4},
                                                 {s->ft_clean, 6 * T * 4}, {s->episode, E * 4}, {s->ring, RB},
                                                 {s->anchors, AB}, {s->anchor_obj, EP * 4}, {s->n_anchored, EP * 4}};
        size_t off = 0;
        cudaError_t e = cudaSuccess;
        for (auto& q : part) {
            if (q.n == 0) continue;
            if (e == cudaSuccess)
                e = back ? cudaMemcpyAsync(q.p, keep + off, q.n, cudaMemcpyDeviceToDevice, st)
                         : cudaMemcpyAsync(keep + off, q.p, q.n, cudaMemcpyDeviceToDevice, st);
            off += q.n;
        }
        return e;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tg_tune_report rep{};
    for (int k = 0; k < TG_SENSOR_KERNEL_COUNT; ++k) rep.sensor_chosen[k] = -1;
    const int old_p = s->schedule, old_s = s->sorted;
    const bool prof = s->profiling;
    s->profiling = false;
    cudaError_t err = save(false);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    tg_status r = TG_OK;
    const int old_threads[3] = {s->sensor_threads[0], s->sensor_threads[1], s->sensor_threads[2]};
    // one variant: a warm-up step, then `steps` timed steps; false on failure
    auto time_variant = [&](int kernel, int threads) {
        r = enqueue_step(s, in, st, false);
        if (r != TG_OK) return false;
        err = cudaEventRecord(e0, st);
        for (int k = 0; k < steps && r == TG_OK && err == cudaSuccess; ++k) r = enqueue_step(s, in, st, false);
        if (r != TG_OK || err != cudaSuccess) return false;
        err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess || rep.n >= (int)(sizeof(rep.cand) / sizeof(rep.cand[0]))) return false;
        tg_tune_candidate& c = rep.cand[rep.n++];
        c.schedule = s->schedule;
        c.sorted = s->sorted;
        c.ms_per_step = (double)ms / steps;
        c.kernel = kernel;
        c.threads = threads;
        return true;
    };
    // the step kernel's schedules first
    const int sort_options = s->n_objects > 1 ? 2 : 1;
    bool ok = err == cudaSuccess;
    for (int ps = 0; ps < TG_SCHED_COUNT && ok; ++ps)
        for (int so = 0; so < sort_options && ok; ++so) {
            s->schedule = ps;
            s->sorted = sort_options == 2 ? 1 - so : s->sorted;
            ok = time_variant(-1, step_threads(ps));
        }
    int best = 0;
    if (ok) {
        for (int i = 1; i < rep.n; ++i)
            if (rep.cand[i].ms_per_step < rep.cand[best].ms_per_step) best = i;
        s->schedule = rep.cand[best].schedule;
        s->sorted = rep.cand[best].sorted;
    }
    // then each sensor kernel's launch shape, on the chosen schedule
    for (int k = 0; k < TG_SENSOR_KERNEL_COUNT && ok; ++k) {
        if (!sensor_kernel_on(s, k)) continue;
        const int first = rep.n;
        for (int t : {128, 256, 512}) {
            s->sensor_threads[k] = t;
            if (!(ok = time_variant(k, t))) break;
        }
        if (!ok) break;
        int kb = first;
        for (int i = first + 1; i < rep.n; ++i)
            if (rep.cand[i].ms_per_step < rep.cand[kb].ms_per_step) kb = i;
        s->sensor_threads[k] = rep.cand[kb].threads;
        rep.sensor_chosen[k] = kb;
    }
    if (ok) err = save(true);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    s->profiling = prof;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(keep);
    if (!ok || r != TG_OK || err != cudaSuccess || rep.n == 0) {
        s->schedule = old_p;
        s->sorted = old_s;
        for (int k = 0; k < 3; ++k) s->sensor_threads[k] = old_threads[k];
        if (r != TG_OK) return r;
        return cuda_fail(s, err == cudaSuccess ? cudaErrorUnknown : err, "autotune");
    }
    rep.chosen = best;
    if (report) *report = rep;
    return TG_OK;
}

tg_status tg_profile_enable(tg_scene* s, int32_t on) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    s->profiling = on != 0;
    return TG_OK;
}

tg_status tg_profile_read(tg_scene* s, double* pose_ms, double* step_ms, int64_t* n_steps) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    double tp = 0.0, ts = 0.0;
    const size_t n = s->ev_pending.size() / 3;
    for (size_t i = 0; i < n; ++i) {
        cudaEvent_t* e = &s->ev_pending[3 * i];
        CK(s, cudaEventSynchronize(e[2]));
        float a = 0.f, b = 0.f;
        CK(s, cudaEventElapsedTime(&a, e[0], e[1]));
        CK(s, cudaEventElapsedTime(&b, e[1], e[2]));
        tp += a;
        ts += b;
    }
    for (cudaEvent_t e : s->ev_pending) s->ev_pool.push_back(e);
    s->ev_pending.clear();
    if (pose_ms) *pose_ms = tp;
    if (step_ms) *step_ms = ts;
    if (n_steps) *n_steps = (int64_t)n;
    return TG_OK;
}

size_t tg_channel_bytes(const tg_scene* s, int32_t ch) {
    if (!s) return 0;
    const size_t T = (size_t)s->T, EL = (size_t)s->E * s->L;
    switch (ch) {
    case TG_CH_CONTACT: return T;
    case TG_CH_DEPTH: return T * 4;
    case TG_CH_DIST: return (s->sensors & TG_SENSOR_DIST) ? T * 4 : 0;
    case TG_CH_FORCE_TORQUE: return T * 24;
    case TG_CH_LINK_WRENCH: return EL * kLinkOut * 4;
    case TG_CH_LINK_COUNT: return EL * 8;
    case TG_CH_STATE_FLAGS: return T;
    case TG_CH_PROX: return (s->sensors & TG_SENSOR_PROX) ? T * 4 : 0;
    case TG_CH_MARKER:
        return (s->sensors & TG_SENSOR_MARKERS)
                   ? (size_t)s->E * s->markers.pads_per_env * s->markers.rows * s->markers.cols * 12
                   : 0;
    case TG_CH_PC_FT: return (s->sensors & TG_SENSOR_PCPROX) ? T * 24 : 0;
    case TG_CH_SHEAR_ANCHORS: return s->n_anchored ? (size_t)s->E * s->markers.pads_per_env * 4 : 0;
    default: return 0;
    }
}

tg_status tg_get_buffer(tg_scene* s, int32_t ch, int32_t noisy, void** ptr, size_t* bytes) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    if (!ptr) return fail(s, TG_ERR_INVALID_ARG, "ptr is NULL");
    void* p = nullptr;
    switch (ch) {
    case TG_CH_DEPTH: p = noisy ? s->depth_noisy : s->depth_clean; break;
    case TG_CH_DIST: p = (s->sensors & TG_SENSOR_DIST) ? s->dist : nullptr; break;
    case TG_CH_FORCE_TORQUE: p = noisy ? s->ft_noisy : s->ft_clean; break;
    case TG_CH_LINK_WRENCH: p = s->link_out; break;
    case TG_CH_LINK_COUNT: p = s->link_count; break;
    case TG_CH_STATE_FLAGS: p = s->flags; break;
    case TG_CH_PROX: p = (s->sensors & TG_SENSOR_PROX) ? (noisy ? s->prox_noisy : s->prox_clean) : nullptr; break;
    case TG_CH_MARKER: p = (s->sensors & TG_SENSOR_MARKERS) ? s->marker_u : nullptr; break;
    case TG_CH_PC_FT: p = (s->sensors & TG_SENSOR_PCPROX) ? s->pc_ft : nullptr; break;
    case TG_CH_SHEAR_ANCHORS: p = s->n_anchored; break;
    default: break;
    }
    if (!p) return fail(s, TG_ERR_INVALID_ARG, "channel has no device view (or its sensor is off)");
    *ptr = p;
    if (bytes) *bytes = tg_channel_bytes(s, ch);
    return TG_OK;
}

tg_status tg_read_taxels(tg_scene* s, int32_t ch, int32_t noisy, void* dst, size_t dst_bytes, tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    const size_t need = tg_channel_bytes(s, ch);
    if (need == 0) return fail(s, TG_ERR_INVALID_ARG, "unknown channel or sensor not enabled");
    if (!dst || dst_bytes != need) return fail(s, TG_ERR_INVALID_ARG, "dst is NULL or dst_bytes != tg_channel_bytes");
    cudaStream_t st = (cudaStream_t)stream;
    if (ch == TG_CH_CONTACT) {
        if (is_device_ptr(dst)) {
            CK(s, launch_unpack_contact(s->flags, s->T, noisy ? (s->P.ring_k > 1 ? 3 : 2) : 0, (uint8_t*)dst, st));
        } else {
            CK(s, launch_unpack_contact(s->flags, s->T, noisy ? (s->P.ring_k > 1 ? 3 : 2) : 0, s->s_contact, st));
            CK(s, cudaMemcpyAsync(dst, s->s_contact, need, cudaMemcpyDeviceToHost, st));
        }
        return TG_OK;
    }
    void* p = nullptr;
    tg_status r = tg_get_buffer(s, ch, noisy, &p, nullptr);
    if (r != TG_OK) return r;
    CK(s, cudaMemcpyAsync(dst, p, need, cudaMemcpyDefault, st));
    return TG_OK;
}

tg_status tg_sync(tg_scene* s, tg_stream stream) {
    if (!s) return fail(nullptr, TG_ERR_INVALID_ARG, "scene is NULL");
    CK(s, cudaStreamSynchronize((cudaStream_t)stream));
    CK(s, cudaGetLastError());
    unsigned h[4] = {0, 0, 0, 0};
    CK(s, cudaMemcpy(h, s->err, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[0] || h[1] || h[2]) {
        CK(s, cudaMemset(s->err, 0, sizeof(h)));
        if (h[2])
            return fail(s, TG_ERR_TIMEOUT, "a bulk copy of the pipelined step kernel did not complete in time (" +
                                               std::to_string(h[2]) + " CTAs stopped)");
        if (h[1])
            return fail(s, TG_ERR_TIMEOUT, "a tensor-core MMA of the learned-SDF query did not complete in time (" +
                                               std::to_string(h[1]) + " work items skipped)");
        return fail(s, TG_ERR_NUMERIC, "non-finite signed distances were seen (" + std::to_string(h[0]) + " taxel queries)");
    }
    return TG_OK;
}

const char* tg_last_error(const tg_scene* s) { return s ? s->last_error.c_str() : g_create_error.c_str(); }

static const uint64_t kStateMagic = 0x3130455441545354ull;  // "TSTATE01"
// with prev_out the hysteresis x_{t-1} of channels 0-6 is stored as the clean
// outputs (not gain times them): such checkpoints carry their own tag, so
// that one of the other form is refused rather than misread
static const uint64_t kStateMagicOut = 0x3230455441545354ull;  // "TSTATE02"
static uint64_t state_magic(const tg_scene* s) { return s->P.prev_out ? kStateMagicOut : kStateMagic; }

// shear anchor slots of the scene (0 when the shear anchors are off)
static size_t shear_slots(const tg_scene* s) {
    return s->anchors ? (size_t)s->E * s->markers.pads_per_env * s->markers.shear_n : 0;
}

// where channel c of the hysteresis x_{t-1} lives: hyst_prev, or with
// prev_out (channels 0-6) the clean depth and force/torque outputs
static float* prev_channel(tg_scene* s, int c) {
    const size_t T = (size_t)s->T;
    if (s->P.prev_out && c < 7) return c == 0 ? s->depth_clean : s->ft_clean + (size_t)(c - 1) * T;
    return s->hyst_prev + (size_t)c * T;
}

tg_status tg_save_state(tg_scene* s, void* buf, size_t* size) {
    if (!s || !size) return fail(s, TG_ERR_INVALID_ARG, "scene or size is NULL");
    const size_t T = (size_t)s->T, E = (size_t)s->E;
    const size_t A = shear_slots(s), EP = A ? E * s->markers.pads_per_env : 0;
    const size_t RB = s->ring ? (size_t)s->P.ring_k * 8 * T * 4 : 0;
    const size_t need = 32 + T + 3 * 8 * T * 4 + E * 4 + A * 8 + EP * 4 + RB;
    if (!buf) { *size = need; return TG_OK; }
    if (*size != need) return fail(s, TG_ERR_INVALID_ARG, "state buffer size mismatch");
    CK(s, cudaDeviceSynchronize());
    unsigned char* p = (unsigned char*)buf;
    uint64_t hdr[4] = {state_magic(s), (uint64_t)T, (uint64_t)E, (uint64_t)A};
    memcpy(p, hdr, 32);
    p += 32;
    CK(s, cudaMemcpy(p, s->flags, T, cudaMemcpyDeviceToHost)); p += T;
    // hysteresis x_{t-1} per channel; with prev_out channels 0-6 are the
    // clean depth and force/torque outputs
    for (int c = 0; c < 8; ++c, p += T * 4)
        CK(s, cudaMemcpy(p, prev_channel(s, c), T * 4, cudaMemcpyDeviceToHost));
    CK(s, cudaMemcpy(p, s->hyst_xi, 8 * T * 4, cudaMemcpyDeviceToHost)); p += 8 * T * 4;
    CK(s, cudaMemcpy(p, s->drift, 8 * T * 4, cudaMemcpyDeviceToHost)); p += 8 * T * 4;
    CK(s, cudaMemcpy(p, s->episode, E * 4, cudaMemcpyDeviceToHost)); p += E * 4;
    if (A) {
        CK(s, cudaMemcpy(p, s->anchors, A * 8, cudaMemcpyDeviceToHost)); p += A * 8;
        CK(s, cudaMemcpy(p, s->anchor_obj, EP * 4, cudaMemcpyDeviceToHost)); p += EP * 4;
    }
    if (RB) CK(s, cudaMemcpy(p, s->ring, RB, cudaMemcpyDeviceToHost));
    return TG_OK;
}

tg_status tg_load_state(tg_scene* s, const void* buf, size_t size) {
    if (!s || !buf) return fail(s, TG_ERR_INVALID_ARG, "scene or buf is NULL");
    const size_t T = (size_t)s->T, E = (size_t)s->E;
    const size_t A = shear_slots(s), EP = A ? E * s->markers.pads_per_env : 0;
    const size_t RB = s->ring ? (size_t)s->P.ring_k * 8 * T * 4 : 0;
    const size_t need = 32 + T + 3 * 8 * T * 4 + E * 4 + A * 8 + EP * 4 + RB;
    if (size != need) return fail(s, TG_ERR_INVALID_ARG, "state buffer size mismatch");
    const unsigned char* p = (const unsigned char*)buf;
    uint64_t hdr[4];
    memcpy(hdr, p, 32);
    if (hdr[0] != state_magic(s) || hdr[1] != T || hdr[2] != E || hdr[3] != A) return fail(s, TG_ERR_INVALID_ARG, "state buffer is not from a scene of this shape");
    p += 32;
    CK(s, cudaDeviceSynchronize());
    CK(s, cudaMemcpy(s->flags, p, T, cudaMemcpyHostToDevice)); p += T;
    for (int c = 0; c < 8; ++c, p += T * 4)
        CK(s, cudaMemcpy(prev_channel(s, c), p, T * 4, cudaMemcpyHostToDevice));
    CK(s, cudaMemcpy(s->hyst_xi, p, 8 * T * 4, cudaMemcpyHostToDevice)); p += 8 * T * 4;
    CK(s, cudaMemcpy(s->drift, p, 8 * T * 4, cudaMemcpyHostToDevice)); p += 8 * T * 4;
    CK(s, cudaMemcpy(s->episode, p, E * 4, cudaMemcpyHostToDevice)); p += E * 4;
    if (A) {
        CK(s, cudaMemcpy(s->anchors, p, A * 8, cudaMemcpyHostToDevice)); p += A * 8;
        CK(s, cudaMemcpy(s->anchor_obj, p, EP * 4, cudaMemcpyHostToDevice)); p += EP * 4;
    }
    if (RB) CK(s, cudaMemcpy(s->ring, p, RB, cudaMemcpyHostToDevice));
    return TG_OK;
}

static tg_status mesh_common(const float* verts, int32_t nv, const int32_t* faces, int32_t nf, cudaStream_t st,
                             float** tri, float** trin) {
    std::vector<float> t, tn;
    if (const char* m = build_triangles(verts, nv, faces, nf, &t, &tn)) return fail(nullptr, TG_ERR_INVALID_ARG, m);
    cudaError_t e = cudaMallocAsync((void**)tri, t.size() * sizeof(float), st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "mesh alloc");
    e = cudaMallocAsync((void**)trin, tn.size() * sizeof(float), st);
    if (e != cudaSuccess) { cudaFreeAsync(*tri, st); return cuda_fail(nullptr, e, "mesh alloc"); }
    cudaMemcpyAsync(*tri, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(*trin, tn.data(), tn.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    e = cudaStreamSynchronize(st);  // the host vectors die at return
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "mesh upload");
    return TG_OK;
}

tg_status tg_bake_grid(const float* verts, int32_t nv, const int32_t* faces, int32_t nf, const int32_t dims[3],
                       const float lo[3], const float hi[3], int32_t fp16, void* out, tg_stream stream) {
    if (!dims || !lo || !hi || !out) return fail(nullptr, TG_ERR_INVALID_ARG, "dims, lo, hi and out are required");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || !(hi[a] > lo[a])) return fail(nullptr, TG_ERR_INVALID_ARG, "grid needs dims >= 2 and lo < hi");
    if (!is_device_ptr(out)) return fail(nullptr, TG_ERR_INVALID_ARG, "out must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    float *tri = nullptr, *trin = nullptr;
    tg_status r = mesh_common(verts, nv, faces, nf, st, &tri, &trin);
    if (r != TG_OK) return r;
    int d3[3] = {dims[0], dims[1], dims[2]};
    cudaError_t e = launch_mesh_bake(tri, trin, nf, d3, lo, hi, fp16, out, st);
    cudaFreeAsync(tri, st);
    cudaFreeAsync(trin, st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bake launch");
    return TG_OK;
}

tg_status tg_mesh_sdf(const float* verts, int32_t nv, const int32_t* faces, int32_t nf, const float* points, int64_t n,
                      float* phi, float* grad, tg_stream stream) {
    if (n < 0 || (n > 0 && (!points || !phi))) return fail(nullptr, TG_ERR_INVALID_ARG, "points and phi are required");
    if (n > 0 && (!is_device_ptr(points) || !is_device_ptr(phi) || (grad && !is_device_ptr(grad))))
        return fail(nullptr, TG_ERR_INVALID_ARG, "points, phi and grad must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    float *tri = nullptr, *trin = nullptr;
    tg_status r = mesh_common(verts, nv, faces, nf, st, &tri, &trin);
    if (r != TG_OK) return r;
    cudaError_t e = launch_mesh_sdf_points(tri, trin, nf, points, n, phi, grad, st);
    cudaFreeAsync(tri, st);
    cudaFreeAsync(trin, st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "mesh sdf launch");
    return TG_OK;
}

}  // extern "C"
