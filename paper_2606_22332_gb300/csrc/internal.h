// internal.h -- device-side data layout of a scene and the launch wrappers
// shared by the translation units of libtg.so.  Not part of the C-ABI.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/tg.h"

namespace tg {

// Index of a taxel in the scene's per-taxel arrays.  A scene holds fewer
// than 2^31 taxels, so the step kernels index with 32 bits: an address is
// then one wide multiply-add on the array's (uniform) base.
using tidx = uint32_t;
constexpr int64_t kMaxSceneTaxels = (int64_t)1 << 31;

constexpr int kMaxLinks = 255;       // u8 link ids
constexpr int kItemCap = 1024;       // max taxels per work item (one CTA)
// CTA shapes of the step kernel: threads per CTA and the resident CTAs per
// SM its register budget is set for (512 x 2, or 384 x 3 at 56 registers;
// one item's shared memory, ~75 KB, lets three CTAs share an SM)
constexpr int kStepShapes = 2;
constexpr int kStepShapeThreads[kStepShapes] = {512, 384};
constexpr int kStepShapeBlocks[kStepShapes] = {2, 3};
constexpr int kLinkRec = 40;         // floats per (env, link) pose record
constexpr int kLinkOut = 18;         // floats per (env, link) output record
constexpr int kItemMaxLinks = 32;    // links per work item

// Step control in device memory.  Direct steps pass step and pose_dt as
// kernel arguments; a captured CUDA graph reads them from here instead and
// its last node advances them, so replays need no host work:
// replay r of a graph captured at (step0, tau0) runs step0 + r with
// pose_dt = tau0 + r dtau.  `counter` is the persistent step kernel's work
// counter, zeroed before every step.
struct StepCtl {
    uint32_t step;
    uint32_t replay;
    float tau0_hi, tau0_lo, dtau_hi, dtau_lo;
    uint32_t counter;
    uint32_t pad;
};

// A noise group with the host-derived constants the kernel uses.
struct NoiseDev {
    float gain_lo, gain_span;    // gain = lo + span * u
    float beta, decay;           // decay = exp(-dt / tau)
    float bias, sigma_white, sigma_rw, quant;
    float stuck_lo, stuck_span;
    int gain_on;
};

struct ParamsDev {
    float k, c, alpha, k_t, k_omega, mu;  // mu < 0: no clamp
    float eta_on_hi, eta_on_lo, eta_off_hi, eta_off_lo;  // thresholds as float pairs
    uint32_t dead_threshold24;            // rint(p_dead * 2^24)
    float chi;
    float xt_w[9];                        // L1-normalised 3x3 Gaussian, row-major
    uint64_t seed;
    uint32_t rk[20];                  // Philox round keys of the seed: (k0, k1) + r (0x9E3779B9, 0xBB67AE85)
    float rho;                        // probe-radius noise half-width (m), 0 = off
    float pc_radius, pc_k, pc_ks, pc_density;  // point-cloud proximity
    NoiseDev depth, ft, prox;
    // proximity rays
    int prox_rays;
    float prox_range, prox_cos, prox_sin;
    float prox_az_cos[16], prox_az_sin[16];
    // per-step domain randomisation of (mu, k, scale)
    int dr_on;
    float dr_lo[3], dr_hi[3];
    // read delay of the noisy readout (steps) with uniform jitter; ring_k =
    // delay + jitter + 1 slots of history (1: off)
    int delay, jitter, ring_k;
    // contact-depth backend of mesh objects: 0 signed distance, 1 raycast
    int depth_backend;
    // 1 when the noisy chain starts from the clean readings (no probe-radius
    // noise, no read delay): the hysteresis x_{t-1} of the depth and
    // force/torque channels, gain times last step's noisy-chain input, is
    // then gain times last step's clean output, read back from the output
    // arrays instead of being kept in hyst_prev (channels 0-6 unused)
    int prev_out;
};

// Object table entry (object frame); its size is a multiple of 16 bytes so
// that an entry can be bulk-copied.
struct alignas(16) ObjDev {
    int kind;
    float radius;
    float half[3];
    // grid
    int dims[3];
    float lo[3];
    float hi[3];
    float inv_h_hi[3], inv_h_lo[3];   // (dims-1)/(hi-lo) as a float pair
    float h[3];
    int fp16;
    const void* cells;                // cell-major corners: [cell][8] binary16 or float
    // mesh
    int n_verts, n_faces;
    const float* tri;                 // [n_faces][9]: a, b, c vertices
    const float* tri_n;               // [n_faces][3]: unit outward normals
    // raycast contact-depth backend (scenes that select it): the mesh's
    // bounding volume hierarchy (BvhNode / BvhTri of bvh.cuh) and each
    // reordered triangle's original face index
    const void* bvh_nodes;
    const void* bvh_tris;
    const int32_t* bvh_face;
    // and a coarse grid over the mesh's box of lower bounds on the distance
    // from any point of a cell to the mesh ([kBvhLbCells^3], cell-major x
    // fastest), to pass over probes no triangle can reach
    const float* bvh_lb;
    float bvh_lb_lo[3], bvh_lb_inv_h[3];
    // learned SDF (kind TG_OBJ_NEURAL; the grid fields hold its fallback grid)
    float nlo[3], nhi[3], ninv_ext[3];
    const uint32_t* ntable;           // [16][2^16] binary16 pairs
    const uint16_t* nweights;         // 6,208 bfloat16: W1 [64][32], W2 [64][64], W3 [64]
    // tracked surface points (point-cloud proximity), sorted by cell of a
    // uniform grid of cell size pc_radius over their box (object frame)
    const float4* pc_pts;             // [n] x, y, z, 0; null: no cloud
    const int32_t* pc_start;          // [cells + 1] first point of each cell
    int32_t pc_dims[3];
    float pc_lo[3];
    float pc_inv_h;
    int32_t pc_n;
};
static_assert(sizeof(ObjDev) % 16 == 0, "bulk-copyable object entries");

// One CTA of the step kernel: a run of whole links of one env.
struct Item {
    int32_t env;
    int16_t link_begin, link_end;     // [begin, end) over the env's link slots
    int64_t taxel_begin;              // global index of the first taxel
    int32_t n_taxels;
    int32_t pad;                      // in the per-step sorted copy: the env's object index
};

// Static layout of one work item for the pipelined step kernel, built at
// scene creation: the item's links' first taxels relative to the item, their
// lattices, and (when every link has the same rows x cols lattice holding
// rows * cols taxels) that lattice for the index arithmetic.  352 bytes, a
// multiple of 16 so that it can be bulk-copied.
struct alignas(16) ItemMeta {
    int32_t nl;                                  // links
    int32_t uni_len, uni_rows, uni_cols, uni_wrap;
    float uni_inv_len, uni_inv_cols;
    int32_t start[kItemMaxLinks + 1];            // first taxel of each link; start[nl] = taxels
    uint16_t rows[kItemMaxLinks], cols[kItemMaxLinks];
    uint8_t wrap[kItemMaxLinks];
    int32_t pad[8];
};
static_assert(sizeof(ItemMeta) == 352, "ItemMeta layout");

// One work item of this step as the pipelined step kernel reads it, in the
// step's item order (object-sorted or env order): where its taxels are, its
// env, the object the env holds this step and the env's episode.
struct alignas(16) SlotRec {
    int64_t taxel_begin;
    int32_t n_taxels, env;
    int32_t item, oid;
    uint32_t episode;
    int16_t link_begin, link_end;
};
static_assert(sizeof(SlotRec) == 32, "SlotRec layout");

// Per (env, link) lattice: where its taxels start within the item's env.
struct LinkLattice {
    int32_t env_offset;               // first taxel of the link, relative to the env
    uint16_t rows, cols;
    uint8_t wrap, present, pad0, pad1;
};

struct StepArgs {
    // static geometry
    const float *x, *y, *z, *nx, *ny, *nz, *R;
    const Item* items;
    const LinkLattice* lattice;       // [E*L]
    const ObjDev* objects;
    int n_objects;
    int n_envs, max_links;
    int64_t n_taxels;
    int64_t gid0;
    uint32_t sensors;
    ParamsDev P;
    // per-step inputs (device)
    const int32_t* obj_id;
    const Item* items_sorted;         // this step's items in object-sorted order, or null (items in env order)

    const float* link_rec;            // [E*L][kLinkRec] from the pose kernel
    uint32_t step;
    StepCtl* ctl;                     // work counter; the step too when step_from_ctl
    int step_from_ctl;
    int n_items;
    int persistent;                   // step kernel: CTAs take items from ctl->counter
    int shape;                        // step kernel CTA shape (kStepShapeThreads index)
    int resident_ctas;                // persistent grid size (SMs x resident CTAs per SM)
    // pipelined step kernel
    const ItemMeta* metas;            // [n_items] static item layout
    const SlotRec* slots;             // [n_items] this step's items in order
    int sms;                          // streaming multiprocessors (one CTA each)
    // state
    uint8_t* flags;
    float* hyst_prev;                 // [8][T]
    float* hyst_xi;                   // [8][T]
    float* drift;                     // [8][T]
    const uint32_t* episode;          // [E]
    float* ring;                      // [ring_k][8][T] read-delay history (ring_k > 1)
    int64_t env_gid0;                 // global id of env 0 (per-env draws)
    // outputs
    float* depth_clean;
    float* depth_noisy;
    float* dist;
    float* ft_clean;                  // [6][T]
    float* ft_noisy;                  // [6][T]
    float* link_out;                  // [E*L][kLinkOut]
    int32_t* link_count;              // [E*L][2]
    unsigned int* err;                // [0] non-finite count, [1] learned-SDF MMA wait timeouts
    float* pc_ft;                     // [6][T] point-cloud proximity force/torque (sensor on)
    float* prox_clean;                // [T] (proximity on)
    float* prox_noisy;                // [T]
    // learned-SDF objects: phi (scaled) of every taxel of a neural item and
    // the raw object-frame gradient of its near-contact taxels, from the
    // neural query kernel that runs before the step kernel
    const float* nq_phi;              // [T]
    const float* nq_grad;             // [3][T]
    const float* nq_phi_lo;           // [T] low part of phi (raycast meshes: phi = hi + lo)
    int any_neural;
    int all_grid;                     // every object is a plain SDF grid (the step kernel's grid-only form)
};

// Elastomer marker pads (one CTA per (env, pad)).
constexpr int kMaxPadMarkers = 1024;
constexpr int kMaxPadRadius = 4;
struct MarkerArgs {
    int n_envs, max_links, pads_per_env, rows, cols, radius;
    float pitch, alpha;
    const int32_t* pad_link;          // [E][P]
    const float* pad_frame;           // [E][P][9]
    const float* link_rec;            // pose records
    const int32_t* obj_id;
    const ObjDev* objects;
    int n_objects;
    // per-offset constants over the (2 radius + 1)^2 neighbourhood, offset o = source - target
    float w_norm[(2 * kMaxPadRadius + 1) * (2 * kMaxPadRadius + 1)];  // s_d g(r)
    float w_tan[(2 * kMaxPadRadius + 1) * (2 * kMaxPadRadius + 1)];   // s_d (c g / g_bar + (1 - c) rho / rho_bar)
    float* u;                         // [E][P][rows*cols][3]
    unsigned int* err;
    // shear anchors (off when shear_n == 0)
    int shear_n;                      // anchor slots per pad
    float s_s, lambda_s, eta_enter, eta_exit, half_t;  // half_t: half the elastomer thickness
    float2* anchors;                  // [E][P][shear_n]: (tangent, bitangent), NaN = none
    int32_t* anchor_obj;              // [E][P]: object the anchors belong to, -1 = none
    int32_t* n_anchored;              // [E][P]
};

struct PoseArgs {
    int n_envs, max_links;
    const float* link_pose;
    const float* link_vel;
    const float* obj_pose;
    const float* obj_vel;
    const float* env_params;          // may be null
    const LinkLattice* lattice;
    float def_mu, def_k;
    float tau_hi, tau_lo;             // pose_dt as a float pair
    float* link_rec;
    // per-step domain randomisation
    int dr_on;
    float dr_lo[3], dr_hi[3];
    uint64_t seed;
    int64_t env_gid0;
    uint32_t step;
    const StepCtl* ctl;               // non-null: step and pose_dt from here
};

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`.  The attribute is per device; each (kernel, device) keeps a
// high-water mark that only grows, so launches sized earlier keep working.
// Thread-safe.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

cudaError_t launch_pose(const PoseArgs& a, cudaStream_t s);
// pipelined step kernel (step_pipe.cu): threads per CTA 512, 768 or 1024
constexpr int kPipeShapes = 3;
constexpr int kPipeThreads[kPipeShapes] = {1024, 768, 512};
cudaError_t configure_pipe_kernels();
cudaError_t launch_step_pipe(const StepArgs& a, int n_items, int threads, cudaStream_t s);
// the step's SlotRec array: items in object-sorted order (sorted != 0) or in env order
cudaError_t launch_slot_records(const Item* items, int n_items, const int32_t* obj_id, int n_objects,
                                const uint32_t* episode, int sorted, SlotRec* out, cudaStream_t s);
cudaError_t launch_step(const StepArgs& a, int n_items, cudaStream_t s);
cudaError_t configure_step_kernels();
cudaError_t launch_set_ctl(StepCtl* ctl, StepCtl value, cudaStream_t s);
cudaError_t launch_advance_ctl(StepCtl* ctl, cudaStream_t s);
int step_kernel_resident_ctas(int shape);
cudaError_t launch_order_items(const Item* items, int n_items, const int32_t* obj_id, int n_objects, Item* sorted,
                               cudaStream_t s);
cudaError_t launch_reset(const StepArgs& a, int n_items, const uint8_t* env_mask, uint32_t episode,
                         uint32_t* episode_arr, cudaStream_t s);
constexpr int kItemMaxLinksHost = 32;   // links per work item (matches the step kernel)
cudaError_t launch_mesh_sdf_points(const float* tri, const float* tri_n, int n_faces, const float* points,
                                   int64_t n, float* phi, float* grad, cudaStream_t s);
cudaError_t launch_mesh_bake(const float* tri, const float* tri_n, int n_faces, const int dims[3],
                             const float lo[3], const float hi[3], int fp16, void* out, cudaStream_t s);
cudaError_t launch_build_cells(const void* values, const int dims[3], int fp16, void* cells, cudaStream_t s);
// sensor kernels: `threads` per CTA is 128, 256 or 512 (the autotuner's shapes)
cudaError_t launch_prox(const StepArgs& a, int n_items, int threads, cudaStream_t s);
cudaError_t launch_pc_prox(const StepArgs& a, int n_items, int threads, cudaStream_t s);
cudaError_t launch_markers(const MarkerArgs& m, int threads, cudaStream_t s);
// anchor_obj = -1 for the pads of the masked envs (all when mask is null)
cudaError_t launch_shear_reset(int32_t* anchor_obj, int n_envs, int pads_per_env, const uint8_t* mask,
                               cudaStream_t s);
// contact bit `bit` of every flag byte (0 clean, 2 noisy, 3 reported noisy with a read delay)
cudaError_t launch_unpack_contact(const uint8_t* flags, int64_t n, int bit, uint8_t* out, cudaStream_t s);

// learned SDF (nsdf.cu)
struct NsdfNet {
    float lo[3], hi[3];
    uint32_t* table;                  // [16][2^16] binary16 pairs (inference copy)
    uint16_t* weights;                // [6208] bfloat16 (inference copy)
    float* master;                    // [6208 + 2 * 16 * 2^16] FP32 masters: weights, then table
    float* adam_m;
    float* adam_v;
    int32_t adam_t;
};
cudaError_t nsdf_alloc(NsdfNet* n);
void nsdf_free(NsdfNet* n);
cudaError_t nsdf_init(NsdfNet* n, uint64_t seed, cudaStream_t s);
cudaError_t nsdf_sync_masters(NsdfNet* n, cudaStream_t s);   // masters <- inference copies, Adam state zeroed
// err: device word counting CTAs that stopped on an MMA wait timeout
cudaError_t launch_nsdf_eval(const ObjDev& o, const float* pts, int64_t n, float* phi, float* grad, unsigned* err,
                             cudaStream_t s);
// training forward/backward on points[idx[b]] (idx null: b), gradients accumulated into g_w [6208] and
// g_table [16][2^16][2]; per-CTA partial sums of |out - label| into loss_part [ceil(n/128)]
cudaError_t launch_nsdf_train_step(const ObjDev& o, const float* pts, const float* labels, const uint32_t* idx,
                                   int64_t n, float* g_part, float* g_w, float* g_table, float* loss_part,
                                   cudaStream_t s);
cudaError_t launch_nsdf_sample(uint64_t seed, uint32_t step, int64_t n_points, int32_t batch, uint32_t* idx,
                               cudaStream_t s);
cudaError_t launch_nsdf_adam(NsdfNet* n, const float* g_w, const float* g_table, float lr, float inv_batch_scale,
                             cudaStream_t s);
cudaError_t launch_nsdf_step_query(const StepArgs& a, int n_items, float* phi, float* grad, cudaStream_t s);
// raycast backend in the step: phi = s * (distance to the nearest triangle within reach) as a float pair and
// that triangle's normal, for every taxel of an env whose object is a mesh (raycast.cu)
cudaError_t launch_raycast_step_query(const StepArgs& a, int n_items, float* phi_hi, float* phi_lo, float* normal,
                                      cudaStream_t s);
// host BVH upload for a mesh object (raycast.cu); returns an error message or null
const char* upload_mesh_bvh(const float* verts, int nv, const int32_t* faces, int nf, ObjDev* t,
                            std::vector<void*>* bufs);
int nsdf_train_ctas(int64_t n);       // partial-gradient rows launch_nsdf_train_step writes
ObjDev nsdf_objdev(const NsdfNet& n); // a learned-SDF object over the network's own buffers
const NsdfNet* nsdf_net(const tg_nsdf* h);

}  // namespace tg
