/*
 * tg.h -- C-ABI of the GB300-native tactile contact-query library.
 *
 * What it computes: the per-(environment, taxel) sensor read of Tactile
 * Genesis (arxiv 2606.22332), Appendix A:
 *   probe transform            q_j = p_L + R_L x_j, a_j = R_L n_j      (Eq. 1)
 *   contact depth (sdf)        d_j = [R_j - phi(q_j)]_+, m_j = grad phi (Eq. 2)
 *   contact bit (Schmitt)      on above eta_on, held above eta_off      (Eq. 3)
 *   kinematic force/torque     f = k_n s m + c_n s v_n - k_t v_t,
 *                              tau = x cross f - k_w ((w_C - w_L).m) m  (Eqs. 4-9)
 *                              with the tangential part clamped to the
 *                              Coulomb cone |f_t| <= mu |f_n|
 *   noise model                gain, viscoelastic hysteresis, 3x3 spatial
 *                              crosstalk, bias + white + random-walk drift,
 *                              quantisation, dead taxels         (Eqs. 25-31)
 *   per-link sums              sum f, sum tau (clean and noisy), contact
 *                              counts (agg_bool), agg_force      (Eq. 32)
 *
 * Conventions.
 *   - SI units.  Quaternions are (w, x, y, z); any non-zero norm is accepted
 *     and the rotation of the normalised quaternion is used.
 *   - Every call returns tg_status; no C++ exception crosses this boundary.
 *     tg_last_error() holds a message for the last failing call on a scene.
 *   - Pointers documented as "host or device" may be either; the library
 *     tells them apart with cudaPointerGetAttributes and copies host data on
 *     the call's stream.  Caller-owned inputs must stay valid until the
 *     stream work they feed has completed.
 *   - The library owns the scene's device state and outputs (cudaMalloc at
 *     tg_create_scene, cudaFree at tg_destroy_scene).  Views returned by
 *     tg_get_buffer stay valid until tg_destroy_scene; their contents are
 *     those of the last completed step.
 *   - Asynchronous device faults and the device error word (non-finite
 *     inputs) surface at the next tg_sync().
 *   - A scene is not thread-safe: one host thread at a time per scene.
 *   - Per-taxel arrays are in CSR order: env e owns taxels
 *     [taxel_offsets[e], taxel_offsets[e+1]); within an env, the taxels of
 *     link 0 come first, each link's rows x cols lattice in row-major order.
 *     Multi-channel per-taxel arrays are channel-major ([channel][T]).
 */
#ifndef TG_H
#define TG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tg_scene tg_scene;          /* opaque, owned by the library */
typedef void* tg_stream;                   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    TG_OK = 0,
    TG_ERR_INVALID_ARG = 1,   /* bad pointer, size, layout or parameter */
    TG_ERR_OOM = 2,           /* device allocation failed */
    TG_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    TG_ERR_STATE = 4,         /* call out of order (e.g. step before objects) */
    TG_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    TG_ERR_NUMERIC = 6,       /* non-finite values were seen in a step */
    TG_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} tg_status;

/* Noise knobs of one sensor group ("Sensor Noise Model", Eqs. 25-30). */
typedef struct {
    double gain_lo, gain_hi;   /* per-probe gain U[lo, hi] drawn at reset; (1, 1) = off */
    double beta, tau;          /* hysteresis strength and time constant (s); beta = 0 = off */
    double bias;               /* constant bias b */
    double sigma_white;        /* white noise sigma */
    double sigma_rw;           /* random-walk drift sigma per step */
    double quant;              /* quantisation step q; 0 = off (ties to even) */
    double stuck_lo, stuck_hi; /* dead-taxel readout U[lo, hi] drawn per episode */
} tg_noise_group;

/* Contact and noise parameters.  Doubles on the host; the kernels use FP32
   (and compensated FP32 for the geometry of near-contact taxels). */
typedef struct {
    double k, c, alpha, k_t, k_omega; /* KinematicTaxel (Eqs. 8-9): k_n, c_n, alpha, k_t, k_omega */
    double mu;                        /* Coulomb clamp coefficient; < 0 = no clamp */
    double eta_on, eta_off;           /* ContactProbe thresholds (Eq. 3), eta_off <= eta_on */
    double dt;                        /* simulation step in seconds (hysteresis decay) */
    double p_dead;                    /* dead-taxel probability per episode */
    double chi, xt_sigma;             /* crosstalk strength, Gaussian sigma in lattice steps */
    uint64_t seed;                    /* Philox4x32-10 key */
    tg_noise_group depth, ft, prox;   /* per sensor group */
    /* proximity rays (TG_SENSOR_PROX): n rays from the probe centre, ray 0
       along the probe normal, the others on a cone of half-angle prox_cone
       (rad) at equal azimuths from the tangent n x z (n x x when n is along z);
       reading = mean over rays of hit (1 - t / prox_range), t the distance to
       the first surface crossing along the ray */
    int32_t prox_rays;                /* 1..16 */
    double prox_range, prox_cone;
    /* per-step domain randomisation (dr_on = 0: off).  For every env and
       step, mu, k and the object scale are drawn uniformly on [lo, hi]
       (index 0 = lo, 1 = hi) from Philox at counter (global env id, step,
       tag 32, 0): mu from word 0, k from word 1, scale from word 2, each
       formed as lo + (hi - lo) u and rounded to binary32 (bounds are taken
       as binary32).  Replaces tg_step_inputs.env_params, which must then be
       NULL. */
    int32_t dr_on;
    double dr_mu[2], dr_k[2], dr_scale[2];
    /* largest probe error (mm, at the largest object scale) for which a
       NEURAL object's network is used instead of its grid (0.2) */
    double nsdf_max_err_mm;
    /* probe-radius noise rho (m, 0 = off; at most 5e-4): the noisy readout
       of a taxel sees the radius max(0, R + eps), eps = rho (2u - 1) with u
       the 24-bit uniform of word 0 of Philox at counter (global taxel id,
       step, tag 20, taxel id high), formed in binary32 (Appendix "Sensor Noise
       Model", probe-level imperfections).  The noisy depth, the force the
       force/torque noise chain starts from and the noisy contact bit (its
       own Schmitt state) use that radius; the clean readout keeps R, and the
       proximity rays do not depend on it. */
    double probe_radius_noise;
    /* point-cloud ProximityTaxel (TG_SENSOR_PCPROX; Appendix A
       "ProximityTaxel"): every object's tracked surface points
       (tg_object_desc.cloud) within pc_radius of a taxel contribute
       P = pc_radius - |p - q|; the taxel reports, in its link frame,
       f = pc_k rho sum P a + pc_ks rho sum P v_t and
       tau = pc_k rho sum P (p - q) x a, with a the taxel normal, v_t the
       point's velocity relative to the taxel's without its component along
       a, rho = pc_density / max(N, 1) and N the env object's point count.
       The object scale scales the points. */
    double pc_radius, pc_k, pc_ks, pc_density;
    /* read delay (Appendix "Sensor Noise Model", base noise: the noisy
       readout is formed from y_{t - Delta_read}, with optional uniform
       jitter), in steps: the noisy depth, force/torque and contact bit of
       step t are formed from the noisy chain's input (depth and force/torque
       before gain, hysteresis and crosstalk, and the contact bit) of step
       t - read_delay - j, j uniform on {0..read_jitter}, one draw per env and
       step: Philox at counter (global env id, step, tag 33, 0), j = ((w0 >> 8)
       (read_jitter + 1)) >> 24.  The noise draws, drift and dead override
       stay those of step t; before an episode's first read_delay + j steps
       the reset state (0) is read.  History is kept per step index, mod
       read_delay + read_jitter + 1 (at most 64 together), in a ring of that
       many slots x 8 channels per taxel.  0, 0 = off. */
    int32_t read_delay, read_jitter;
    /* contact-depth backend of mesh objects (Appendix A, "Probe geometry and
       contact-depth query", two contact-depth backends): 0 the signed
       distance (sdf); 1 raycast: a taxel's depth is R minus the distance from
       its probe centre to the nearest triangle within R (0 when none is; a
       probe centre more than R inside the mesh is clear), its contact normal
       that triangle's normal, found through a bounding volume hierarchy
       built at tg_upload_objects.  Other object kinds keep their signed
       distance.  Not combined with probe_radius_noise. */
    int32_t depth_backend;
} tg_params;

/* sensor mask bits (depth, contact and force/torque are always computed) */
#define TG_SENSOR_DIST 0x1u           /* SurfaceDistanceProbe output phi - R */
#define TG_SENSOR_PROX 0x2u           /* proximity by rays (geometry-aware ProximityTaxel form) */
#define TG_SENSOR_MARKERS 0x4u        /* ElastomerTaxel marker dilation on planar pads */
#define TG_SENSOR_PCPROX 0x8u         /* point-cloud ProximityTaxel (objects' tracked surface points) */

/* Elastomer marker pads (ElastomerTaxel, Eqs. 18-21): every env carries
   pads_per_env planar pads of rows x cols markers at `pitch`, each fixed in a
   link frame.  Marker depth h = max(0, -phi) (no probe radius); the
   displacement of marker j sums, over markers i within `radius` of j on the
   pad, s_d (r_ij w_ij + n h_i^alpha g(r_ij)) with r_ij the in-plane offset
   x_j - x_i, g(r) = exp(-lambda_d |r|^2), w_ij = h_i (c g / g_bar +
   (1 - c) rho / rho_bar), rho = 1 / (|r|^2 + eps^2); g_bar and rho_bar are
   the peaks of r g(r) and r rho(r).  Output per marker: (normal, tangent,
   normal x tangent) components.

   Shear anchors (Eqs. 19-20), on when shear_points > 0: the env object's
   tracked surface points (tg_object_desc.cloud) are taken into each pad's
   frame, z = (z_t, z_b, z_n) along tangent, bitangent = normal x tangent and
   normal.  The elastomer is the box under the pad (rows x pitch along the
   tangent, cols x pitch along the bitangent, `thickness` deep); a point
   whose SDF to it is below -eta_enter anchors at e = (z_t, z_b), an anchored
   point whose SDF rises above +eta_exit lets go, and every anchored point
   with penetration h = max(0, -SDF) > 0 adds
   s_s Pi_n(z - e) h exp(-lambda_s |Pi_n(x_j - z)|^2) to marker j.  The
   anchors are per (env, pad, point) state; a step on another object than the
   one they were taken on, or a reset of the env, clears them. */
typedef struct {
    int32_t pads_per_env;             /* P >= 0 */
    int32_t rows, cols;               /* rows * cols <= 1024 */
    double pitch;
    const int32_t* pad_link;          /* host [E][P]: link slot carrying the pad (a present link) */
    const float* pad_frame;           /* host [E][P][9]: origin, unit normal, unit tangent (link frame) */
    double s_d, alpha, lambda_d, c, eps;
    int32_t radius;                   /* neighbourhood half-width in markers, 0..4 */
    int32_t shear_points;             /* anchor slots per pad, 0 (shear off) .. 65536; every object's
                                         n_cloud must fit */
    double s_s, lambda_s;             /* shear scale, Gaussian rate (1/m^2) */
    double eta_enter, eta_exit;       /* anchor thresholds (m), both >= 0 */
    double thickness;                 /* elastomer thickness (m), > 0 */
} tg_pad_desc;

typedef struct {
    int32_t n_envs;                   /* E >= 1 */
    int32_t max_links;                /* L, 1..255: poses are [E][L] */
    const int64_t* taxel_offsets;     /* host [E+1], non-decreasing, [0] = 0 */
    const int32_t* link_rows;         /* host [E*L]; rows x cols taxels per link (0 x 0 = absent) */
    const int32_t* link_cols;         /* host [E*L] */
    const uint8_t* link_wrap;         /* host [E*L] or NULL: 1 = lattice columns wrap around */
    const float *x, *y, *z;           /* host or device [T]: link-frame probe position x_j */
    const float *nx, *ny, *nz;        /* host or device [T]: link-frame unit normal n_j */
    const float* R;                   /* host or device [T]: probe radius; 0 = inactive filler */
    tg_params params;
    uint32_t sensors;                 /* TG_SENSOR_* mask */
    int64_t taxel_gid0;               /* global id of taxel 0 in the RNG counters (sharding) */
    int32_t env_gid0;                 /* global id of env 0 */
    tg_pad_desc pads;                 /* used when sensors has TG_SENSOR_MARKERS */
} tg_scene_desc;

/* Create a scene: validates the layout, copies the taxel geometry to the
   device, allocates state and outputs, sets every env to episode 0 (dead
   masks drawn, state zeroed).  T = taxel_offsets[E]; a link lattice may hold
   at most tg_max_link_taxels() taxels.  Errors: TG_ERR_INVALID_ARG,
   TG_ERR_OOM, TG_ERR_CUDA.  *out is NULL on failure. */
tg_status tg_create_scene(const tg_scene_desc* desc, tg_scene** out);
void tg_destroy_scene(tg_scene* scene);
int32_t tg_max_link_taxels(void);

/* Object geometry in its own frame (Appendix A, "two contact-depth
   backends", the sdf form). */
typedef enum {
    TG_OBJ_SPHERE = 0,   /* radius */
    TG_OBJ_BOX = 1,      /* half[3], centred at the origin */
    TG_OBJ_PLANE = 2,    /* half-space z <= 0 */
    TG_OBJ_MESH = 3,     /* closed, outward-oriented triangle mesh: exact distance, winding-number sign */
    TG_OBJ_GRID = 4,     /* sampled SDF: trilinear, node (i,j,k) at lo + (i,j,k)(hi-lo)/(dims-1) */
    TG_OBJ_NEURAL = 5    /* learned SDF (tg_nsdf) with a GRID fallback, see tg_upload_objects */
} tg_object_kind;

/* ---- learned signed distance ("neural SDF", configs 3-4 of the evaluation)
   A multiresolution hash encoding (16 levels x 2 binary16 features, 2^16
   entries per level) of the object-frame point over a box, feeding a
   32 -> 64 -> 64 -> 1 ReLU MLP with bfloat16 weights and no biases; the output
   is the signed distance in millimetres.  Level l has N_l = floor(16 2^(l/3))
   cells per axis (16 .. 512); vertex (i,j,k) is entry i + (N+1)(j + (N+1)k)
   while (N+1)^3 <= 2^16, else (i ^ j 2654435761 ^ k 805459861) mod 2^16.
   Inference runs the layers on tensor cores (bfloat16 operands, FP32
   accumulation: the encoding and both hidden activations are rounded to
   bfloat16).  Outside the box phi = phi(clamp q) + |q - clamp q|.
   Parameter layout: table [16][2^16][2] binary16 bits; weights 6,208
   bfloat16 bits = W1 [64][32], then W2 [64][64], then W3 [64] (row = output
   unit).  A tg_nsdf owns device parameters, FP32 master copies and Adam
   state; not thread-safe. */
typedef struct tg_nsdf tg_nsdf;
#define TG_NSDF_TABLE_ENTRIES (16 * 65536)
#define TG_NSDF_WEIGHTS 6208

/* New network over the box [lo, hi] (object frame, m), initialised from
   `seed`: table uniform in +-1e-4, weights uniform in +-sqrt(6 / (fan_in +
   fan_out)).  Errors: TG_ERR_INVALID_ARG (lo >= hi), TG_ERR_OOM. */
tg_status tg_nsdf_create(const float lo[3], const float hi[3], uint64_t seed, tg_nsdf** out);
void tg_nsdf_destroy(tg_nsdf* net);
/* Set / get the parameters (host or device buffers of the layout above);
   setting also resets the Adam state and the FP32 masters to the values. */
tg_status tg_nsdf_set_params(tg_nsdf* net, const uint16_t* table, const uint16_t* weights);
tg_status tg_nsdf_get_params(tg_nsdf* net, uint16_t* table, uint16_t* weights);
/* phi (m) at n object-frame points (device [n][3]) into device phi [n];
   grad (device [n][3] or NULL): the raw gradient d phi / d q of the network
   (FP32, taken at the clamped point; not normalised).  Asynchronous; a
   tensor-core wait that timed out (no result written for the rest of that
   CTA's points) is reported as TG_ERR_TIMEOUT by the next tg_nsdf_probe. */
tg_status tg_nsdf_eval(tg_nsdf* net, const float* points, int64_t n, float* phi, float* grad, tg_stream stream);
/* Mean over the n points (device [n][3]) of |out - label_mm| and its
   gradients, the training forward and backward: FP32 activations on the
   stored binary16 / bfloat16 parameters, gradients into device g_weights
   [6208] and g_table [16][2^16][2] (FP32); *loss written on the host after
   the work completes (the call synchronises `stream`). */
tg_status tg_nsdf_loss_grad(tg_nsdf* net, const float* points, const float* labels_mm, int64_t n, double* loss,
                            float* g_weights, float* g_table, tg_stream stream);
/* `steps` Adam steps (beta1 0.9, beta2 0.99, eps 1e-15) on minibatches of
   `batch` points drawn uniformly (Philox, `seed`) from the n labelled points
   (device [n][3] and [n], labels in mm); learning rate lr0 (lr_final /
   lr0)^(t / steps).  losses (host [steps] or NULL): each step's minibatch
   loss; the call synchronises `stream` when losses is given. */
tg_status tg_nsdf_train(tg_nsdf* net, const float* points, const float* labels_mm, int64_t n, int32_t steps,
                        int32_t batch, double lr0, double lr_final, uint64_t seed, float* losses, tg_stream stream);
/* Error probe against the exact mesh distance: over n probe points (device
   [n][3]), the maximum and mean |phi_net - phi_mesh| in mm.  Synchronous. */
/* message of the last failed tg_nsdf_* call on this thread */
const char* tg_nsdf_last_error(void);
tg_status tg_nsdf_probe(tg_nsdf* net, const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                        const float* points, int64_t n, double* max_err_mm, double* mean_err_mm, tg_stream stream);

typedef struct {
    int32_t kind;
    float radius;                     /* SPHERE */
    float half[3];                    /* BOX */
    int32_t n_verts, n_faces;         /* MESH */
    const float* verts;               /* host or device [n_verts][3] */
    const int32_t* faces;             /* host or device [n_faces][3], indices < n_verts */
    int32_t dims[3];                  /* GRID nodes per axis (x, y, z), each >= 2 */
    float lo[3], hi[3];               /* GRID box, lo < hi */
    int32_t fp16;                     /* GRID: 1 = values are IEEE binary16 */
    const void* values;               /* GRID: host or device [dims z][dims y][dims x] */
    const tg_nsdf* nsdf;              /* NEURAL: the network (its parameters are copied) */
    double nsdf_err_mm;               /* NEURAL: probe error (tg_nsdf_probe max); < 0 = not probed */
    const float* cloud;               /* any kind: host or device [n_cloud][3] tracked surface points
                                         (object frame) for TG_SENSOR_PCPROX, or NULL */
    int64_t n_cloud;                  /* 0 .. 2^24 */
} tg_object_desc;

/* Upload (replace) the scene's object table.  Per env, tg_step_inputs.obj_id
   picks one object.  The library copies everything.  A query outside a grid's
   box reads phi(clamp(q)) + |q - clamp(q)|.  A NEURAL object carries a
   network and a GRID (dims, lo, hi, fp16, values): the network answers the
   contact query when 0 <= nsdf_err_mm * s_max <= params.nsdf_max_err_mm
   (s_max = dr_scale hi under domain randomisation, else 1), else the grid
   does; proximity rays always march the grid.  tg_object_info reports the
   choice.  Errors: TG_ERR_INVALID_ARG, TG_ERR_OOM, TG_ERR_CUDA. */
tg_status tg_upload_objects(tg_scene* scene, const tg_object_desc* objs, int32_t n);
/* kind in use for object i (TG_OBJ_NEURAL or, after a fallback, TG_OBJ_GRID)
   and the probe error it was uploaded with (NaN for other kinds). */
tg_status tg_object_info(const tg_scene* scene, int32_t i, int32_t* kind_used, double* nsdf_err_mm);

/* Start a new episode for the envs whose env_mask byte is non-zero (host or
   device [E]; NULL = all): dead masks are redrawn from (seed, taxel id,
   episode), hysteresis, drift and Schmitt state are zeroed, and so are the
   envs' clean depth and force/torque outputs (they read zero until the
   envs' next step).  Ordered on `stream`. */
tg_status tg_reset_envs(tg_scene* scene, const uint8_t* env_mask, uint32_t episode, tg_stream stream);

/* Per-step inputs (host or device pointers, caller-owned). */
typedef struct {
    const float* link_pose;   /* [E][L][7] p(3), q(4) of every link at time 0 of the advance */
    const float* link_vel;    /* [E][L][6] v(3), omega(3), world frame */
    const float* obj_pose;    /* [E][7] */
    const float* obj_vel;     /* [E][6] */
    const int32_t* obj_id;    /* [E], index into the object table */
    const float* env_params;  /* [E][3] {mu, k, scale} per env, or NULL = params.mu, params.k, 1 */
    double pose_dt;           /* advance: p += v pose_dt, R = exp([omega] pose_dt) R */
    uint32_t step;            /* RNG counter of this step */
} tg_step_inputs;

/* One sensor step for every env: enqueued on `stream`, asynchronous.
   Inputs in host memory are copied to the device on the scene's own copy
   stream, into one of two staging sets used in turn, so that a step's
   copies overlap the kernels of the step before it; `stream` waits for
   them.  As with any asynchronous copy, the host buffers must not change
   until `stream` has passed this step (pinned buffers make the copies
   asynchronous; pageable ones are copied before the call returns).
   Errors: TG_ERR_STATE (no objects), TG_ERR_INVALID_ARG (NULL input, or an
   obj_id in host memory outside [0, n_objects): nothing runs; object
   indices in device memory are clamped into that range by the kernels),
   TG_ERR_CUDA (launch failure).  Non-finite signed distances (from a NaN or
   infinite pose, say) are counted on the device: those taxels read as clear
   of the surface, and the next tg_sync returns TG_ERR_NUMERIC with the count
   and clears it. */
tg_status tg_step_sensors(tg_scene* scene, const tg_step_inputs* in, tg_stream stream);

/* Step replay through a CUDA graph (one vectorised launch sequence per step,
   "Batched Simulation" of the paper's system section).
   tg_graph_capture records the launches of one step, exactly as
   tg_step_sensors(scene, in) enqueues them, into a graph owned by the scene.
   The graph reads in's buffers in place on every replay, so they must be
   device pointers that stay valid and are refilled by the caller between
   replays; host pointers give TG_ERR_INVALID_ARG.  Replay r (counted from
   the capture or the last tg_graph_seek) runs RNG step in->step + r with
   pose_dt = in->pose_dt + r * pose_dt_per_step: the step index lives in
   device memory and the graph's last node advances it, so a replay needs
   no host work.  tg_graph_launch enqueues n_steps replays on `stream`;
   tg_graph_seek resets the replay counter to (step, pose_dt) in stream
   order.  The captured schedule (tg_set_schedule) is fixed until release.
   Errors: TG_ERR_STATE (no objects / nothing captured), TG_ERR_INVALID_ARG,
   TG_ERR_CUDA. */
tg_status tg_graph_capture(tg_scene* scene, const tg_step_inputs* in, double pose_dt_per_step, tg_stream stream);
tg_status tg_graph_launch(tg_scene* scene, int32_t n_steps, tg_stream stream);
tg_status tg_graph_seek(tg_scene* scene, uint32_t step, double pose_dt, double pose_dt_per_step, tg_stream stream);
tg_status tg_graph_release(tg_scene* scene);

/* Work schedule of the step kernel.  Work items are runs of whole links of
   one env (at most 1,024 taxels).
     TG_SCHED_GRID        one 512-thread CTA per work item, two resident
                          per SM;
     TG_SCHED_PERSISTENT  resident 512-thread CTAs take items from an atomic
                          counter;
     TG_SCHED_GRID_384 / TG_SCHED_PERSISTENT_384  the same with 384-thread
                          CTAs, three resident per SM (each thread takes
                          more of the item's taxels; a third item in flight
                          per SM covers more of each item's waits);
     TG_SCHED_PIPE_1024 / _768 / _512  pipelined: one CTA of that many
                          threads per SM runs its share of the items in turn,
                          and bulk copies bring each item's taxel geometry,
                          link poses and noise state into shared memory while
                          the item before it computes.
   sorted = 1: items run in the order of the object their env holds (a
   counting sort each step), so concurrent CTAs share object grids in L2.
   Results are bit-identical across schedules.

   Launch shapes of the sensor kernels (proximity rays, point-cloud
   proximity, elastomer markers): 128, 256 or 512 threads per CTA (default
   256), set by tg_set_sensor_threads.  Results are bit-identical across
   shapes.

   tg_autotune times every schedule (x sorted / env order when there are
   several objects) on `steps` steps of the given inputs (after one warm-up
   step each) and keeps the fastest; then, on that schedule, each sensor
   kernel the scene runs at each of its shapes, keeping the fastest.  It
   restores the noise state and the shear anchors it found (the output
   buffers then hold the last trial's step).
   Errors: TG_ERR_STATE (a captured graph exists), TG_ERR_INVALID_ARG. */
typedef enum {
    TG_SCHED_GRID = 0,
    TG_SCHED_PERSISTENT = 1,
    TG_SCHED_PIPE_1024 = 2,
    TG_SCHED_PIPE_768 = 3,
    TG_SCHED_PIPE_512 = 4,
    TG_SCHED_GRID_384 = 5,
    TG_SCHED_PERSISTENT_384 = 6,
    TG_SCHED_COUNT = 7
} tg_schedule;
typedef enum {
    TG_KERNEL_PROX = 0,      /* proximity rays (TG_SENSOR_PROX) */
    TG_KERNEL_PCPROX = 1,    /* point-cloud proximity (TG_SENSOR_PCPROX) */
    TG_KERNEL_MARKERS = 2,   /* elastomer markers (TG_SENSOR_MARKERS) */
    TG_SENSOR_KERNEL_COUNT = 3
} tg_sensor_kernel;
typedef struct {
    int32_t schedule, sorted;  /* the step kernel's schedule of this trial */
    double ms_per_step;        /* whole step, CUDA events */
    int32_t kernel;            /* -1: a step-kernel schedule was timed; else the
                                  tg_sensor_kernel whose launch shape was timed */
    int32_t threads;           /* threads per CTA of that kernel */
} tg_tune_candidate;
typedef struct {
    int32_t n, chosen;                 /* chosen: candidate of the step schedule kept */
    int32_t sensor_chosen[3];          /* per tg_sensor_kernel: candidate kept, -1 if not tuned */
    tg_tune_candidate cand[32];
} tg_tune_report;
tg_status tg_set_schedule(tg_scene* scene, int32_t schedule, int32_t sorted);
tg_status tg_get_schedule(const tg_scene* scene, int32_t* schedule, int32_t* sorted);
tg_status tg_set_sensor_threads(tg_scene* scene, int32_t kernel, int32_t threads);
tg_status tg_get_sensor_threads(const tg_scene* scene, int32_t kernel, int32_t* threads);
tg_status tg_autotune(tg_scene* scene, const tg_step_inputs* in, int32_t steps, tg_tune_report* report,
                      tg_stream stream);

typedef enum {
    TG_CH_CONTACT = 0,        /* uint8 [T]: 0/1 */
    TG_CH_DEPTH = 1,          /* float [T] */
    TG_CH_DIST = 2,           /* float [T] (needs TG_SENSOR_DIST); clean only */
    TG_CH_FORCE_TORQUE = 3,   /* float [6][T]: fx fy fz tx ty tz, link frame */
    TG_CH_LINK_WRENCH = 4,    /* float [E*L][18]: F_clean T_clean F_noisy T_noisy agg_clean agg_noisy */
    TG_CH_LINK_COUNT = 5,     /* int32 [E*L][2]: contact count clean, noisy (agg_bool = count > 2) */
    TG_CH_STATE_FLAGS = 6,    /* uint8 [T]: bit0 clean contact, bit1 dead, bit2 noisy contact (its Schmitt
                                 state); with a read delay, bit3 the reported (delayed) noisy contact */
    TG_CH_PROX = 7,           /* float [T] (needs TG_SENSOR_PROX) */
    TG_CH_MARKER = 8,         /* float [E*P*rows*cols][3] (needs TG_SENSOR_MARKERS); clean only */
    TG_CH_PC_FT = 9,          /* float [6][T]: point-cloud proximity force/torque, link frame (needs
                                 TG_SENSOR_PCPROX); clean only */
    TG_CH_SHEAR_ANCHORS = 10  /* int32 [E*P]: anchored points per pad after the last step (needs
                                 TG_SENSOR_MARKERS with shear_points > 0) */
} tg_channel;

/* Copy one output channel (clean or noisy) into dst (host or device),
   ordered on `stream` after the last step.  dst_bytes must equal the
   channel's size (tg_channel_bytes).  Errors: TG_ERR_INVALID_ARG. */
tg_status tg_read_taxels(tg_scene* scene, int32_t channel, int32_t noisy, void* dst, size_t dst_bytes,
                         tg_stream stream);
size_t tg_channel_bytes(const tg_scene* scene, int32_t channel);

/* Device view of a library-owned output buffer (no copy).  CONTACT has no
   view: read it, or decode TG_CH_STATE_FLAGS.  Views are read-only: without
   probe-radius noise or a read delay the next step reads last step's clean
   depth and force/torque back as the hysteresis state (gain times the
   clean reading is x_{t-1} of Eqs. 29-30), so writing into them changes the
   next step's noisy readout.  Errors: TG_ERR_INVALID_ARG. */
tg_status tg_get_buffer(tg_scene* scene, int32_t channel, int32_t noisy, void** dev_ptr, size_t* bytes);

/* Wait for the scene's work on `stream` and report device-side errors
   (TG_ERR_NUMERIC when non-finite values were seen since the last sync,
   TG_ERR_CUDA on an asynchronous fault). */
tg_status tg_sync(tg_scene* scene, tg_stream stream);
const char* tg_last_error(const tg_scene* scene);

/* Checkpoint: the per-taxel state (flags, hysteresis, drift), per-env
   episode numbers and, with shear anchors on, the anchors of every pad.  With buf == NULL, *size receives the needed size.
   Philox draws are counter-based, so a restored scene replays bit-exactly.
   A checkpoint restores a scene of the same shape and noise-chain form
   (with or without probe-radius noise or a read delay: without them the
   hysteresis x_{t-1} of the depth and force/torque channels is stored as the
   clean outputs it derives from); any other buffer is refused.
   Synchronous.  Errors: TG_ERR_INVALID_ARG (size or shape mismatch). */
tg_status tg_save_state(tg_scene* scene, void* buf, size_t* size);
tg_status tg_load_state(tg_scene* scene, const void* buf, size_t size);

/* Kernel timing for measurement.  While enabled, every tg_step_sensors
   records CUDA events on its stream around its two kernels (the pose
   prologue: pose advance and the object-sorted work order; and the fused
   step), and so does every graph replay of a step that was captured while
   timing was enabled (each replay records into events of its own).  tg_profile_read waits for the recorded events and returns the
   summed device time in milliseconds of the prologue kernels and of the
   step kernel, and the number of steps since the previous read, then clears
   them. */
tg_status tg_profile_enable(tg_scene* scene, int32_t on);
tg_status tg_profile_read(tg_scene* scene, double* pose_ms, double* step_ms, int64_t* n_steps);

/* Exact signed distance to a closed, outward-oriented triangle mesh sampled
   at the nodes of a grid (the grid bake that turns a mesh into a
   TG_OBJ_GRID): unsigned distance by closest point over every face, negative
   where the generalised winding number exceeds 1/2.  Computed in FP32 with a
   compensated re-evaluation of the nearest faces, then rounded once to float
   or binary16.  out: device [dims z][dims y][dims x].  Stateless,
   asynchronous on `stream`.  Errors: TG_ERR_INVALID_ARG, TG_ERR_CUDA. */
tg_status tg_bake_grid(const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                       const int32_t dims[3], const float lo[3], const float hi[3], int32_t fp16,
                       void* out, tg_stream stream);

/* The same exact mesh SDF at n arbitrary points (device [n][3]); phi device
   [n]; grad device [n][3] (unit gradient) or NULL. */
tg_status tg_mesh_sdf(const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                      const float* points, int64_t n, float* phi, float* grad, tg_stream stream);

/* Largest mesh tg_mesh_sdf_noalloc accepts. */
#define TG_NOALLOC_MAX_FACES 65536

/* tg_mesh_sdf without any device allocation.  The paper has no counterpart:
   this entry point exists for callers that cannot call cudaMalloc, such as
   an application whose own allocator owns all of the GPU's memory (a
   framework with a fixed memory budget that forbids allocations from outside
   it), or code on a path where cudaMalloc's implicit device-wide
   synchronisation is not acceptable.  tg_mesh_sdf copies the mesh into a
   triangle list it allocates for each call; this variant builds that list on
   the GPU in a device array inside the library, sized for
   TG_NOALLOC_MAX_FACES faces (3 MiB, held by every GPU that loads the
   library until the process exits).
   verts [n_verts][3], faces [n_faces][3], points [n][3], phi [n] and grad
   [n][3] (or NULL) must all be device memory.  phi is bit-identical to
   tg_mesh_sdf's; grad too, except where a point's gradient is the normal of
   the face it is nearest (a face interior, or a point on the surface): this
   variant normalises the face normal in FP32 on the GPU, tg_mesh_sdf in FP64
   on the host, so those may differ in the last bits.  Meshes over
   TG_NOALLOC_MAX_FACES faces, host pointers or bad sizes return
   TG_ERR_INVALID_ARG and run nothing.  The mesh is not read on the host, so
   an invalid face cannot be rejected there the way tg_mesh_sdf rejects it:
   a face index outside [0, n_verts) (never read out of bounds), a face
   with two equal indices, or a face whose FP32 cross product (each product
   rounded on its own) is zero (zero area) makes every phi and grad value of
   the call NaN.  The first call on each device looks up the
   array's device address once; make that first call before any stream
   capture.  Every call shares the array and clears what must start at zero
   (the invalid-face counter): calls whose GPU work overlaps (different
   streams or host threads) race on it, so the caller must order them.
   Asynchronous on `stream`. */
tg_status tg_mesh_sdf_noalloc(const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                              const float* points, int64_t n, float* phi, float* grad, tg_stream stream);


/* ---- TemperatureGrid (Appendix "TemperatureGrid Sensor Model") -----------

   G grids of nx x ny x nz cells (one per voxelized sensor link; cell (i,j,k)
   at flat index (i*ny + j)*nz + k, per-grid voxel size (dx, dy, dz)).  One
   step advances every grid's cell temperatures T (Celsius) by
   1. implicit spectral diffusion: the grid mirror-padded to twice its size on
      every axis (zero-flux walls), every Fourier mode divided by
      1 + alpha dt max(k^2, k2_floor), alpha = k / (rho c_p), cropped back;
   2. the internal source: T += dt q / (dz rho c_p), q in W/m^2 per cell;
   3. contact conduction: a contact on cell c with a body at T_other of
      conductivity k_b over area A adds dt k_eff (T_other - T_c) (A / V)^2 /
      (rho c_p), k_eff = 2 k k_b / (k + k_b), V the cell volume (the flux
      k_eff dT / L over L = V / A, times A / V); every contact reads the field
      after the source and the changes add;
   4. radiation and convection on every cell of a face of the grid:
      T -= dt (emissivity sigma (T_K^4 - T_amb,K^4) + h (T - T_amb)) / (rho c_p),
      T_K = T + 273.15, as the paper prints it;
   and the measured readout follows with a first-order lag:
   T_meas += dt / tau (T - T_meas), or T_meas = T when tau <= 0.
   Buffers are device-resident and library-owned. */
typedef struct tg_temp tg_temp;

typedef struct {
    int32_t n_grids;                  /* G >= 1 */
    int32_t nx, ny, nz;               /* each 4, 8, 16 or 32; nx*ny*(nz+1) <= 12288 */
    const float* voxel;               /* host [G][3]: dx, dy, dz (m), > 0 */
    const float* material;            /* host [G][7]: k (W/m/K) >= 0, rho (kg/m^3) > 0, c_p (J/kg/K) > 0,
                                         emissivity >= 0, h (W/m^2/K) >= 0, tau (s), base temperature (C) */
    double k2_floor;                  /* floor of k^2 (1/m^2) that regularises the zero mode, >= 0 */
} tg_temp_desc;

typedef struct {
    double dt;                        /* step (s), > 0 */
    double t_amb;                     /* ambient temperature (C) */
    const float* source;              /* device [G][cells] (W/m^2) or NULL */
    int32_t n_contacts;               /* C >= 0 */
    const int32_t* contact_offsets;   /* host or device [G+1]: grid g's contacts are offsets[g] .. offsets[g+1]-1 */
    const int32_t* contact_cell;      /* host or device [C]: flat cell index */
    const float* contact_temp;        /* host or device [C]: T_other (C) */
    const float* contact_k;           /* host or device [C]: k_b (W/m/K), > 0 */
    const float* contact_area;        /* host or device [C]: A (m^2), > 0 (tg_contact_area) */
} tg_temp_inputs;

/* Create G grids at their base temperatures (T = T_meas = base).  Errors:
   TG_ERR_INVALID_ARG (sizes, non-finite or out-of-range values), TG_ERR_OOM,
   TG_ERR_CUDA.  *out is NULL on failure. */
tg_status tg_temp_create(const tg_temp_desc* desc, tg_temp** out);
void tg_temp_destroy(tg_temp* grids);
/* Back to the base temperature for the masked grids (grid_mask host or
   device [G], NULL = all), ordered on `stream`. */
tg_status tg_temp_reset(tg_temp* grids, const uint8_t* grid_mask, tg_stream stream);
/* Overwrite the fields from host or device [G][cells] arrays (measured NULL:
   the measured readout takes `field`). */
tg_status tg_temp_set(tg_temp* grids, const float* field, const float* measured, tg_stream stream);
/* One step, ordered on `stream`.  Host contact arrays are checked (offsets
   from 0 to C, non-decreasing; cells in range; k_b, A > 0) and staged, and the
   call waits for the staging; device arrays are used in place (the kernel
   clamps offsets and skips cells out of range).  Errors: TG_ERR_INVALID_ARG,
   TG_ERR_CUDA. */
tg_status tg_temp_step(tg_temp* grids, const tg_temp_inputs* in, tg_stream stream);
/* Copy T (measured = 0) or T_meas (measured = 1), [G][cells] float, into dst
   (host or device); dst_bytes must be 4 G nx ny nz. */
tg_status tg_temp_read(tg_temp* grids, int32_t measured, float* dst, size_t dst_bytes, tg_stream stream);
/* Device view of T or T_meas (no copy). */
tg_status tg_temp_buffer(tg_temp* grids, int32_t measured, float** ptr);
/* Contact area of n_pairs contact manifolds (Appendix "TemperatureGrid Sensor
   Model", contact area estimation): points device [n_pairs][max_points][3]
   with n_points device [n_pairs] valid, depth device [n_pairs] the
   penetration delta.  The points are projected on their best-fit plane,
   ordered by polar angle about their centroid, and the shoelace area taken;
   fewer than three points give a disk of radius delta (pi delta^2); the
   result is floored at pi (d_w delta)^2.  max_points 1..16.  area: device
   [n_pairs]. */
tg_status tg_contact_area(const float* points, const int32_t* n_points, const float* depth, int32_t n_pairs,
                          int32_t max_points, double d_w, float* area, tg_stream stream);
const char* tg_temp_last_error(void);


/* ---- raycast contact-depth backend ("Two contact-depth backends") --------

   A bounding volume hierarchy over one triangle mesh (its own frame).  Per
   probe at q with radius R, the paper's raycast backend runs on every nearby
   triangle a sphere-triangle closest-point test (penetration R - dist) and a
   ray-triangle test along the probe's sensing direction (penetration R - t);
   the deepest wins and the contact normal is that triangle's face normal.  A
   ray's hit lies on its triangle, so t >= dist and the ray test never gives
   the deeper value: the depth is R - (distance to the nearest triangle within
   R), 0 when there is none, and that is what tg_raycast_depth computes. */
typedef struct tg_mesh_bvh tg_mesh_bvh;

/* Build the tree of verts (host [n_verts][3]) and faces (host [n_faces][3],
   counter-clockwise seen from outside gives the outward normal).  Errors:
   TG_ERR_INVALID_ARG (indices out of range, non-finite vertices, an empty
   mesh), TG_ERR_OOM, TG_ERR_CUDA. */
tg_status tg_mesh_bvh_create(const float* verts, int32_t n_verts, const int32_t* faces, int32_t n_faces,
                             tg_mesh_bvh** out);
void tg_mesh_bvh_destroy(tg_mesh_bvh* bvh);
/* Depth at n probes: probes device [n][3] in the mesh's frame with the mesh
   scaled by `scale` (> 0), radius device [n] (R <= 0: inactive, depth 0);
   depth device [n]; normal device [n][3] (unit face normal, mesh frame; 0
   where the depth is 0) and face device [n] (the face index, -1 where the
   depth is 0) may be NULL.  Ordered on `stream`.  Errors: TG_ERR_INVALID_ARG,
   TG_ERR_CUDA. */
tg_status tg_raycast_depth(const tg_mesh_bvh* bvh, const float* probes, const float* radius, int64_t n, double scale,
                           float* depth, float* normal, int32_t* face, tg_stream stream);
const char* tg_mesh_bvh_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TG_H */
