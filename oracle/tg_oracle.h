/*
 * tg_oracle.h -- plain, slow FP64 CPU oracle for the tactile contact query
 * and noise model of "Tactile Genesis" (arxiv 2606.22332), Appendix A.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA path (no headers, helpers, tables or constants) and
 * never reads anything the CUDA path produced.
 *
 * Everything is double precision.  Inputs that the product takes as FP32
 * (poses, taxel geometry, grid values, mesh vertices) are read as float and
 * widened exactly; FP16 grid values are widened exactly from their bits.
 *
 * Conventions: SI units; quaternions (w, x, y, z); rotation matrices are
 * row-major 3x3; per-taxel multi-channel arrays are channel-major
 * (array[c * T + i]).
 */
#ifndef TG_ORACLE_H
#define TG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- object kinds -------------------------------------------------------- */
enum { OR_SPHERE = 0, OR_BOX = 1, OR_PLANE = 2, OR_MESH = 3, OR_GRID = 4, OR_NEURAL = 5 };

/* ---- learned SDF (tg_oracle_nsdf.c): hash encoding + bfloat16 MLP -------- */
#define OR_NSDF_LEVELS 16
#define OR_NSDF_FEATURES 2
#define OR_NSDF_TABLE 65536u
#define OR_NSDF_HIDDEN 64
#define OR_NSDF_IN (OR_NSDF_LEVELS * OR_NSDF_FEATURES)

typedef struct {
    double lo[3], hi[3];      /* encoding box, object frame (m) */
    const uint16_t* table;    /* [16][2^16][2] binary16 bits */
    const uint16_t* w1;       /* [64][32] bfloat16 bits, row = hidden unit */
    const uint16_t* w2;       /* [64][64] */
    const uint16_t* w3;       /* [64] */
} or_nsdf;

typedef struct {
    int32_t kind;
    double radius;            /* OR_SPHERE */
    double half[3];           /* OR_BOX half extents */
    int32_t n_verts, n_faces; /* OR_MESH */
    const float* verts;       /* [n_verts][3] object frame */
    const int32_t* faces;     /* [n_faces][3], outward (counter-clockwise) */
    int32_t dims[3];          /* OR_GRID nodes per axis (x, y, z) */
    double lo[3], hi[3];      /* OR_GRID box corners, object frame */
    int32_t fp16;             /* OR_GRID: 1 = values are binary16 bits */
    const void* values;       /* OR_GRID values [z][y][x]; OR_NEURAL: its fallback grid, marched by proximity rays */
    const or_nsdf* nsdf;      /* OR_NEURAL */
} or_object;

/* ---- noise knobs of one sensor group (Appendix A, "Sensor Noise Model") -- */
typedef struct {
    double gain_lo, gain_hi;  /* per-probe gain range drawn at reset (1,1 = off) */
    double beta, tau;         /* viscoelastic hysteresis (beta = 0: off) */
    double bias;              /* constant bias b */
    double sigma_white;       /* white noise sigma */
    double sigma_rw;          /* random-walk drift sigma per step */
    double quant;             /* quantisation step q (0 = off) */
    double stuck_lo, stuck_hi;/* dead-taxel stuck readout range */
} or_noise_group;

typedef struct {
    /* contact model (KinematicTaxel, Eqs. 4-9, plus the Coulomb clamp) */
    double k, c, alpha, k_t, k_omega;
    double mu;                /* friction coefficient; mu < 0 means no clamp */
    double eta_on, eta_off;   /* ContactProbe thresholds (Eq. 3) */
    double dt;                /* simulation step (s) */
    uint64_t seed;            /* Philox key */
    double p_dead;            /* dead-taxel probability */
    or_noise_group depth, ft, prox;
    double chi, xt_sigma;     /* spatial crosstalk strength and Gaussian sigma (lattice steps) */
    /* proximity by rays: n_rays (0 = off) over range prox_range (m); ray 0
       along the probe normal, the others on a cone of half-angle prox_cone */
    int32_t prox_rays;
    double prox_range, prox_cone;
    /* per-step domain randomisation (dr_on = 0: off): for every env and step,
       mu, k and the object scale uniform on [lo, hi] (index 0 lo, 1 hi) */
    int32_t dr_on;
    double dr_mu[2], dr_k[2], dr_scale[2];
    /* probe-radius noise (0 = off): the noisy readout of a taxel sees the
       radius max(0, R + eps), eps uniform on [-rho, rho], drawn per taxel and
       step (the clean readout keeps R) */
    double rho;
    /* read delay ("Base noise (every sensor)": the noisy readout is formed
       from y_{t - Delta_read}): the taxel sensor's noisy chain (depth,
       force/torque, noisy contact bit) reads its input from delay + j steps
       earlier, j uniform on {0..jitter} per env and step (0, 0 = off) */
    int32_t delay, jitter;
    /* contact-depth backend of mesh objects ("Two contact-depth backends"):
       0 the signed distance (sdf), 1 raycast: depth = the deepest penetration
       over the triangles within R of the probe, normal = that triangle's */
    int32_t depth_backend;
} or_params;

/* elastomer marker pads (ElastomerTaxel dilation, Eqs. 18-21) */
typedef struct {
    int32_t pads_per_env;        /* P (0 = off) */
    int32_t rows, cols;          /* markers per pad */
    double pitch;                /* marker spacing (m) */
    const int32_t* pad_link;     /* [E][P] link slot carrying the pad */
    const float* pad_frame;      /* [E][P][9]: origin(3), normal(3), tangent(3), link frame */
    double s_d, alpha, lambda_d, c, eps; /* dilation scale, depth power, Gaussian rate, compressibility, regularisation */
    int32_t radius;              /* neighbourhood half-width in markers (2 = 5x5) */
} or_pads;

/* point-cloud ProximityTaxel (Appendix A "ProximityTaxel"): every object
   carries tracked surface points (object frame, unscaled); a taxel's sensing
   sphere of radius R collects the points within it */
typedef struct {
    const float* cloud;          /* [sum of counts][3] tracked points of every object, object frame */
    const int64_t* cloud_off;    /* [n_objects + 1]: object o's points are rows cloud_off[o] .. cloud_off[o+1] - 1 */
    double radius;               /* sensing radius R (m) */
    double k, ks;                /* normal and shear gains */
    double density;              /* density scalar: rho_b = density / max(N_b, 1), N_b the env object's points */
} or_pcprox;

/* ElastomerTaxel shear anchors (Eqs. 19-20): the env object's tracked
   surface points, taken into each pad's frame (sensor frame: tangent,
   bitangent = normal x tangent, normal), anchor when their elastomer SDF
   falls below -eta_enter and release it above +eta_exit.  The elastomer is
   the box under the pad: the marker footprint (rows x pitch along the
   tangent, cols x pitch along the bitangent) and `thickness` deep. */
typedef struct {
    const float* cloud;          /* [sum of counts][3] tracked points of every object, object frame */
    const int64_t* cloud_off;    /* [n_objects + 1] */
    double s_s, lambda_s;        /* shear scale, Gaussian rate */
    double eta_enter, eta_exit;  /* anchor set below -eta_enter, cleared above +eta_exit (m) */
    double thickness;            /* elastomer thickness (m) */
    int64_t n_max;               /* anchor slots per pad (>= every object's point count) */
} or_shear;

typedef struct {
    int32_t n_envs, max_links;
    const int64_t* taxel_offsets; /* [n_envs+1] CSR of this (sub)scene */
    const int64_t* taxel_gid0;    /* [n_envs] global id of each env's first taxel */
    const int32_t* env_gid;       /* [n_envs] global env index */
    const int32_t* link_rows;     /* [n_envs*max_links] lattice rows (axial) */
    const int32_t* link_cols;     /* [n_envs*max_links] lattice cols (around) */
    const uint8_t* link_wrap;     /* [n_envs*max_links] 1: cols wrap around */
    const float *x, *y, *z, *nx, *ny, *nz, *R; /* [T] link-frame probe geometry */
    const or_object* objects;
    int32_t n_objects;
    or_params params;
} or_scene;

typedef struct {
    const float* link_pose;  /* [E][L][7] p, q(w,x,y,z) at time 0 */
    const float* link_vel;   /* [E][L][6] v, omega (world) */
    const float* obj_pose;   /* [E][7] */
    const float* obj_vel;    /* [E][6] */
    const int32_t* obj_id;   /* [E] */
    const float* env_params; /* [E][3] {mu, k, scale} or NULL */
    double pose_dt;          /* seconds to advance every pose by its velocity */
    uint32_t step;           /* RNG step counter */
} or_inputs;

/* channel index for per-taxel state: 0 depth, 1..6 force/torque, 7 proximity */
#define OR_NCH 8

typedef struct {
    uint8_t* flags;     /* [T] bit0 Schmitt state, bit1 dead */
    double* hyst_prev;  /* [OR_NCH][T] x_{t-1} */
    double* hyst_xi;    /* [OR_NCH][T] xi_{t-1} */
    double* drift;      /* [OR_NCH][T] d_{t-1} */
    uint32_t* episode;  /* [E] */
    /* read-delay ring [delay + jitter + 1][OR_RING_CH][T] (NULL when the delay is off):
       slot step mod (delay + jitter + 1) holds that step's noisy-chain input */
    double* ring;
} or_state;

/* channels of the read-delay ring: 0 depth, 1..6 force/torque, 7 the noisy contact bit (0/1) */
#define OR_RING_CH 8

/* per-link record: F_clean(3) T_clean(3) F_noisy(3) T_noisy(3)
   agg_force_clean(3) agg_force_noisy(3) */
#define OR_LINK_REC 18

typedef struct {
    uint8_t* contact_clean; uint8_t* contact_noisy;   /* [T] */
    double* prox_clean; double* prox_noisy;           /* [T] (proximity on) */
    uint8_t* prox_grazing;                            /* [T] 1: a ray grazes the surface (root ill-posed) */
    double* depth_clean; double* depth_noisy;         /* [T] */
    double* dist;                                     /* [T] phi - R */
    double* ft_clean; double* ft_noisy;               /* [6][T] */
    double* link_sums;                                /* [E*L][OR_LINK_REC] */
    int32_t* link_counts;                             /* [E*L][2] clean, noisy */
    uint8_t* depth_tie;                               /* [T] raycast backend: another triangle with a
                                                         different normal is as deep (within 1e-12 m),
                                                         so the normal is either's (NULL: not reported) */
} or_outputs;

/* ---- primitives (exported for the pins) ------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform(uint32_t x);
void or_box_muller(uint32_t x0, uint32_t x1, double* z0, double* z1);
uint16_t or_double_to_half(double x);
double or_half_to_double(uint16_t h);
void or_quat_to_mat(const double q[4], double R[9]);
void or_advance_pose(const double p0[3], const double q0[4], const double v[3],
                     const double w[3], double tau, double p[3], double R[9]);
double or_sdf_sphere(double r, const double q[3], double g[3]);
double or_sdf_box(const double h[3], const double q[3], double g[3]);
double or_sdf_plane(const double q[3], double g[3]);
double or_closest_point_triangle(const double p[3], const double a[3], const double b[3],
                                 const double c[3], double cp[3], int* region);
double or_winding_number(const float* V, const int32_t* F, int32_t nf, const double p[3]);
double or_sdf_mesh(const float* V, const int32_t* F, int32_t nf, const double p[3], double g[3]);
/* raycast depth backend ("Two contact-depth backends"): a probe at q (the
   mesh's frame; the mesh is scaled by `scale`) with radius R and sensing
   direction u (unit, from the probe towards the object) tests every
   triangle twice: a sphere-triangle closest-point test (penetration
   R - dist) and a ray-triangle test from q along u (penetration R - t for a
   hit at t >= 0).  The deepest penetration of either test over all
   triangles wins; n_out is the unit face normal (winding order) of the
   triangle that gave it (the first in face order on a tie), face_out its
   index.  Returns the depth (0 with n_out = 0 and face_out = -1 when nothing
   penetrates); ray_pen, if not NULL, receives the deepest penetration of the
   ray test alone (-inf when the ray hits nothing). */
double or_raycast_depth(const float* V, const int32_t* F, int32_t nf, double scale, const double q[3],
                        const double u[3], double R, double n_out[3], int32_t* face_out, double* ray_pen);
double or_sdf_grid(const or_object* o, const double q[3], double g[3]);
double or_sdf_object(const or_object* o, const double q[3], double g[3]);
int or_schmitt(int prev, double d, double eta_on, double eta_off);
void or_taxel_force(const or_params* P, double k, double mu, double d, const double x[3],
                    const double mbar[3], const double vrel[3], const double dw_dot_m,
                    double f[3], double tau[3]);
void or_crosstalk_weights(double sigma, double w[9]);

/* batched helpers for the pins */
void or_sdf_object_batch(const or_object* o, const double* q, int64_t n, double* phi, double* g);
void or_bake_grid(const float* V, const int32_t* F, int32_t nf, const int32_t dims[3],
                  const double lo[3], const double hi[3], int32_t fp16, void* out, int32_t threads);

double or_ray_first_root(const or_object* o, double scale, const double q0[3], const double d[3], double tmax,
                         int* grazing);
void or_dr_draw(const or_params* P, uint32_t env_gid, uint32_t step, double out[3]);
void or_prox_ray_dirs(const double n[3], int n_rays, double cone, double dirs[][3]);
double or_marker_kernel_g(double lambda_d, double r2);

/* learned SDF (round = 1: activations rounded to bfloat16 as on tensor cores) */
double or_bf16_to_double(uint16_t b);
uint16_t or_double_to_bf16(double x);
int32_t or_nsdf_resolution(int32_t level);
uint32_t or_nsdf_index(int32_t level, int64_t i, int64_t j, int64_t k);
double or_nsdf_eval(const or_nsdf* n, const double q[3], int32_t round, double grad_raw[3]);
double or_nsdf_flip_bound(const or_nsdf* n, const double q[3]);
void or_nsdf_normal(const or_nsdf* n, const double q[3], int32_t round, double g[3]);
void or_nsdf_normal_batch(const or_nsdf* n, int64_t B, const double* pts, int32_t round, double* g);
double or_nsdf_loss_grad(const or_nsdf* n, int64_t B, const double* pts, const double* labels_mm, int32_t round,
                         double* g_w1, double* g_w2, double* g_w3, double* g_table);
void or_adam_step(int64_t n, double* theta, double* m, double* v, const double* g, double lr, double beta1,
                  double beta2, double eps, int32_t t);
void or_nsdf_eval_batch(const or_nsdf* n, int64_t B, const double* pts, int32_t round, double* phi, double* grad_raw);
void or_nsdf_flip_bound_batch(const or_nsdf* n, int64_t B, const double* pts, double* out);

/* ---- whole-scene operations ------------------------------------------------- */
void or_reset(const or_scene* S, const uint8_t* env_mask, uint32_t episode, or_state* st);
int32_t or_read_delay(const or_params* P, uint32_t env_gid, uint32_t step);
int or_step(const or_scene* S, const or_inputs* in, or_state* st, or_outputs* out, int32_t threads);
/* marker displacements u [E][P][rows*cols][3] (pad frame: normal, tangent, normal x tangent) */
void or_markers(const or_scene* S, const or_pads* pads, const or_inputs* in, double* u, double* h_out, int32_t threads);
/* point-cloud proximity of every taxel: ft [6][T], link-frame force (rows 0-2)
   and torque (rows 3-5); inactive taxels read zero */
void or_pc_prox(const or_scene* S, const or_pcprox* pc, const or_inputs* in, double* ft, int32_t threads);
/* one step of the shear anchors of every pad.  State: anchors [E][P][n_max][2]
   (the anchor's tangent and bitangent coordinates, NaN = none) and
   anchor_obj [E][P] (the object they were taken on, -1 = none; a different
   object clears them).  Out: u [E][P][rows*cols][3] the shear displacement
   of every marker (normal, tangent, bitangent components), n_anchored [E][P],
   margin [E][P] the least distance of a point's SDF from the threshold it
   faces (-eta_enter for a free point, +eta_exit for an anchored one: how far
   the anchor decisions are from being taken the other way), and
   drag [E][P] = s_s sum (h + |Pi_n(z - e)|) over the anchored points whose
   SDF is below 1e-6 m (the scale of the shear's sensitivity to an error in
   the points' coordinates). */
void or_shear_step(const or_scene* S, const or_pads* pads, const or_shear* sh, const or_inputs* in, double* anchors,
                   int32_t* anchor_obj, double* u, int32_t* n_anchored, double* margin, double* drag,
                   int32_t threads);

#ifdef __cplusplus
}
#endif
#endif
