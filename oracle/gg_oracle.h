/*
 * gg_oracle.h -- FP64 CPU oracle for the granular contact step of GranularGym
 * (arxiv 2306.01369).  TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline leg may call it; the product path never does.
 * It shares no code, header or constant table with the CUDA library.
 *
 * Precision: dynamics in FP64.  Decisions that turn floating point into an
 * integer (cell index, hash bucket, "in contact or not", which SDF branch is
 * active) are taken in FP32 with one fixed evaluation order and no fused
 * multiply-add, because the method is run in FP32 and both sides must take
 * those decisions identically.  Compile with -ffp-contract=off.
 */
#ifndef GG_ORACLE_H
#define GG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double dt;          /* time step (Alg. 1, Eq. 4-5) */
  double gravity[3];  /* external acceleration, F_ext / m (Eq. 1) */
  double mu;          /* Coulomb friction coefficient (Eq. 3) */
  double alpha;       /* Baumgarte factor (Sec. II-A, last paragraph) */
  int32_t pja_iters;  /* iterations n of Alg. 1 */
  int32_t n_threads;  /* OpenMP threads for the per-particle loops (results do not depend on it) */
  float cell_size;    /* grid cell edge c (Eq. 6 uses c = 2r); must be >= 2 r_max */
  uint32_t hash_size; /* n_h of Eq. 6 */
  double cyclic_z[2]; /* cyclic vertical boundary (gear tower, Sec. III): if cyclic_z[1] > cyclic_z[0], a
                         particle below cyclic_z[0] after a step moves up by cyclic_z[1] - cyclic_z[0] */
  int32_t pja_weight; /* effective mass of a contact update: 0 = mass splitting, w = 1 / (n_i/m_i + n_j/m_j)
                         (the reading of Alg. 1 used throughout); 1 = Alg. 1 as printed, where particle i
                         adds the whole projected correction J b to its own velocity: w = m_i for every
                         contact, nothing shared with the partner or among i's contacts (an ablation;
                         free bodies are not supported with it) */
} orc_params;

enum { ORC_PLANE = 0, ORC_BOX = 1, ORC_BOX_MINUS_BOX = 2, ORC_OPEN_BOX = 3, ORC_GRID = 4, ORC_TUBE = 5 };

typedef struct {
  int32_t kind;       /* ORC_* */
  int32_t is_free;    /* 0: kinematic (driven by its twist), 1: free rigid body */
  double shape[12];   /* BOX/OPEN_BOX: half extents [0..2]; BOX_MINUS_BOX: A half [0..2], B half [3..5], B centre [6..8];
                         GRID: body-frame position of sample (0, 0, 0) [0..2], sample spacing h [3];
                         TUBE: radius [0] of the inside of a vertical cylinder (no caps) */
  double pos[3];      /* world position of the body origin */
  double quat[4];     /* orientation (w, x, y, z), body -> world */
  double lin_vel[3];  /* world-frame twist: velocity of the origin ... */
  double ang_vel[3];  /* ... and angular velocity */
  double mass;        /* free bodies only */
  double inertia[3];  /* free bodies only: principal moments in the body frame */
  const float *grid;  /* GRID: SDF samples float[nz][ny][nx], x fastest (Sec. II-C gridded SDF) */
  uint32_t grid_dims[3]; /* GRID: nx, ny, nz (each >= 2) */
} orc_body;

typedef struct {
  int64_t n_pp;        /* directed particle-particle contacts (each pair counted twice) */
  int64_t n_body;      /* particle-body contacts */
  int64_t n_corner;    /* free-box-corner / body contacts */
  int32_t max_pp;      /* largest particle-particle count of one particle */
  int32_t max_body;    /* largest particle-body count of one particle */
  double max_psi;      /* largest penetration depth */
  double ncp_residual; /* fixed-point residual of the last solve (see orc_step) */
} orc_stats;

/* (float)(1/c) in double then rounded: the reciprocal both sides use for binning. */
float orc_inv_cell(float cell_size);

/* Eq. 6 cell index per axis, floor(x * inv_c + 0.5) in FP32 (the paper's round(x / 2r)). */
int32_t orc_cell_index(float x, float inv_cell);

/* Eq. 6 bucket of integer cell (k0, k1, k2): xor of p_j (k_j - q), uint32 wrap, mod n_h. */
uint32_t orc_hash(int32_t k0, int32_t k1, int32_t k2, uint32_t n_h);

/* Bucket of every particle (x: n*3 doubles, rounded to FP32 before binning). */
void orc_cell_keys(uint32_t n, const double *x, float inv_cell, uint32_t n_h, uint32_t *keys);

/* Permutation listing particle ids in ascending (key, id) order. */
void orc_sort_perm(uint32_t n, const uint32_t *keys, uint32_t *perm);

/*
 * Contact lists (Sec. II-B query, Sec. II-C sphere and SDF tests), CSR by particle id.
 * Particle partners ascending by id, then bodies ascending by index.
 * brute != 0 tests every pair instead of walking the 27 neighbour buckets.
 * Any output pointer may be NULL; pass NULL arrays first to learn the totals
 * (returned in st).  pp_geom: 4 per contact (normal from partner into particle, psi).
 * bc_geom: 7 per contact (normal, psi, contact point).  Returns 0 on success.
 */
int orc_contacts(const orc_params *p, uint32_t n, const double *x, const double *r,
                 uint32_t n_bodies, const orc_body *bodies, int brute,
                 uint32_t *pp_off, uint32_t *pp_j, double *pp_geom,
                 uint32_t *bc_off, uint32_t *bc_b, double *bc_geom, orc_stats *st);

/*
 * One time step: contacts, I projected-Jacobi iterations (Alg. 1 read with mass
 * splitting and accumulated-impulse clamping), symplectic Euler (Eq. 4-5).
 * x, v (n*3) and bodies are updated in place.  twist (n_bodies*6, may be NULL)
 * overrides the twist of kinematic bodies for this step.  wrench (n_bodies*6,
 * may be NULL) receives force and torque on each body, = -(sum of impulses
 * given to its contact partners) / dt.  pp_lam / bc_lam (3 per contact, CSR
 * order of orc_contacts, may be NULL) receive the final impulses.  Returns 0, -1 on a
 * contact-capacity failure, -2 for pja_weight = 1 with a free body.
 */
int orc_step(const orc_params *p, uint32_t n, double *x, double *v, const double *r,
             const double *m, uint32_t n_bodies, orc_body *bodies, const double *twist,
             double *wrench, double *pp_lam, double *bc_lam, orc_stats *st);

/*
 * Depth observations (the paper's Sec. III-A "sky" and "ego" cameras), per pixel by
 * brute force.  kind 0 (height): orthographic, looking down; pixel (u, v) samples the
 * point (pos[0] - extent[0]/2 + (u + 1/2) extent[0]/width, pos[1] - ... same in y);
 * its value is the highest particle surface point above it, max z_i + sqrt(r_i^2 - d^2)
 * over spheres whose horizontal distance d to the point is <= r_i (else `empty`).
 * kind 1 (depth): pinhole at pos, orientation quat (camera x right, y down, z along the
 * optical axis), vertical field of view fov_y; pixel (u, v) looks along the unit ray
 * ((u + 1/2 - W/2) / f, (v + 1/2 - H/2) / f, 1), f = (H/2) / tan(fov_y / 2); its value is
 * the distance along the ray to the first surface in [near_clip, far_clip]: spheres
 * exactly, bodies in body_mask by sphere tracing (march_steps steps, hit when the SDF
 * is below march_eps); far_clip if none.  Decisions (coverage, ray-sphere hit, the
 * tracing) are taken in FP32 in a fixed order; sphere values are FP64.
 * out: height * width values, row v = 0 first.
 */
typedef struct {
  int32_t kind, width, height;
  double pos[3], quat[4], extent[2];
  double fov_y, near_clip, far_clip, empty;
  uint32_t body_mask, march_steps;
  double march_eps;
} orc_camera;

void orc_render(const orc_camera *cam, uint32_t n, const double *x, const double *r, uint32_t n_bodies,
                const orc_body *bodies, double *out);

/* Signed distance of world point xw to body b (FP64), for tests and losses. */
double orc_sdf(const orc_body *b, const double *xw, double *normal_world);

/* Smooth mass in the scoop cavity: sum_i m_i sigmoid(-f_B(y_i) / eps), B = cavity box. */
double orc_scoop_loss(uint32_t n, const double *x, const double *m, const orc_body *scoop, double eps);

#ifdef __cplusplus
}
#endif
#endif
