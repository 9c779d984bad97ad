/*
 * gg.h -- C ABI of libgg.so, a GB300 (sm_103a) implementation of the per-time-step
 * granular contact pipeline of GranularGym (arxiv 2306.01369):
 *
 *   bin spheres with the spatial hash of Eq. 6 and a sort        (Sec. II-B, Alg. 2's role)
 *   build particle-particle contacts over the 27 neighbour cells (Sec. II-B, II-C)
 *   build particle-body contacts against signed distance functions (Sec. II-C, Eq. 7)
 *   solve the frictional contact NCP (Eq. 1-3) with projected Jacobi (Alg. 1, Baumgarte)
 *   reduce contact impulses into a wrench per rigid body        (Sec. III-C, force readback)
 *   integrate with symplectic Euler                             (Eq. 4-5)
 *
 * Problem statement (Sec. II): n spheres with positions x and velocities v (3 x n),
 * and rigid bodies with pose X in SE(3) and twist in se(3) that are driven by time
 * (kinematic).  Free rigid bodies that take contact reactions go beyond the paper
 * (its Sec. V names two-way coupling as future work).
 *
 * Conventions
 *  - All arithmetic on the device is FP32.  Arrays are row-major, little-endian.
 *  - Particle arrays passed in or read back are in the caller's particle order
 *    ("id" order), which is also the library's storage order; the bucket sort
 *    produces a list of slots, not a reordered copy of the particles.
 *  - Host pointers are borrowed for the duration of the call only; the library
 *    copies what it needs.  Exception: pinned host buffers given to gg_set_particles
 *    and gg_readback are read or written by work enqueued on the stream, so they must
 *    stay valid (and, for inputs, unchanged) until that work has run.  Device pointers (flag *_on_device != 0) must be
 *    cudaMalloc'ed memory of the current device; they too are read only during the
 *    call (or, for async calls, by work enqueued on the given stream).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Every call returns a gg_status; no C++ exception crosses the ABI.  Device-side
 *    errors (capacity overflow, non-finite state) are latched in a device status
 *    word and reported by the next call that synchronises (gg_sync, gg_readback).
 *  - A gg_sim is not thread-safe; use one host thread per simulation.
 */
#ifndef GG_H
#define GG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GG_ABI_VERSION 2u

/* Only the functions declared here are exported from libgg.so. */
#if defined(__GNUC__)
#define GG_API __attribute__((visibility("default")))
#else
#define GG_API
#endif

typedef struct gg_sim gg_sim;

typedef enum {
  GG_OK = 0,
  GG_ERR_INVALID_ARG = 1,       /* bad pointer, size, parameter or field */
  GG_ERR_OOM = 2,               /* device or host allocation failed */
  GG_ERR_CUDA = 3,              /* a CUDA runtime call failed (see gg_last_error) */
  GG_ERR_CONTACT_OVERFLOW = 4,  /* a particle had more contacts than its capacity */
  GG_ERR_DEVICE_TIMEOUT = 5,    /* a bounded device-side wait gave up */
  GG_ERR_NONFINITE = 6,         /* a position or velocity became NaN or infinite */
  GG_ERR_UNSUPPORTED = 7,       /* valid request the library does not implement */
  GG_ERR_NO_DEVICE = 8,         /* no usable CUDA device */
  GG_ERR_INTERNAL = 9           /* a device-side invariant failed (a bucket list walk longer
                                   than the particle count, or, in a library built with
                                   -DGG_DEBUG, an index check); the access was skipped */
} gg_status;

/* Rigid-body geometry as signed distance functions (Sec. II-C): closed forms, or
 * samples on a regular grid.  Body frame: origin at pos. */
typedef enum {
  GG_BODY_PLANE = 0,          /* half-space z_body <= 0; surface z_body = 0, normal +z_body */
  GG_BODY_BOX = 1,            /* solid box; shape[0..2] = half extents */
  GG_BODY_BOX_MINUS_BOX = 2,  /* box A (half extents shape[0..2]) minus box B (half extents
                                 shape[3..5], centre shape[6..8]): an excavation scoop */
  GG_BODY_OPEN_BOX = 3,       /* container: inside of a box with no lid, walls at x = +-shape[0],
                                 y = +-shape[1], floor at z = -shape[2]; walls are unbounded in +z */
  GG_BODY_GRID = 4,           /* SDF sampled on a regular grid, trilinear interpolation (Sec. II-C);
                                 samples from gg_set_body_grid (shape ignored).  Kinematic only. */
  GG_BODY_TUBE = 5            /* inside of a vertical cylinder of radius shape[0], no caps (the wall
                                 of the gear tower, Sec. III): f = shape[0] - |(y_x, y_y)| */
} gg_body_kind;

typedef struct {
  uint32_t struct_size;      /* sizeof(gg_params): ABI versioning, must be set */
  float dt;                  /* time step Delta t (Alg. 1, Eq. 4-5), > 0 */
  float gravity[3];          /* external acceleration F_ext / m (Eq. 1) */
  float mu;                  /* Coulomb friction coefficient (Eq. 3), >= 0 */
  float alpha;               /* Baumgarte factor: normal bias alpha psi / dt (Sec. II-A), >= 0 */
  uint32_t pja_iters;        /* projected-Jacobi iterations n of Alg. 1, >= 1 */
  float cell_size;           /* grid cell edge c (Eq. 6 uses c = 2r); 0 -> float(2.002 r_max)
                                per environment; otherwise must be >= 2 r_max of every environment */
  uint32_t hash_factor;      /* hash table size n_h = hash_factor * n_env (Sec. II-B proposes 2);
                                0 -> 2; ignored when hash_size != 0 */
  uint32_t hash_size;        /* explicit n_h for every environment (tests); 0 -> hash_factor * n_env.
                                A bucket may hold at most 1024 particles (its own cell's and those
                                of cells sharing its Eq. 6 value): a step whose binning crowds one
                                bucket beyond that (a cell far above 2 r_max, a table far below n)
                                cuts that bucket's walks short and reports GG_ERR_INVALID_ARG */
  uint32_t max_contacts;     /* particle-particle contact capacity per particle, 1..32; 0 -> 16 */
  uint32_t max_body_contacts;/* particle-body contact capacity per particle, 1..8; 0 -> 4 */
  uint32_t max_bodies;       /* bodies per environment, 1..64; 0 -> 8 */
  float density;             /* mass = density 4/3 pi r^3 when no masses are given; 0 -> 2500 */
  uint32_t tuning;           /* 0: the first gg_step times every launch-shape set (binning
                                included) on a copy of the state (restored bit-exactly) and keeps
                                the fastest; k >= 1: fixed set k (see gg_tuning_count; sets 7-9,
                                11-12 bin by linked lists, sets 9, 10, 12 cap the sweep at 40
                                registers, sets 11-13 find pairs over half the stencil and mirror
                                them, sets 14-15 (sort, lists) run detection and every sweep in one
                                cooperative launch, sets 16-18 (sort, lists, lists with the half
                                stencil) reverse every other sweep and preload the first round's
                                records, sets 19-20 (sort, lists) run the paper's OneLoop: every
                                iteration walks the cells again and computes each response as it
                                finds the contact, set 21 is set 11 with 128-thread sweep
                                blocks, set 22 is set 18 with the 40-register sweep and no
                                preloaded round).  Results do not depend on it. */
  uint32_t wrench_history;   /* per-step body wrenches kept for readback; 0 -> 1 */
  uint32_t max_free_bodies;  /* free rigid bodies over all environments (beyond the paper's
                                kinematic bodies, Sec. V two-way coupling); 0 -> none */
  uint32_t free_contact_capacity; /* particle contacts per free body per step, 1..8192; 0 -> 4096 */
  uint32_t barrier_test_phantoms; /* testing aid, 0 in normal use: phantom participants that every
                                     grid barrier of the fused sweep waits for, so each wait runs
                                     out (bounded) and the step reports GG_ERR_DEVICE_TIMEOUT */
  uint32_t binning;          /* 1: counting sort of (bucket, id), contiguous buckets; 2: a lock-free
                                linked list per bucket, the paper's Alg. 2 (pushed with an atomic
                                exchange); 0: either, as the tuning set says (tuning = 0: the
                                autotuner times both).  Results are identical; with lists the
                                sort-order readbacks sort the step's keys on demand. */
  float cyclic_z[2];         /* cyclic vertical boundary (the gear tower of Sec. III): when
                                cyclic_z[1] > cyclic_z[0], a particle whose z falls below cyclic_z[0]
                                in a step moves up by cyclic_z[1] - cyclic_z[0], velocity unchanged.
                                The contact search does not wrap.  {0, 0}: off */
  uint32_t wait_limit_us;    /* bound of every device-side wait (the grid barrier of the fused
                                sweep), microseconds at the SM's maximum clock; past it the step
                                reports GG_ERR_DEVICE_TIMEOUT.  0 -> 500,000 */
  uint32_t hash_tune;        /* 1 (with hash_size = hash_factor = 0): the autotuner also picks n_h
                                among 2n, 4n and 8n per environment (tables sized for 8n), then,
                                when cell_size = 0, the cell edge among 2.002, 2.2 and 2.5 r_max.
                                Positions, velocities and contacts depend on neither; the bucket
                                keys and the sort-order readbacks are those of the n_h and cell
                                edge in use (gg_hash_size, gg_cell_size).  0: both fixed as above */
  uint32_t pja_weight;       /* effective mass of a contact update (Alg. 1): 0 = mass splitting,
                                w = 1 / (n_i/m_i + n_j/m_j) with n_i the contact count of particle i
                                (the library's reading, whose fixed point solves Eq. 1-3); 1 = Alg. 1
                                as printed, where each particle adds the whole projected correction
                                to its own velocity, w = m_i (an ablation: it over-corrects and an
                                isolated pair alternates between bouncing and passing through with
                                the iteration count).  1 is not supported with free bodies or
                                differentiation (GG_ERR_UNSUPPORTED) */
} gg_params;

typedef struct {
  uint32_t kind;             /* gg_body_kind */
  uint32_t is_free;          /* 0: kinematic, follows its twist (paper); 1: free rigid body that
                                takes contact reactions (needs max_free_bodies; box corners also
                                collide with the environment's non-free bodies) */
  float shape[12];           /* see gg_body_kind */
  float pos[3];              /* world position of the body origin (translation of 0_X_b) */
  float quat[4];             /* orientation (w, x, y, z), body -> world; normalised by the library */
  float lin_vel[3];          /* world-frame twist: velocity of the origin ... */
  float ang_vel[3];          /* ... and angular velocity (rad/s) */
  float mass;                /* free bodies: mass (> 0) */
  float inertia[3];          /* free bodies: principal moments of inertia, body frame (> 0) */
} gg_body;

/* Fields for gg_readback.  Sizes: gg_field_bytes().  n = particles, H = hash table
 * entries (all environments), K = max_contacts, Kb = max_body_contacts,
 * B = environments x max_bodies. */
typedef enum {
  GG_FIELD_POS = 0,            /* float[n][4]: x, y, z, radius */
  GG_FIELD_VEL = 1,            /* float[n][3] */
  GG_FIELD_BODY_STATE = 2,     /* float[B][16]: pos[3], quat[4], lin_vel[3], ang_vel[3], 0, 0, 0 */
  GG_FIELD_BODY_WRENCH = 3,    /* float[wrench_history][B][6]: force, torque on each body over the
                                  last wrench_history steps, oldest first, newest in the last row
                                  (rows before the first step are zero) (Sec. III-C force readback) */
  GG_FIELD_CELL_KEY = 4,       /* uint32[n]: hash bucket of each particle at the last binning
                                  (environment base + Eq. 6 value) */
  GG_FIELD_SORT_PERM = 5,      /* uint32[n]: particle ids in ascending (bucket, id) order */
  GG_FIELD_CELL_START = 6,     /* uint32[H + 1]: first sorted slot of each bucket, then n */
  GG_FIELD_CONTACTS = 7,       /* uint32[n][2 + K + Kb]: particle-particle count, particle-body
                                  count, partner ids (ascending), body indices (ascending, local to
                                  the environment); unused entries 0xFFFFFFFF */
  GG_FIELD_CONTACT_GEOM = 8,   /* float[n][K][4]: unit normal from partner into particle, psi */
  GG_FIELD_CONTACT_IMPULSE = 9,/* float[n][K][3]: accumulated impulse on the particle, last solve */
  GG_FIELD_BODY_CONTACT_GEOM = 10, /* float[n][Kb][8]: normal (body into particle), psi, contact point, 0 */
  GG_FIELD_BODY_CONTACT_IMPULSE = 11, /* float[n][Kb][3] */
  GG_FIELD_STATS = 12,         /* gg_stats */
  GG_FIELD_STATE = 13,         /* opaque checkpoint for gg_set_state (bit-exact resume) */
  GG_FIELD_POS_VEL = 14        /* float[n][4] as GG_FIELD_POS, then float[n][3] as GG_FIELD_VEL: both
                                  in one copy and, to the host, one wait (a pinned host buffer,
                                  16-byte aligned, is written by one kernel over the host link) */
} gg_field;

typedef struct {
  uint64_t steps;          /* time steps taken since creation (or the restored checkpoint) */
  uint32_t n_pp;           /* directed particle-particle contacts at the last step (pairs x 2) */
  uint32_t n_body;         /* particle-body contacts at the last step */
  uint32_t max_pp;         /* largest particle-particle count of one particle, last step */
  uint32_t max_body;       /* largest particle-body count of one particle, last step */
  uint32_t status_flags;   /* latched device flags: 1 pp overflow, 2 body overflow, 4 non-finite */
  float max_psi;           /* largest penetration depth at the last step */
  uint32_t n_active;       /* particles with at least one contact at the last step (the others'
                              velocity estimates stay their unconstrained velocity, and the
                              sweeps leave them alone) */
} gg_stats;

GG_API uint32_t gg_abi_version(void);
GG_API const char *gg_status_string(gg_status s);

/*
 * Create a single-environment simulation of n spheres (the problem of Sec. II: sphere
 * positions and velocities, bodies added with gg_set_bodies).
 * pos_radius: float[n][4] (x, y, z, radius > 0); vel: float[n][3] (NULL -> 0);
 * mass: float[n] (> 0; NULL -> density 4/3 pi r^3).  All device memory the step
 * needs is allocated here, at capacity; gg_step allocates nothing.
 * On success *out owns the simulation (free with gg_destroy).
 */
GG_API gg_status gg_create(const gg_params *params, uint32_t n, const float *pos_radius, const float *vel,
                    const float *mass, int inputs_on_device, gg_sim **out);

/*
 * Create n_envs independent environments stepped together (batched mode; the
 * paper's "multiple independent simulations", Sec. III-A).  env_offsets:
 * uint32[n_envs + 1], env e owns particles [env_offsets[e], env_offsets[e+1]),
 * env_offsets[0] = 0, non-decreasing.  Each environment gets its own hash range
 * and bodies; results are bit-identical to stepping each environment alone.
 */
GG_API gg_status gg_create_batch(const gg_params *params, uint32_t n_envs, const uint32_t *env_offsets,
                          const float *pos_radius, const float *vel, const float *mass,
                          int inputs_on_device, gg_sim **out);

/* Replace the bodies of environment env (n_bodies <= max_bodies; host array): rigid
 * bodies with a pose in SE(3), a twist in se(3) and a signed distance function (Sec. II,
 * Sec. II-C).  Synchronous with respect to previously enqueued steps. */
GG_API gg_status gg_set_bodies(gg_sim *sim, uint32_t env, uint32_t n_bodies, const gg_body *bodies);

/*
 * Samples of GG_BODY_GRID body `body` of environment env (Sec. II-C): values =
 * float[dims[2]][dims[1]][dims[0]], x fastest, values[k][j][i] = f at body-frame point
 * origin + spacing (i, j, k); dims >= 2 each, spacing > 0.  A particle's SDF value is
 * the trilinear interpolant of its cell's eight samples, evaluated in FP32 in this
 * order: u = (y - origin) * float(1 / spacing) per axis, cell = floor(u) (at most
 * dims - 2), t = u - cell, lerp(a, b, t) = a + t (b - a) along x, then y, then z; the
 * normal is the interpolant's unit gradient (+z where it vanishes).  Points outside
 * [origin, origin + spacing (dims - 1)] are not in contact, so the samples must
 * extend at least r_max beyond the geometry.  The library copies the samples
 * (allocating device memory outside gg_step); gg_set_bodies drops them.
 */
GG_API gg_status gg_set_body_grid(gg_sim *sim, uint32_t env, uint32_t body, const uint32_t dims[3],
                                  const float origin[3], float spacing, const float *values, int on_device);

/*
 * Prescribe the twist of kinematic body `body` of environment env for the next
 * n_steps steps (the paper's bodies are driven by time, Sec. II): twist = float[n_steps][6] (world-frame lin_vel, ang_vel), step k
 * counted from the current step.  Past the table the body keeps its own twist.
 * Allocates device memory (outside gg_step).
 */
GG_API gg_status gg_set_trajectory(gg_sim *sim, uint32_t env, uint32_t body, uint32_t n_steps,
                            const float *twist, int twist_on_device);

/* Overwrite particle positions/radii (float[n][4]) and velocities (float[n][3]; NULL
 * keeps them), asynchronously on `stream` (the state x, v of Sec. II).  Returns
 * GG_ERR_INVALID_ARG for a null position buffer.  Masses are kept.  Host buffers that are
 * pinned (cudaHostAlloc, cudaHostRegister; positions 16-byte aligned) are read by one
 * kernel over the host link; pageable ones are copied.  Either way the caller's buffers
 * must stay unchanged until the work on `stream` has run. */
GG_API gg_status gg_set_particles(gg_sim *sim, const float *pos_radius, const float *vel, int on_device,
                           void *stream);

/* Enqueue n_steps time steps on `stream`: each one binning (Eq. 6), contacts (Sec. II-B,
 * II-C, Eq. 7), the projected-Jacobi sweeps (Alg. 1), the wrenches (Sec. III-C) and the
 * integration (Eq. 4-5), replayed from one captured CUDA graph.  Returns without
 * waiting; see gg_sync for device-side errors. */
GG_API gg_status gg_step(gg_sim *sim, uint32_t n_steps, void *stream);

/* Wait for `stream` and report the latched device status (GG_OK or the first error).
 * Library plumbing; the paper has no counterpart. */
GG_API gg_status gg_sync(gg_sim *sim, void *stream);

/*
 * One turn of a host-driven loop (an environment that exchanges the state with its
 * caller every step, as the paper's learning tasks do, Sec. III-A): the particle state
 * from host buffers (pos_radius
 * float[n][4], vel float[n][3] or NULL to keep the velocities), one time step, and the
 * new state into out (float[7 n]: positions float[n][4], then velocities float[n][3],
 * the GG_FIELD_POS_VEL layout), waited for.  The same work and results, bit for bit, as
 * gg_set_particles + gg_step(1) + gg_readback(GG_FIELD_POS_VEL).  When all three host
 * buffers are pinned (positions and out 16-byte aligned) and stage timing is off, the
 * transfers and the step are one graph (kept while the buffers' device addresses and
 * the launch shape stay the same); otherwise the three calls run.  Host buffers only
 * (device tensors: the three calls).  Returns the step's status like gg_readback.
 */
GG_API gg_status gg_step_io(gg_sim *sim, const float *pos_radius, const float *vel, float *out, void *stream);

/* Size in bytes of a readback field (0 for a null simulation or an unknown field). */
GG_API size_t gg_field_bytes(const gg_sim *sim, gg_field field);

/*
 * Copy `field` into dst (bytes must equal gg_field_bytes, else GG_ERR_INVALID_ARG):
 * the state x, v (Sec. II), the body wrenches (Sec. III-C force readback), the binning
 * of Eq. 6, the contacts and their impulses (Alg. 1).  dst on the device:
 * asynchronous on `stream`; on the host: waits for `stream`.  Returns the latched
 * device status when it waited (the copy is made either way).
 */
GG_API gg_status gg_readback(gg_sim *sim, gg_field field, void *dst, size_t bytes, int dst_on_device,
                      void *stream);

/*
 * Depth observations computed on the device (Sec. III-A: the "sky" and "ego" cameras).
 *  GG_CAMERA_HEIGHT: orthographic, looking down.  Pixel (u, v) samples the point
 *    (pos[0] - extent[0]/2 + (u + 1/2) extent[0]/width, pos[1] - extent[1]/2 + (v + 1/2)
 *    extent[1]/height) (FP32, in that order); its value is the highest particle surface
 *    above it, max z_i + sqrt(r_i^2 - d^2) over the spheres whose horizontal distance d
 *    to the point is <= r_i, else `empty`.
 *  GG_CAMERA_DEPTH: pinhole at pos with orientation quat (unit; camera -> world; camera
 *    x right, y down, z along the optical axis), vertical field of view fov_y.  Pixel
 *    (u, v) looks along the unit ray ((u + 1/2 - width/2)/f, (v + 1/2 - height/2)/f, 1),
 *    f = (height/2) / tan(fov_y/2); its value is the distance along the ray to the first
 *    surface in [near_clip, far_clip]: spheres exactly, the bodies in body_mask (bit b =
 *    body b of the environment, b < 32) by sphere tracing (march_steps steps from
 *    near_clip, a hit when the SDF falls below march_eps); far_clip if none.
 * Images are float[height][width], row v = 0 first, at most 4096 x 4096.
 */
typedef enum { GG_CAMERA_HEIGHT = 0, GG_CAMERA_DEPTH = 1 } gg_camera_kind;

typedef struct {
  uint32_t struct_size;  /* sizeof(gg_camera) */
  uint32_t kind;         /* gg_camera_kind */
  uint32_t width, height;
  float pos[3];          /* DEPTH: camera origin; HEIGHT: centre of the image rectangle (x, y) */
  float quat[4];         /* DEPTH: orientation (w, x, y, z), camera -> world */
  float extent[2];       /* HEIGHT: rectangle size along world x and y */
  float fov_y;           /* DEPTH: radians, in (0, pi) */
  float near_clip, far_clip;  /* DEPTH: 0 < near_clip < far_clip */
  float empty;           /* HEIGHT: value of pixels no particle covers */
  uint32_t body_mask;    /* DEPTH */
  uint32_t march_steps;  /* DEPTH: 0 -> 64 */
  float march_eps;       /* DEPTH: 0 -> 1e-4 */
} gg_camera;

/* Render environment env's current state into out (float[height][width]); out on the
 * device: asynchronous on `stream`, else waits.  May allocate a scratch image (outside
 * gg_step). */
GG_API gg_status gg_render(gg_sim *sim, uint32_t env, const gg_camera *camera, float *out, int out_on_device,
                           void *stream);

/* Restore a GG_FIELD_STATE checkpoint taken from a simulation with the same sizes
 * (GG_ERR_INVALID_ARG otherwise).  Checkpoint and resume: beyond the paper. */
GG_API gg_status gg_set_state(gg_sim *sim, const void *state, size_t bytes, int on_device, void *stream);

/*
 * Stage timing (measurement; the paper has no counterpart).  gg_enable_timing(sim, 1) records CUDA events inside every
 * subsequent step: the library keeps a second step graph with the events (captured
 * at its first use; switching back and forth afterwards costs nothing), and
 * gg_enable_timing(sim, 0) returns to the plain one.  The events break the
 * overlap of consecutive kernels at stage boundaries, so an instrumented step is
 * slower (~18 us on a 262,144-sphere step).  gg_stage_ms then waits for the
 * last enqueued step and writes its device time in milliseconds per stage into
 * ms[GG_NUM_STAGES]: binning + sort, contact build, all projected-Jacobi
 * iterations, integration + wrench.  Returns GG_ERR_INVALID_ARG when timing is off.
 */
#define GG_NUM_STAGES 4
GG_API gg_status gg_enable_timing(gg_sim *sim, int on);
GG_API gg_status gg_stage_ms(gg_sim *sim, float *ms);

/* Kernel launches one step enqueues (all of them this library's own kernels; 0 for a
 * null simulation).  Measurement; the paper has no counterpart. */
GG_API uint32_t gg_kernels_per_step(const gg_sim *sim);

/*
 * Differentiation (beyond the paper, whose Sec. V lists it as future work).
 * Reverse-mode gradients of a loss on the final state w.r.t. the per-step twists of
 * one kinematic body (the tool) and w.r.t. mu, through contact generation, the
 * projected-Jacobi iterations and the integrator, with the contact set and the
 * active set of every projection fixed as the forward found them (piecewise
 * differentiation).  Single environment, kinematic bodies only.
 *
 * gg_tape_reserve: allocate checkpoint and tape memory for n_steps taped steps with a
 *   full-state checkpoint every `checkpoint_every` steps (recompute in between).  The
 *   reverse pass recomputes a segment once, keeping every step's contact arrays and
 *   iterates, so the tape memory is min(checkpoint_every, n_steps) step tapes of
 *   about n ((I + 1) (16 + 12 K + 12 Kb) + 20 K + 36 Kb + 4) bytes each (K, Kb: the
 *   contact capacities, I: the sweeps per step); GG_ERR_OOM if it does not fit
 *   (a smaller checkpoint_every needs less).
 * gg_step_taped: enqueue n_steps (<= reserved) forward steps saving the checkpoints;
 *   the tool's twist for those steps must come from gg_set_trajectory.
 * gg_backward: gradients of L given dL/dx_N (float[n][3]), dL/dv_N (float[n][3]; NULL
 *   = 0) and dL/d(tool pose at N) (float[7]: d/dpos[3], d/dquat[4] with quat (w,x,y,z);
 *   NULL = 0), N = the end of the taped run.  Writes dL/dtwist (float[n_steps][6]:
 *   d/dlin_vel, d/dang_vel, world frame) and dL/dmu (float[1]).  Inputs and outputs
 *   on the device when on_device != 0.  Re-runs the forward from the checkpoints and
 *   leaves the simulation in its end-of-run state, also when it returns an error
 *   partway through the reverse pass (the end state is copied back before the return;
 *   after a GG_ERR_CUDA that copy may itself have failed, and the state is then
 *   undefined).  Synchronises `stream`.
 */
GG_API gg_status gg_tape_reserve(gg_sim *sim, uint32_t n_steps, uint32_t checkpoint_every);
GG_API gg_status gg_step_taped(gg_sim *sim, uint32_t tool_body, uint32_t n_steps, void *stream);
GG_API gg_status gg_backward(gg_sim *sim, const float *dL_dpos, const float *dL_dvel, const float *dL_dpose,
                             float *dL_dtwist, float *dL_dmu, int on_device, void *stream);

/* Hash table size n_h in use for environment `env` (Eq. 6's modulus); 0 for a bad
 * argument. */
GG_API uint32_t gg_hash_size(const gg_sim *sim, uint32_t env);

/* Cell edge c in use for environment `env` (Eq. 6's 2r, the grid the keys are computed
 * on); 0 for a bad argument. */
GG_API float gg_cell_size(const gg_sim *sim, uint32_t env);

/* Number of fixed launch-shape sets accepted by gg_params.tuning, and the set chosen
 * (the paper's loop-structure and binning choices, Sec. II-D, Alg. 2, among them). */
GG_API uint32_t gg_tuning_count(void);
GG_API uint32_t gg_tuning_selected(const gg_sim *sim);

/* What set k (1..gg_tuning_count()) does, as GG_TUNE_* bits; 0 when k is out of range.
 * Every set gives the same results; the bits only describe how the step is launched. */
#define GG_TUNE_LISTS 1u /* binning by per-bucket linked lists (else the counting sort) */
#define GG_TUNE_FUSED 2u /* all sweeps in one cooperative launch with grid barriers */
#define GG_TUNE_LEAN 4u  /* the sweep capped at 40 registers */
#define GG_TUNE_HALF 8u  /* pair search over half the stencil, then a mirroring pass */
#define GG_TUNE_DETECT 16u /* detection and all sweeps in one cooperative launch, a grid barrier
                              between them (the paper's TwoLoopsFused, Sec. II-D); without free
                              bodies (with them the set runs the split launches) */
#define GG_TUNE_SERP 32u   /* serpentine sweeps: every other sweep visits the particles in reverse,
                              starting on the data the previous stage left in L2 */
#define GG_TUNE_PRELOAD 64u /* the sweep loads the records of the first two contact slots
                               together with the counts */
#define GG_TUNE_ONELOOP 128u /* OneLoop (Sec. II-D): each iteration re-walks the neighbour cells
                                and computes the responses there, not from stored records */

GG_API uint32_t gg_tuning_flags(uint32_t k);

/* Time every launch-shape set gg_params.binning allows on the current state (3 steps
 * each, the state restored bit-exactly before each trial and at the end) and keep the
 * fastest; with gg_params.hash_tune, then time that set at n_h = 4n and 8n as well and
 * keep the fastest table size.  gg_step does this once, on its first call, when gg_params.tuning = 0; call
 * it again when the workload changes character (a bed that has settled, a tool that
 * starts digging).  A no-op when gg_params.tuning fixes the set.  Waits for `stream`;
 * allocates a state copy for the duration of the call. */
GG_API gg_status gg_autotune(gg_sim *sim, void *stream);

/* Last error message of this simulation (never NULL). */
GG_API const char *gg_last_error(const gg_sim *sim);  /* plumbing; no counterpart in the paper */

/* Free the simulation and all its device memory (NULL: no-op).  Plumbing; no
 * counterpart in the paper. */
GG_API void gg_destroy(gg_sim *sim);

/*
 * Binning and bucket sort of one particle set with no device allocation.
 * The paper has no counterpart: this is a library convenience for callers that
 * cannot allocate device memory themselves or let a library do it (code running
 * inside a framework's memory pool, allocator-free real-time loops, plug-ins
 * handed device pointers only).  It computes what one step's binning computes
 * for a single environment -- the Eq. 6 bucket of every particle, the particle
 * ids in ascending (bucket, id) order, and the bucket start table -- and gives
 * the same values as GG_FIELD_CELL_KEY, GG_FIELD_SORT_PERM and
 * GG_FIELD_CELL_START of a gg_sim with the same positions, cell_size and
 * hash_size.
 *
 * pos_radius: device float[n][4]; keys, perm: device uint32[n]; cell_start: device
 * uint32[n_h + 1]; all caller-owned, on the current device; enqueued on `stream`.
 * Limits: n <= GG_NOALLOC_MAX_PARTICLES, 1 <= n_h <= GG_NOALLOC_MAX_BUCKETS, else
 * GG_ERR_INVALID_ARG (nothing is enqueued).  Calls no cudaMalloc or cudaFree.
 * Bucket occupancy: ordering a bucket by id costs its occupancy per particle, so a
 * bucket holding more than GG_NOALLOC_MAX_OCCUPANCY particles is not ordered: its
 * ids appear in perm in an unspecified order (still exactly the bucket's members;
 * keys and cell_start stay exact, and cell_start shows which buckets these are).
 * With cell_size near 2 r_max and n_h >= n a bucket holds a few particles.
 * Scratch: a fixed static device array of about 12.6 MB that every GPU which loads
 * libgg.so holds until the process exits; every call on a device reuses it and
 * clears its histogram first, so calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  The first call
 * on each device looks up that array's device address (with the device current);
 * make that first call before any CUDA stream capture.
 */
#define GG_NOALLOC_MAX_PARTICLES (1u << 20)
#define GG_NOALLOC_MAX_BUCKETS (1u << 21)
#define GG_NOALLOC_MAX_OCCUPANCY 1024u
GG_API gg_status gg_bin_sort_noalloc(const float *pos_radius, uint32_t n, float cell_size, uint32_t n_h,
                                     uint32_t *keys, uint32_t *perm, uint32_t *cell_start, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GG_H */
