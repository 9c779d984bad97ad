// gg_device.cuh -- device-side layout and FP32 helpers of the granular contact step.
//
// Integer decisions (cell index, hash bucket, contact yes/no, active SDF branch)
// use explicitly rounded FP32 intrinsics (__fmul_rn, __fadd_rn, __fsub_rn,
// __fsqrt_rn) so that nvcc cannot contract them into FMAs: the result is then a
// function of the FP32 inputs alone, fixed by the evaluation order written here.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gg {

constexpr uint32_t kHashP1 = 73856093u;  // Eq. 6 primes
constexpr uint32_t kHashP2 = 19349663u;
constexpr uint32_t kHashP3 = 83492791u;
constexpr uint32_t kHashQ = 100u;        // Eq. 6 offset q

constexpr uint32_t kFlagPPOverflow = 1u;
constexpr uint32_t kFlagBodyOverflow = 2u;
constexpr uint32_t kFlagNonFinite = 4u;
constexpr uint32_t kFlagTimeout = 8u;    // a bounded device-side wait gave up
constexpr uint32_t kFlagListBound = 16u; // a bucket list walk passed n entries (lists not emptied)
constexpr uint32_t kFlagDebugCheck = 32u; // an index check of the GG_DEBUG build failed
constexpr uint32_t kFlagBucketBound = 64u; // a bucket held more than kMaxBucket particles

// Most particles one bucket may hold.  With cells of about 2 r_max a bucket holds a
// particle or two (its own cell's, plus those of cells that share its Eq. 6 value);
// only a cell size far above 2 r_max or a table far smaller than n crowds one.  The
// in-bucket ordering and every bucket walk stop at this many entries and latch
// kFlagBucketBound, so a crowded bucket costs at most this much work per particle
// and the step reports an error instead of running for minutes.
constexpr uint32_t kMaxBucket = 1024;

constexpr uint32_t kListEnd = 0xffffffffu;  // end of a bucket's linked list
constexpr int kMaxK = 32;   // particle-particle capacity limit
constexpr int kMaxKb = 8;   // particle-body capacity limit
constexpr int kScanItems = 16;          // counts per thread in the bucket scan
constexpr int kScanThreads = 256;
constexpr int kScanTile = kScanItems * kScanThreads;
constexpr int kWrenchChunk = 1024;      // particles per wrench partial

struct DevEnv {
  uint32_t off, n;        // particle range [off, off + n)
  uint32_t hbase, nh;     // bucket range [hbase, hbase + nh)
  float inv_cell;         // float(1 / c)
  uint32_t nbodies;       // active bodies (slots [e * maxb, e * maxb + nbodies))
  uint32_t chunk0, nchunks;  // wrench partial chunks of this environment
  uint64_t nh_magic;      // floor((2^64 - 1) / nh) + 1, for the exact remainder below
};

// x mod d without a division: Lemire, Kaser & Kurz, "Faster remainder by direct
// computation" (Software: Practice and Experience, 2019); exact for all 32-bit x and d
// >= 1 with magic = floor((2^64 - 1) / d) + 1 (wrapping to 0 for d = 1).
__host__ __device__ __forceinline__ uint64_t remainder_magic(uint32_t d) { return ~0ull / d + 1ull; }
__device__ __forceinline__ uint32_t fast_mod(uint32_t x, uint64_t magic, uint32_t d) {
  const uint64_t low = magic * (uint64_t)x;
  return (uint32_t)__umul64hi(low, (uint64_t)d);
}

struct DevBody {
  uint32_t kind, is_free;
  float shape[12];
  float p[3];       // pose at the start of the current step
  float q[4];       // (w, x, y, z)
  float R[9];       // rotation of q, row-major, body -> world, FP32 fixed order
  float v[3], w[3]; // twist used during the current step
  float own_v[3], own_w[3];  // the body's own twist (kinematic), or its state (free)
  float mass, inertia[3];
  const float *traj;  // float[traj_len][6] or null
  uint32_t traj_len;
  uint32_t traj_start;  // step index at which traj[0] applies
  uint32_t env, active;
  uint32_t fid;         // free bodies: index into the free-body arrays
  // kind 4 (grid): samples float[gn[2]][gn[1]][gn[0]]; shape[0..2] origin, shape[3]
  // spacing h, shape[4] float(1 / h)
  const float *grid;
  uint32_t gn[3];
  // radius about p outside which the body's SDF exceeds the distance beyond this radius
  // (closed solids: box, box minus box, sampled grids; 0 for unbounded bodies): a
  // particle farther than bound_r + r from p cannot touch it, so its SDF is not evaluated
  float bound_r;
};

// Programmatic dependent launch (sm_90 and later).  A kernel launched with programmatic
// stream serialization may be scheduled while its predecessor in the stream drains; it
// touches no memory before griddepcontrol.wait, which returns once the predecessor grid
// has completed and its writes are visible.  launch_dependents, issued right after,
// lets the successor's blocks be scheduled once every block of this grid has issued
// it.  For a normal launch both are no-ops.  Every kernel of the step calls this first.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory");
}

// A corner of a free box touching a non-free body of its environment.
struct CornerContact {
  uint32_t o, valid;
  float n[3], psi;   // normal (other body -> box), penetration
  float xc[3];       // contact point
  float lam[3];      // accumulated impulse on the box
};

struct DevCtrl {
  uint32_t step;      // steps taken (low 32 bits)
  uint32_t status;    // latched flags
  uint32_t n_pp, n_body, max_pp, max_body;
  uint32_t max_psi_bits;  // max psi as the bits of a non-negative float
  uint32_t bar_count;     // grid barrier: arrivals in the current round
  uint32_t bar_gen;       // grid barrier: completed rounds
  uint32_t bar_abort;     // set when a barrier wait gave up (later barriers return at once)
  uint32_t bar_extra;     // phantom arrivals a barrier waits for (0; tests set it to force a timeout)
  uint32_t blocks_done;     // k_wrench_bodies: blocks finished this step (0 between steps)
  uint32_t n_active;        // particles with at least one contact this step
};

// Index checks of the debug build (-DGG_DEBUG): GG_GUARD(ctrl, cond) is `cond`, and a
// false `cond` also latches kFlagDebugCheck (the step then reports GG_ERR_INTERNAL);
// callers skip the access it guards.  In the release build it is `true` and costs
// nothing.  (compute-sanitizer is not available to this build's tests; these checks
// and the invariance tests stand in for it.)
#ifdef GG_DEBUG
__device__ __forceinline__ bool gg_guard(DevCtrl *c, bool ok) {
  if (!ok) atomicOr(&c->status, kFlagDebugCheck);
  return ok;
}
#define GG_GUARD(ctrl, cond) ::gg::gg_guard((ctrl), (cond))
#else
#define GG_GUARD(ctrl, cond) true
#endif

// Everything a step's kernels read or write; passed by value to each kernel.
struct StepArgs {
  uint32_t n, n_envs, nh_total, nh_pad, maxb, K, Kb, n_chunks, wrench_hist;
  float dt, mu, ab;       // ab = alpha / dt
  float g[3];
  float cyc_lo, cyc_h;    // cyclic vertical boundary: z < cyc_lo moves up by cyc_h (cyc_h > 0), else off
  long long wait_cycles;  // bound of device-side waits (SM clock cycles)
  uint32_t lists;         // binning: 0 counting sort (contiguous buckets), 1 linked lists (Alg. 2)
  uint32_t lit;           // contact weight: 0 mass splitting (U.w = n_i / m_i, w = 1 / (U_i.w + U_j.w));
                          // 1 Alg. 1 as printed (U.w = 1 / m_i, w = 1 / U_i.w = m_i)
  uint32_t *head;         // lists: first particle of each bucket (kListEnd: empty), nh_pad entries
  uint32_t *next;         // lists: next particle of the same bucket, [n]
  uint32_t *pcnt;         // half-stencil pair search: entries per particle (0 between steps), [n]
  uint32_t *pscr;         // half-stencil pair search: unsorted partners, [2K][n]
  // id order
  float4 *pos_id;   // x, y, z, r
  float4 *vel_id;   // vx, vy, vz, 1/m
  uint32_t *env_of;
  uint32_t *key_id;
  // buckets
  uint32_t *cnt;    // nh_pad entries, zero between steps
  uint32_t *start;  // nh_pad + 1
  uint2 *range;     // nh_pad: (start, end) of every bucket, one load in the bucket walk
  uint32_t *bsum;   // scan block sums
  // sorted slots: particle id of each slot, ascending (bucket, id), and that
  // particle's position (the bucket walk reads candidates without an id hop)
  uint32_t *sid_tmp, *sid;
  float4 *pos_s;
  // per particle (id order)
  float4 *U[2];     // velocity estimate, w = n_contacts / m
  uint32_t *ccount; // pp | body << 8
  uint32_t *cj;     // [K][n] partner id
  float4 *cn;       // [K][n] normal (partner -> particle), psi
  float *clam;      // [3][K][n]
  uint32_t *bj;     // [Kb][n] global body index
  float4 *bn;       // [Kb][n] normal (body -> particle), psi
  float4 *bxc;      // [Kb][n] contact point
  float *blam;      // [3][Kb][n]
  // environments and bodies
  DevEnv *envs;
  DevBody *bodies;
  uint32_t *chunk_env;    // environment of each wrench chunk
  float *wpart;           // [n_chunks][maxb][6]
  float *wrench;          // [wrench_hist][n_envs * maxb][6]
  DevCtrl *ctrl;
  // free rigid bodies
  uint32_t F, Lcap;       // free-body slots, contact-list capacity per free body
  uint32_t *ncb;          // [n_envs * maxb] contacts per body this step
  uint32_t *fcount;       // [F] particle contacts of each free body
  uint32_t *flist;        // [F][Lcap] (particle * Kb + k), sorted ascending
  uint32_t *fgb;          // [F] global body index of each free slot (or ~0u)
  CornerContact *fcc;     // [F][8 * maxb]
};

// ---------------------------------------------------------------------------
// FP32 decisions
// ---------------------------------------------------------------------------

__device__ __forceinline__ int32_t cell_of(float x, float inv_cell) {
  float t = __fmul_rn(x, inv_cell);
  t = __fadd_rn(t, 0.5f);
  return (int32_t)floorf(t);
}

__device__ __forceinline__ uint32_t hash_cell(int32_t k0, int32_t k1, int32_t k2, uint32_t nh) {
  uint32_t a = ((uint32_t)k0 - kHashQ) * kHashP1;
  uint32_t b = ((uint32_t)k1 - kHashQ) * kHashP2;
  uint32_t c = ((uint32_t)k2 - kHashQ) * kHashP3;
  return (a ^ b ^ c) % nh;
}

// Eq. 6 with the exact fast remainder; same value as hash_cell.
// Eq. 6's "mod n_h" of a hash value: a mask when n_h is a power of two (the paper's
// 2n heuristic gives one for power-of-two n), else the exact remainder above.
__device__ __forceinline__ uint32_t mod_nh(uint32_t h, const DevEnv &E) {
  return (E.nh & (E.nh - 1u)) == 0u ? (h & (E.nh - 1u)) : fast_mod(h, E.nh_magic, E.nh);
}

__device__ __forceinline__ uint32_t hash_cell_fm(int32_t k0, int32_t k1, int32_t k2, const DevEnv &E) {
  const uint32_t a = ((uint32_t)k0 - kHashQ) * kHashP1;
  const uint32_t b = ((uint32_t)k1 - kHashQ) * kHashP2;
  const uint32_t c = ((uint32_t)k2 - kHashQ) * kHashP3;
  return mod_nh(a ^ b ^ c, E);
}

// squared distance ((dx dx + dy dy) + dz dz) and the sum of radii squared
__device__ __forceinline__ bool sphere_hit(float4 a, float4 b, float *d2out, float3 *dout) {
  float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
  float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  float rs = __fadd_rn(a.w, b.w);
  *d2out = d2;
  *dout = make_float3(dx, dy, dz);
  return d2 <= __fmul_rn(rs, rs);
}

__device__ __forceinline__ void quat_to_R(const float *q, float *R) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  R[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
  R[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
  R[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
  R[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
  R[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
  R[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
  R[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
  R[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
  R[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
}

// y = R^T (x - p), each component summed R[0k]d0 + R[1k]d1 first, then + R[2k]d2
__device__ __forceinline__ float3 world_to_body(const DevBody &b, float3 x) {
  float d0 = __fsub_rn(x.x, b.p[0]), d1 = __fsub_rn(x.y, b.p[1]), d2 = __fsub_rn(x.z, b.p[2]);
  float y[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    y[k] = __fadd_rn(__fadd_rn(__fmul_rn(b.R[k], d0), __fmul_rn(b.R[3 + k], d1)), __fmul_rn(b.R[6 + k], d2));
  return make_float3(y[0], y[1], y[2]);
}

// Box SDF: branch 0..2 inside (nearest face axis), 3 outside.
__device__ __forceinline__ float box_sdf(float3 y, const float *h, int *branch) {
  float q0 = __fsub_rn(fabsf(y.x), h[0]);
  float q1 = __fsub_rn(fabsf(y.y), h[1]);
  float q2 = __fsub_rn(fabsf(y.z), h[2]);
  float m0 = fmaxf(q0, 0.0f), m1 = fmaxf(q1, 0.0f), m2 = fmaxf(q2, 0.0f);
  float s = __fadd_rn(__fadd_rn(__fmul_rn(m0, m0), __fmul_rn(m1, m1)), __fmul_rn(m2, m2));
  float o = __fsqrt_rn(s);
  float mx = fmaxf(fmaxf(q0, q1), q2);
  float f = __fadd_rn(o, fminf(mx, 0.0f));
  *branch = (mx > 0.0f) ? 3 : ((q0 >= q1 && q0 >= q2) ? 0 : ((q1 >= q2) ? 1 : 2));
  return f;
}

// Gridded SDF (Sec. II-C): trilinear interpolation of the eight samples of y's cell, in
// FP32 and in this order: u = (y - o) * float(1/h); cell = floor(u) (at most n - 2);
// t = u - cell; lerp(a, b, t) = a + t (b - a) along x (four edges), then y, then z.
// Outside the sampled box (or NaN): +inf, branch -1; inside, branch = the cell index.
__device__ __forceinline__ float lerp_rn(float a, float b, float t) {
  return __fadd_rn(a, __fmul_rn(t, __fsub_rn(b, a)));
}

struct GridCell {
  int32_t i[3];
  float t[3];
};

__device__ __forceinline__ bool grid_cell(const DevBody &b, float3 y, GridCell *c) {
  const float yy[3] = {y.x, y.y, y.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = __fmul_rn(__fsub_rn(yy[k], b.shape[k]), b.shape[4]);
    if (!(u >= 0.0f && u <= (float)(b.gn[k] - 1u))) return false;
    int32_t ik = (int32_t)floorf(u);
    if (ik > (int32_t)b.gn[k] - 2) ik = (int32_t)b.gn[k] - 2;
    c->i[k] = ik;
    c->t[k] = __fsub_rn(u, (float)ik);
  }
  return true;
}

__device__ __forceinline__ float grid_sdf(const DevBody &b, float3 y, int *branch) {
  GridCell c;
  if (!b.grid || !grid_cell(b, y, &c)) {
    *branch = -1;
    return __int_as_float(0x7f800000);
  }
  const size_t nx = b.gn[0], nxy = (size_t)b.gn[0] * b.gn[1];
  const size_t base = (size_t)c.i[2] * nxy + (size_t)c.i[1] * nx + (size_t)c.i[0];
  const float *v = b.grid + base;
  const float c00 = lerp_rn(v[0], v[1], c.t[0]);
  const float c10 = lerp_rn(v[nx], v[nx + 1], c.t[0]);
  const float c01 = lerp_rn(v[nxy], v[nxy + 1], c.t[0]);
  const float c11 = lerp_rn(v[nxy + nx], v[nxy + nx + 1], c.t[0]);
  *branch = (int)base;
  return lerp_rn(lerp_rn(c00, c10, c.t[1]), lerp_rn(c01, c11, c.t[1]), c.t[2]);
}

// Gradient of the trilinear interpolant of the cell (per unit t, i.e. h times the
// gradient in y) and, when hess != nullptr, its mixed second derivatives per unit t:
// hess = (d2f/dtx dty, d2f/dtx dtz, d2f/dty dtz) (the pure ones vanish).
__device__ __forceinline__ float3 grid_dt(const DevBody &b, float3 y, int branch, float3 *hess) {
  const size_t nx = b.gn[0], nxy = (size_t)b.gn[0] * b.gn[1];
  const float *v = b.grid + (size_t)branch;
  float t[3];
  const float yy[3] = {y.x, y.y, y.z};
  const int32_t i[3] = {(int32_t)((size_t)branch % nx), (int32_t)(((size_t)branch / nx) % b.gn[1]),
                        (int32_t)((size_t)branch / nxy)};
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = (yy[k] - b.shape[k]) * b.shape[4] - (float)i[k];
  float s[2][2][2];
#pragma unroll
  for (int cz = 0; cz < 2; ++cz)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) s[cz][cy][cx] = v[cz * nxy + cy * nx + cx];
  const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
  float3 g = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int cz = 0; cz < 2; ++cz)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) g.x += (s[cz][cy][1] - s[cz][cy][0]) * wy[cy] * wz[cz];
#pragma unroll
  for (int cz = 0; cz < 2; ++cz)
#pragma unroll
    for (int cx = 0; cx < 2; ++cx) g.y += (s[cz][1][cx] - s[cz][0][cx]) * wx[cx] * wz[cz];
#pragma unroll
  for (int cy = 0; cy < 2; ++cy)
#pragma unroll
    for (int cx = 0; cx < 2; ++cx) g.z += (s[1][cy][cx] - s[0][cy][cx]) * wx[cx] * wy[cy];
  if (hess) {
    float hxy = 0.f, hxz = 0.f, hyz = 0.f;
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      hxy += (s[c2][1][1] - s[c2][1][0] - s[c2][0][1] + s[c2][0][0]) * wz[c2];
      hxz += (s[1][c2][1] - s[1][c2][0] - s[0][c2][1] + s[0][c2][0]) * wy[c2];
      hyz += (s[1][1][c2] - s[1][0][c2] - s[0][1][c2] + s[0][0][c2]) * wx[c2];
    }
    *hess = make_float3(hxy, hxz, hyz);
  }
  return g;
}

__device__ __forceinline__ float body_sdf(const DevBody &b, float3 y, int *branch) {
  switch (b.kind) {
  case 0:  // plane
    *branch = 0;
    return y.z;
  case 1:  // box
    return box_sdf(y, b.shape, branch);
  case 2: {  // box minus box
    int ba, bb;
    float fa = box_sdf(y, b.shape, &ba);
    float3 z = make_float3(__fsub_rn(y.x, b.shape[6]), __fsub_rn(y.y, b.shape[7]), __fsub_rn(y.z, b.shape[8]));
    float nfb = -box_sdf(z, b.shape + 3, &bb);
    if (fa >= nfb) {
      *branch = ba;
      return fa;
    }
    *branch = 4 + bb;
    return nfb;
  }
  case 3: {  // open box (container)
    float w[5] = {__fsub_rn(b.shape[0], y.x), __fadd_rn(y.x, b.shape[0]), __fsub_rn(b.shape[1], y.y),
                  __fadd_rn(y.y, b.shape[1]), __fadd_rn(y.z, b.shape[2])};
    float f = w[0];
    int br = 0;
#pragma unroll
    for (int k = 1; k < 5; ++k)
      if (w[k] < f) {
        f = w[k];
        br = k;
      }
    *branch = br;
    return f;
  }
  case 4:
    return grid_sdf(b, y, branch);
  case 5:  // tube: inside of a vertical cylinder, f = R - |(y_x, y_y)|
    *branch = 0;
    return __fsub_rn(b.shape[0], __fsqrt_rn(__fadd_rn(__fmul_rn(y.x, y.x), __fmul_rn(y.y, y.y))));
  }
  *branch = -1;
  return __int_as_float(0x7f800000);  // +inf: never in contact
}

// Unit gradient (body frame) of the branch chosen by body_sdf.
__device__ __forceinline__ float3 box_grad(float3 y, const float *h, int branch) {
  if (branch == 3) {
    float m0 = fmaxf(fabsf(y.x) - h[0], 0.0f), m1 = fmaxf(fabsf(y.y) - h[1], 0.0f),
          m2 = fmaxf(fabsf(y.z) - h[2], 0.0f);
    float inv = rsqrtf(m0 * m0 + m1 * m1 + m2 * m2);
    return make_float3(copysignf(m0 * inv, y.x), copysignf(m1 * inv, y.y), copysignf(m2 * inv, y.z));
  }
  float3 g = make_float3(0.f, 0.f, 0.f);
  if (branch == 0) g.x = (y.x < 0.f) ? -1.f : 1.f;
  if (branch == 1) g.y = (y.y < 0.f) ? -1.f : 1.f;
  if (branch == 2) g.z = (y.z < 0.f) ? -1.f : 1.f;
  return g;
}

__device__ __forceinline__ float3 body_grad(const DevBody &b, float3 y, int branch) {
  switch (b.kind) {
  case 0:
    return make_float3(0.f, 0.f, 1.f);
  case 1:
    return box_grad(y, b.shape, branch);
  case 2:
    if (branch < 4) return box_grad(y, b.shape, branch);
    {
      float3 z = make_float3(y.x - b.shape[6], y.y - b.shape[7], y.z - b.shape[8]);
      float3 g = box_grad(z, b.shape + 3, branch - 4);
      return make_float3(-g.x, -g.y, -g.z);
    }
  case 3: {
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (branch == 0) g.x = -1.f;
    if (branch == 1) g.x = 1.f;
    if (branch == 2) g.y = -1.f;
    if (branch == 3) g.y = 1.f;
    if (branch == 4) g.z = 1.f;
    return g;
  }
  case 5: {
    const float rho = sqrtf(y.x * y.x + y.y * y.y);
    if (!(rho > 0.f)) return make_float3(-1.f, 0.f, 0.f);
    return make_float3(-y.x / rho, -y.y / rho, 0.f);
  }
  case 4: {
    const float3 g = grid_dt(b, y, branch, nullptr);
    const float gn = sqrtf(g.x * g.x + g.y * g.y + g.z * g.z);
    if (!(gn > 0.f)) return make_float3(0.f, 0.f, 1.f);
    const float ig = 1.0f / gn;
    return make_float3(g.x * ig, g.y * ig, g.z * ig);
  }
  }
  return make_float3(0.f, 0.f, 1.f);
}

__device__ __forceinline__ float3 rot_apply(const float *R, float3 g) {
  return make_float3(R[0] * g.x + R[1] * g.y + R[2] * g.z, R[3] * g.x + R[4] * g.y + R[5] * g.z,
                     R[6] * g.x + R[7] * g.y + R[8] * g.z);
}

// Tape of one step for the adjoint: every iterate of the sweep.
struct Tape {
  float4 *Uh;    // [I + 1][n] velocity estimates U^0 .. U^I
  float *lamh;   // [I + 1][3][K][n] pair impulses lambda^0 .. lambda^I
  float *blamh;  // [I + 1][3][Kb][n] body-contact impulses
};

// Adjoint state of one reversed step (particle order unless noted).
struct AdjArgs {
  Tape tp;
  uint32_t I;              // sweeps per step
  uint32_t tool;           // global body index whose twists are differentiated (~0u: none)
  uint32_t nblk;           // blocks of the per-particle adjoint kernels
  uint32_t *twin;          // [K][n] position of contact (j -> i) in j's list
  float4 *Ubar[2];         // adjoint of U^{s+1} / U^s
  float *ubar[2];          // [3][K][n] adjoint of each pair contact's relative velocity, by sweep parity
  float *Lbar, *bLbar;     // [3][K][n], [3][Kb][n] adjoint of lambda^s (carried down the sweeps)
  float *psibar, *nbar;    // [K][n], [3][K][n]
  float *bpsibar, *bnbar, *bxcbar;  // [Kb][n], [3][Kb][n], [3][Kb][n]
  float4 *basebar;         // adjoint of v + dt g
  float4 *xbar_s;          // adjoint of x_{k+1} (working copy)
  float4 *xbar, *vbar;     // id order: in dL/dx_{k+1}, dL/dv_{k+1}; out dL/dx_k, dL/dv_k
  float *part;             // [I + 1][nblk][10] fixed-order partial sums
  float *pose_bar;         // [6] adjoint of the tool pose (p, rotation), updated per step
  float *dtwist;           // [steps][6] output
  double *mubar;           // [1] dL/dmu, accumulated
};

// Pre-projection impulse of one contact update: lambda - w (u - bias n).
__device__ __forceinline__ float3 pja_pre(float3 lam, float3 u, float3 n, float bias, float w) {
  return make_float3(lam.x - w * (u.x - bias * n.x), lam.y - w * (u.y - bias * n.y), lam.z - w * (u.z - bias * n.z));
}

// One projected-Jacobi contact update (Alg. 1 with the accumulated-impulse clamp).
// lam: accumulated impulse on the particle; u: relative velocity particle - partner;
// n: unit normal partner -> particle; bias: alpha psi / dt; w: effective mass.
__device__ __forceinline__ float3 pja_cone(float3 s, float3 n, float mu) {
  const float sx = s.x, sy = s.y, sz = s.z;
  float ln = sx * n.x + sy * n.y + sz * n.z;
  float lnp = fmaxf(ln, 0.0f);
  float tx = sx - ln * n.x, ty = sy - ln * n.y, tz = sz - ln * n.z;
  float t2 = tx * tx + ty * ty + tz * tz;
  float lim = mu * lnp;
  if (t2 > lim * lim) {
    float sc = lim * rsqrtf(t2);
    tx *= sc;
    ty *= sc;
    tz *= sc;
  }
  return make_float3(lnp * n.x + tx, lnp * n.y + ty, lnp * n.z + tz);
}

__device__ __forceinline__ float3 pja_project(float3 lam, float3 u, float3 n, float bias, float w, float mu) {
  return pja_cone(pja_pre(lam, u, n, bias, w), n, mu);
}

}  // namespace gg
