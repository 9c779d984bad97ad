// gg_capi.cu -- host implementation of the C ABI declared in include/gg.h.
//
// All device memory is allocated by gg_create / gg_create_batch (and by
// gg_set_trajectory for its table, gg_set_body_grid for its samples, and lazily by
// the first readback that needs a
// staging buffer); gg_step allocates nothing.  A time step is captured once into
// a CUDA graph and replayed on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gg.h"
#include "gg_device.cuh"
#include "gg_internal.h"

using gg::DevBody;
using gg::DevCtrl;
using gg::DevEnv;
using gg::StepArgs;

namespace {

// One launch-shape set: threads per block of the per-launch sweep, the GG_TUNE_* bits of
// its variants (GG_TUNE_FUSED aside: a set is fused when it names a fused block size),
// and the block size of the cooperative all-sweeps launch.  The iteration count and the
// cooperative grid are filled in at creation.
constexpr gg::LaunchShape shape(int pja_block, uint32_t bits, int fused_block = 0) {
  gg::LaunchShape s{};
  s.pja_block = pja_block;
  s.fused_block = fused_block;
  s.lists = (bits & GG_TUNE_LISTS) ? 1u : 0u;
  s.lean = (bits & GG_TUNE_LEAN) ? 1u : 0u;
  s.half = (bits & GG_TUNE_HALF) ? 1u : 0u;
  s.detect = (bits & GG_TUNE_DETECT) ? 1u : 0u;
  s.serp = (bits & GG_TUNE_SERP) ? 1u : 0u;
  s.pre = (bits & GG_TUNE_PRELOAD) ? 1u : 0u;
  s.one = (bits & GG_TUNE_ONELOOP) ? 1u : 0u;
  return s;
}

// Launch-shape sets accepted by gg_params.tuning (index k-1).
constexpr uint32_t kL = GG_TUNE_LISTS, kLean = GG_TUNE_LEAN, kHalf = GG_TUNE_HALF, kDet = GG_TUNE_DETECT,
                   kSerp = GG_TUNE_SERP, kPre = GG_TUNE_PRELOAD, kOne = GG_TUNE_ONELOOP;
const gg::LaunchShape kShapes[] = {
    shape(256, 0),  shape(128, 0), shape(512, 0), shape(64, 0),       // 1-4: sort, per-launch sweeps
    shape(256, 0, 1024), shape(256, 0, 512),                           // 5-6: all sweeps in one launch
    shape(256, kL), shape(128, kL),                                    // 7-8: lists
    shape(256, kL | kLean), shape(256, kLean),                         // 9-10: 40-register sweeps
    shape(256, kL | kHalf), shape(256, kL | kLean | kHalf), shape(256, kHalf),  // 11-13: half stencil
    shape(256, kDet), shape(256, kL | kDet),                           // 14-15: TwoLoopsFused
    shape(128, kSerp | kPre), shape(128, kL | kSerp | kPre), shape(128, kL | kHalf | kSerp | kPre),  // 16-18
    shape(128, kOne), shape(128, kL | kOne),                           // 19-20: OneLoop
    shape(128, kL | kHalf),                                            // 21
    shape(128, kL | kLean | kHalf | kSerp)};                           // 22
constexpr uint32_t kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// n_h factors the autotuner tries when gg_params.hash_tune is set (the paper's 2n first)
constexpr uint32_t kHashFactors[] = {2, 4, 8};
constexpr uint32_t kNumHashFactors = sizeof(kHashFactors) / sizeof(kHashFactors[0]);
// cell edges (x r_max of each environment) it then tries when the cell size is not fixed
constexpr double kCellFactors[] = {2.002, 2.2, 2.5};
constexpr uint32_t kNumCellFactors = sizeof(kCellFactors) / sizeof(kCellFactors[0]);

constexpr uint32_t kStateMagic = 0x31534747u;  // "GGS1"

struct StateHeader {
  uint32_t magic, n, n_envs, maxb;
  uint64_t steps;
  uint32_t pad[2];
};

}  // namespace

struct gg_sim {
  int device = 0;
  gg_params p{};
  uint32_t n = 0, n_envs = 0, maxb = 0, K = 0, Kb = 0, H = 1;
  uint32_t nh_total = 0, nh_pad = 0, n_chunks = 0;
  uint32_t nh_cap = 0;   // buckets allocated (nh_pad at the largest n_h factor tried)
  uint32_t hf = 2;       // n_h factor in use (hash_size = 0)
  uint32_t cf = 0;       // cell edge in use: kCellFactors[cf] r_max per environment (cell_size = 0)
  std::vector<float> rmax;  // largest radius of each environment
  std::vector<DevEnv> envs;
  std::vector<uint32_t> nbodies;
  std::vector<float *> traj;  // per body slot
  std::vector<float *> grids; // per body slot: samples of GRID bodies
  std::vector<uint32_t> fgb;  // free-body slot -> global body index (~0u when unused)
  uint32_t F = 0, Lcap = 0;
  std::vector<void *> allocs;
  StepArgs a{};
  gg::LaunchShape ls{};
  uint32_t tuning_sel = 1;
  cudaStream_t cap = nullptr;
  // the step graph, captured lazily: [0] plain, [1] with the stage-timing events
  cudaGraph_t graph[2] = {};
  cudaGraphExec_t exec[2] = {};
  // gg_step_io: pinned inputs -> one step -> pinned outputs as one graph, for the
  // device addresses of the last buffers it was given
  cudaGraphExec_t io_exec = nullptr;
  const void *io_ptr[3] = {};
  uint64_t steps = 0;
  void *staging = nullptr;
  size_t staging_bytes = 0;
  DevCtrl *ctrl_host = nullptr;  // pinned mirror of the control word (status reads)
  float *vel3 = nullptr;  // n*3 staging for velocity upload / readback
  uint32_t *render_img = nullptr;  // gg_render scratch (ordered bits per pixel) and ...
  float *render_out = nullptr;     // ... device image for host destinations, ...
  float4 *render_rays = nullptr;   // ... and the depth camera's per-pixel rays
  size_t render_px = 0;
  // differentiation: checkpoints, the tapes of one segment, adjoint buffers
  struct {
    uint32_t n_steps = 0, K = 0, slots = 0, taped = 0, tool = 0xffffffffu;
    size_t state_bytes = 0;
    char *ckpt = nullptr, *seg = nullptr, *fin = nullptr;
    gg::Tape tp{};  // slot 0's tape; slot k's starts k tapes further
    // each step of a segment keeps its own contact arrays (slot k at k times the size)
    uint32_t *ccount = nullptr, *cj = nullptr, *bj = nullptr;
    float4 *cn = nullptr, *bn = nullptr, *bxc = nullptr;
    gg::AdjArgs d{};
    std::vector<void *> allocs;
  } ad;
  bool timing = false;
  bool tuned = false;
  cudaEvent_t ev[5] = {};
  std::string err;
};

namespace {

gg_status fail(gg_sim *s, gg_status st, const std::string &msg) {
  if (s) s->err = msg;
  return st;
}

gg_status cuda_fail(gg_sim *s, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  (void)cudaGetLastError();
  return fail(s, GG_ERR_CUDA, m);
}

#define GG_CUDA(sim, call)                                         \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail((sim), e_, #call);     \
  } while (0)

template <typename T>
gg_status dalloc(gg_sim *s, T **ptr, size_t count) {
  void *p = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(s, GG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  s->allocs.push_back(p);
  *ptr = static_cast<T *>(p);
  return GG_OK;
}

gg_status status_from_flags(gg_sim *s, uint32_t f) {
  if (f & gg::kFlagTimeout) return fail(s, GG_ERR_DEVICE_TIMEOUT, "a grid barrier wait gave up (bounded wait)");
  if (f & gg::kFlagListBound)
    return fail(s, GG_ERR_INTERNAL, "a bucket list walk passed the particle count (cut short)");
  if (f & gg::kFlagDebugCheck)
    return fail(s, GG_ERR_INTERNAL, "a device-side index check of the GG_DEBUG build failed (access skipped)");
  if (f & gg::kFlagBucketBound)
    return fail(s, GG_ERR_INVALID_ARG,
                "a hash bucket held more than " + std::to_string(gg::kMaxBucket) +
                    " particles (cell_size far above 2 r_max, or hash_size far below n); its walks were cut short");
  if (f & gg::kFlagNonFinite) return fail(s, GG_ERR_NONFINITE, "a particle position or velocity became non-finite");
  if (f & (gg::kFlagPPOverflow | gg::kFlagBodyOverflow))
    return fail(s, GG_ERR_CONTACT_OVERFLOW, "a particle exceeded its contact capacity (flags " + std::to_string(f) + ")");
  return GG_OK;
}

// The control word after the work queued on `st` (one copy into pinned memory, one wait).
gg_status read_ctrl(gg_sim *s, DevCtrl *out, cudaStream_t st) {
  if (!s->ctrl_host) GG_CUDA(s, cudaHostAlloc(reinterpret_cast<void **>(&s->ctrl_host), sizeof(DevCtrl), 0));
  GG_CUDA(s, cudaMemcpyAsync(s->ctrl_host, s->a.ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, st));
  GG_CUDA(s, cudaStreamSynchronize(st));
  *out = *s->ctrl_host;
  return GG_OK;
}

void free_graph(gg_sim *s) {
  for (int t = 0; t < 2; ++t) {
    if (s->exec[t]) cudaGraphExecDestroy(s->exec[t]);
    if (s->graph[t]) cudaGraphDestroy(s->graph[t]);
    s->exec[t] = nullptr;
    s->graph[t] = nullptr;
  }
  if (s->io_exec) cudaGraphExecDestroy(s->io_exec);
  s->io_exec = nullptr;
  for (const void *&p : s->io_ptr) p = nullptr;
}

gg_status ensure_staging(gg_sim *s, size_t bytes) {
  if (s->staging_bytes >= bytes) return GG_OK;
  if (s->staging) cudaFree(s->staging);
  s->staging = nullptr;
  s->staging_bytes = 0;
  cudaError_t e = cudaMalloc(&s->staging, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(s, GG_ERR_OOM, "staging allocation failed");
  }
  s->staging_bytes = bytes;
  return GG_OK;
}

bool finite_pos(float v) { return std::isfinite(v); }

// Device address of a caller's pinned (page-locked, registered) host buffer, or null
// for pageable memory: a kernel can then move particle state to or from it over the
// host link directly, without a staging copy.
void *pinned_device_ptr(const void *host) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// One simulation state (what a step reads): particles, bodies, control word.
size_t state_bytes(const gg_sim *s) {
  const size_t nbt = (size_t)s->n_envs * s->maxb;
  return (size_t)s->n * 32 + nbt * sizeof(DevBody) + sizeof(DevCtrl);
}

gg_status save_state(gg_sim *s, char *dst, cudaStream_t st) {
  const size_t n = s->n, nbt = (size_t)s->n_envs * s->maxb;
  if (n) {
    GG_CUDA(s, cudaMemcpyAsync(dst, s->a.pos_id, n * 16, cudaMemcpyDeviceToDevice, st));
    GG_CUDA(s, cudaMemcpyAsync(dst + n * 16, s->a.vel_id, n * 16, cudaMemcpyDeviceToDevice, st));
  }
  GG_CUDA(s, cudaMemcpyAsync(dst + n * 32, s->a.bodies, nbt * sizeof(DevBody), cudaMemcpyDeviceToDevice, st));
  GG_CUDA(s, cudaMemcpyAsync(dst + n * 32 + nbt * sizeof(DevBody), s->a.ctrl, sizeof(DevCtrl),
                             cudaMemcpyDeviceToDevice, st));
  return GG_OK;
}

gg_status restore_state(gg_sim *s, const char *src, cudaStream_t st) {
  const size_t n = s->n, nbt = (size_t)s->n_envs * s->maxb;
  if (n) {
    GG_CUDA(s, cudaMemcpyAsync(s->a.pos_id, src, n * 16, cudaMemcpyDeviceToDevice, st));
    GG_CUDA(s, cudaMemcpyAsync(s->a.vel_id, src + n * 16, n * 16, cudaMemcpyDeviceToDevice, st));
  }
  GG_CUDA(s, cudaMemcpyAsync(s->a.bodies, src + n * 32, nbt * sizeof(DevBody), cudaMemcpyDeviceToDevice, st));
  GG_CUDA(s, cudaMemcpyAsync(s->a.ctrl, src + n * 32 + nbt * sizeof(DevBody), sizeof(DevCtrl),
                             cudaMemcpyDeviceToDevice, st));
  return GG_OK;
}

template <typename T>
gg_status ad_alloc(gg_sim *s, T **ptr, size_t count) {
  void *p = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(s, GG_ERR_OOM, "tape allocation of " + std::to_string(bytes) + " bytes failed");
  }
  s->ad.allocs.push_back(p);
  *ptr = static_cast<T *>(p);
  return GG_OK;
}

// Launch shape k (1-based); a fused shape gets its resident grid from the occupancy.
// Rotation of a float quaternion (w, x, y, z), each entry in the order the step's
// kernels use (host code is compiled without multiply-add contraction).
void rot_from_quat(const float *q, float *R) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y,
              wz = w * z;
  R[0] = 1.0f - 2.0f * (yy + zz);
  R[1] = 2.0f * (xy - wz);
  R[2] = 2.0f * (xz + wy);
  R[3] = 2.0f * (xy + wz);
  R[4] = 1.0f - 2.0f * (xx + zz);
  R[5] = 2.0f * (yz - wx);
  R[6] = 2.0f * (xz - wy);
  R[7] = 2.0f * (yz + wx);
  R[8] = 1.0f - 2.0f * (xx + yy);
}

gg_status set_shape(gg_sim *s, uint32_t k) {
  gg::LaunchShape ls = kShapes[k - 1];
  ls.iters = s->p.pja_iters;
  if (ls.fused_block || ls.detect) {
    int nsm = 0;
    GG_CUDA(s, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device));
    const int per = ls.detect ? gg::detect_sweeps_blocks_per_sm(ls.lists != 0, s->K)
                              : gg::fused_pja_blocks_per_sm(ls.fused_block);
    ls.fused_grid = per > 0 ? (uint32_t)(per * nsm) : 0;
  }
  s->ls = ls;
  s->a.lists = ls.lists;
  s->tuning_sel = k;
  free_graph(s);
  return GG_OK;
}

// Launch-shape sets allowed by gg_params.binning (0: any, 1: sort only, 2: lists only).
bool shape_allowed(const gg_sim *s, uint32_t k) {
  const uint32_t b = s->p.binning;
  return b == 0 || (b == 1 && !kShapes[k - 1].lists) || (b == 2 && kShapes[k - 1].lists);
}

gg_status capture(gg_sim *s);

// tuning == 0: time every launch-shape set on the current state (3 steps each, after
// one untimed step), restoring the state before each trial and at the end, and keep
// the fastest.  Every set gives bit-identical results, so the choice cannot change them.
// Bucket ranges of every environment for n_h = factor x n_env (or the fixed hash_size):
// the host table, the totals and the step arguments.  Does not touch the device.
gg_status layout_hash(gg_sim *s, uint32_t factor) {
  uint64_t hb = 0;
  for (DevEnv &E : s->envs) {
    uint64_t nh = s->p.hash_size ? s->p.hash_size : (uint64_t)factor * E.n;
    if (nh == 0) nh = 1;
    E.hbase = (uint32_t)hb;
    E.nh = (uint32_t)nh;
    E.nh_magic = gg::remainder_magic(E.nh);
    hb += nh;
    if (hb > 0xF0000000ull) return fail(s, GG_ERR_INVALID_ARG, "hash tables exceed 2^32 buckets");
  }
  uint32_t pad = (uint32_t)(((hb + gg::kScanTile - 1) / gg::kScanTile) * gg::kScanTile);
  if (pad == 0) pad = gg::kScanTile;
  if (s->nh_cap && pad > s->nh_cap) return fail(s, GG_ERR_INVALID_ARG, "n_h factor beyond the allocated tables");
  s->nh_total = (uint32_t)hb;
  s->nh_pad = pad;
  s->a.nh_total = s->nh_total;
  s->a.nh_pad = s->nh_pad;
  s->hf = factor;
  return GG_OK;
}

// Switch the n_h factor between steps: new bucket ranges on the device (ordered on
// `st`), graphs recaptured on the next step.  Every list is empty and every histogram
// count zero between steps over the whole allocation, so nothing else changes.
gg_status set_hash_factor(gg_sim *s, uint32_t factor, cudaStream_t st) {
  if (factor == s->hf) return GG_OK;
  gg_status rc = layout_hash(s, factor);
  if (rc != GG_OK) return rc;
  GG_CUDA(s, cudaMemcpyAsync(s->a.envs, s->envs.data(), sizeof(DevEnv) * s->n_envs, cudaMemcpyHostToDevice, st));
  GG_CUDA(s, cudaStreamSynchronize(st));  // the host table may change again before the copy would run
  free_graph(s);
  return GG_OK;
}

// Switch the cell edge of every environment to kCellFactors[f] r_max between steps (no
// effect when gg_params.cell_size fixes it): new reciprocals on the device (ordered on
// `st`), graphs recaptured.  Contacts and dynamics do not depend on it (the pair test is
// exact and every cell within reach is walked); the bucket keys do.
gg_status set_cell_factor(gg_sim *s, uint32_t f, cudaStream_t st) {
  if (s->p.cell_size > 0.f || f == s->cf) return GG_OK;
  for (uint32_t e = 0; e < s->n_envs; ++e) {
    const float c = s->envs[e].n ? (float)(kCellFactors[f] * (double)s->rmax[e]) : 1.0f;
    s->envs[e].inv_cell = (float)(1.0 / (double)c);
  }
  s->cf = f;
  GG_CUDA(s, cudaMemcpyAsync(s->a.envs, s->envs.data(), sizeof(DevEnv) * s->n_envs, cudaMemcpyHostToDevice, st));
  GG_CUDA(s, cudaStreamSynchronize(st));
  free_graph(s);
  return GG_OK;
}

// Time the current graph: one untimed step, then 3 (state restored first).
gg_status time_trial(gg_sim *s, const char *saved, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st, float *ms) {
  gg_status rc = capture(s);
  if (rc != GG_OK) return rc;
  if ((rc = restore_state(s, saved, st)) != GG_OK) return rc;
  cudaError_t ce = cudaGraphLaunch(s->exec[s->timing], st);
  if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
  for (int r = 0; r < 3 && ce == cudaSuccess; ++r) ce = cudaGraphLaunch(s->exec[s->timing], st);
  if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
  if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, e0, e1);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "autotune trial");
  return GG_OK;
}

gg_status autotune(gg_sim *s, cudaStream_t st) {
  s->tuned = true;
  if (s->p.tuning || !s->n) return GG_OK;
  const size_t bytes = state_bytes(s);
  char *saved = nullptr;
  if (cudaMalloc(&saved, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(s, GG_ERR_OOM, "autotune state copy");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.f;
  uint32_t best_k = 1;
  gg_status rc = save_state(s, saved, st);
  if (rc == GG_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = cuda_fail(s, cudaGetLastError(), "cudaEventCreate");
  // launch-shape sets at the n_h in use, then (hash_tune) the n_h factors with the
  // chosen set
  const bool tune_nh = s->p.hash_tune && !s->p.hash_size && !s->p.hash_factor;
  uint32_t best_f = s->hf;
  if (tune_nh) rc = rc == GG_OK ? set_hash_factor(s, kHashFactors[0], st) : rc;
  bool first = true;
  for (uint32_t k = 1; rc == GG_OK && k <= kNumShapes; ++k) {
    if (!shape_allowed(s, k)) continue;
    if ((rc = set_shape(s, k)) != GG_OK ||
        ((kShapes[k - 1].fused_block || kShapes[k - 1].detect) && !s->ls.fused_grid))
      continue;
    float ms = 0.f;
    if ((rc = time_trial(s, saved, e0, e1, st, &ms)) != GG_OK) break;
    if (first || ms < best) {
      best = ms;
      best_k = k;
      best_f = s->hf;
      first = false;
    }
  }
  if (rc == GG_OK && tune_nh) rc = set_shape(s, best_k);
  for (uint32_t f = 1; rc == GG_OK && tune_nh && f < kNumHashFactors; ++f) {
    float ms = 0.f;
    if ((rc = set_hash_factor(s, kHashFactors[f], st)) != GG_OK) break;
    if ((rc = time_trial(s, saved, e0, e1, st, &ms)) != GG_OK) break;
    if (ms < best) {
      best = ms;
      best_f = kHashFactors[f];
    }
  }
  // then the cell edge, with the chosen set and table
  uint32_t best_c = s->cf;
  if (rc == GG_OK && tune_nh && s->p.cell_size <= 0.f) {
    rc = set_hash_factor(s, best_f, st);
    if (rc == GG_OK) rc = set_shape(s, best_k);
    for (uint32_t f = 0; rc == GG_OK && f < kNumCellFactors; ++f) {
      if (f == best_c) continue;
      float ms = 0.f;
      if ((rc = set_cell_factor(s, f, st)) != GG_OK) break;
      if ((rc = time_trial(s, saved, e0, e1, st, &ms)) != GG_OK) break;
      if (ms < best) {
        best = ms;
        best_c = f;
      }
    }
  }
  if (rc == GG_OK) rc = restore_state(s, saved, st);
  if (rc == GG_OK) rc = set_hash_factor(s, best_f, st);
  if (rc == GG_OK) rc = set_cell_factor(s, best_c, st);
  if (rc == GG_OK) rc = set_shape(s, best_k);
  if (rc == GG_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = cuda_fail(s, cudaGetLastError(), "autotune");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(saved);
  return rc;
}

// Capture the step graph of the current timing mode (the other mode's graph stays).
gg_status capture(gg_sim *s) {
  const int t = s->timing ? 1 : 0;
  if (s->exec[t]) cudaGraphExecDestroy(s->exec[t]);
  if (s->graph[t]) cudaGraphDestroy(s->graph[t]);
  s->exec[t] = nullptr;
  s->graph[t] = nullptr;
  GG_CUDA(s, cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = gg::enqueue_step(s->a, s->ls, s->cap, s->timing ? s->ev : nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s->cap, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(s, e, "enqueue_step during capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(s, e2, "cudaStreamEndCapture");
  s->graph[t] = g;
  GG_CUDA(s, cudaGraphInstantiate(&s->exec[t], g, 0));
  return GG_OK;
}

// The step arguments of segment slot k: the simulation's, with that slot's contact arrays.
gg::StepArgs slot_args(const gg_sim *s, uint32_t k) {
  gg::StepArgs a = s->a;
  const size_t n = s->n, KN = (size_t)s->K * n, KbN = (size_t)s->Kb * n;
  a.ccount = s->ad.ccount + k * n;
  a.cj = s->ad.cj + k * KN;
  a.cn = s->ad.cn + k * KN;
  a.bj = s->ad.bj + k * KbN;
  a.bn = s->ad.bn + k * KbN;
  a.bxc = s->ad.bxc + k * KbN;
  return a;
}

// The state regions (the layout save_state writes) between the simulation and `buf`,
// as one copy launch: saving (to buf) or restoring (from buf).
gg::CopyRegions state_regions(gg_sim *s, char *buf, bool save) {
  static_assert(sizeof(DevBody) % 4 == 0 && sizeof(DevCtrl) % 4 == 0, "state regions are copied as words");
  const size_t n = s->n, nbt = (size_t)s->n_envs * s->maxb;
  uint32_t *live[4] = {reinterpret_cast<uint32_t *>(s->a.pos_id), reinterpret_cast<uint32_t *>(s->a.vel_id),
                       reinterpret_cast<uint32_t *>(s->a.bodies), reinterpret_cast<uint32_t *>(s->a.ctrl)};
  uint32_t *saved[4] = {reinterpret_cast<uint32_t *>(buf), reinterpret_cast<uint32_t *>(buf + n * 16),
                        reinterpret_cast<uint32_t *>(buf + n * 32),
                        reinterpret_cast<uint32_t *>(buf + n * 32 + nbt * sizeof(DevBody))};
  const size_t words[4] = {4 * n, 4 * n, nbt * sizeof(DevBody) / 4, sizeof(DevCtrl) / 4};
  gg::CopyRegions c{};
  for (int r = 0; r < 4; ++r) {
    c.dst[r] = save ? saved[r] : live[r];
    c.src[r] = save ? live[r] : saved[r];
    c.words[r] = words[r];
  }
  return c;
}

// The tape of segment slot k.
gg::Tape slot_tape(const gg_sim *s, uint32_t k) {
  gg::Tape t = s->ad.tp;
  const size_t n = s->n, I = s->ls.iters, KN = (size_t)s->K * n, KbN = (size_t)s->Kb * n;
  t.Uh += k * (I + 1) * n;
  t.lamh += k * (I + 1) * 3 * KN;
  t.blamh += k * (I + 1) * 3 * KbN;
  return t;
}

}  // namespace

extern "C" {

uint32_t gg_abi_version(void) { return GG_ABI_VERSION; }

const char *gg_status_string(gg_status s) {
  switch (s) {
  case GG_OK: return "ok";
  case GG_ERR_INVALID_ARG: return "invalid argument";
  case GG_ERR_OOM: return "out of memory";
  case GG_ERR_CUDA: return "CUDA error";
  case GG_ERR_CONTACT_OVERFLOW: return "contact capacity overflow";
  case GG_ERR_DEVICE_TIMEOUT: return "device wait timed out";
  case GG_ERR_NONFINITE: return "non-finite state";
  case GG_ERR_UNSUPPORTED: return "unsupported";
  case GG_ERR_NO_DEVICE: return "no CUDA device";
  case GG_ERR_INTERNAL: return "internal device invariant failed";
  }
  return "unknown status";
}

const char *gg_last_error(const gg_sim *sim) { return sim ? sim->err.c_str() : "null simulation"; }

uint32_t gg_tuning_count(void) { return kNumShapes; }

uint32_t gg_hash_size(const gg_sim *s, uint32_t env) { return (s && env < s->n_envs) ? s->envs[env].nh : 0; }

float gg_cell_size(const gg_sim *s, uint32_t env) {
  if (!s || env >= s->n_envs) return 0.f;
  if (s->p.cell_size > 0.f) return s->p.cell_size;
  return s->envs[env].n ? (float)(kCellFactors[s->cf] * (double)s->rmax[env]) : 1.0f;
}

uint32_t gg_tuning_flags(uint32_t k) {
  if (k < 1 || k > kNumShapes) return 0;
  const gg::LaunchShape &ls = kShapes[k - 1];
  return (ls.lists ? GG_TUNE_LISTS : 0u) | (ls.fused_block ? GG_TUNE_FUSED : 0u) | (ls.lean ? GG_TUNE_LEAN : 0u) |
         (ls.half ? GG_TUNE_HALF : 0u) | (ls.detect ? GG_TUNE_DETECT : 0u) | (ls.serp ? GG_TUNE_SERP : 0u) |
         (ls.pre ? GG_TUNE_PRELOAD : 0u) | (ls.one ? GG_TUNE_ONELOOP : 0u);
}

uint32_t gg_kernels_per_step(const gg_sim *sim) { return sim ? gg::kernels_per_step(sim->a, sim->ls) : 0; }

gg_status gg_enable_timing(gg_sim *s, int on) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (on && !s->ev[0])
    for (cudaEvent_t &ev : s->ev) GG_CUDA(s, cudaEventCreate(&ev));
  s->timing = on != 0;  // selects the step graph; each mode's graph is captured once
  return GG_OK;
}

gg_status gg_stage_ms(gg_sim *s, float *ms) {
  if (!s || !ms) return GG_ERR_INVALID_ARG;
  if (!s->timing || !s->steps) return fail(s, GG_ERR_INVALID_ARG, "gg_stage_ms: timing off or no step taken");
  GG_CUDA(s, cudaEventSynchronize(s->ev[4]));
  for (int k = 0; k < GG_NUM_STAGES; ++k) GG_CUDA(s, cudaEventElapsedTime(&ms[k], s->ev[k], s->ev[k + 1]));
  return GG_OK;
}

uint32_t gg_tuning_selected(const gg_sim *sim) { return sim ? sim->tuning_sel : 0; }

gg_status gg_autotune(gg_sim *s, void *stream) {
  if (!s) return GG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GG_CUDA(s, cudaStreamSynchronize(st));
  return autotune(s, st);
}

void gg_destroy(gg_sim *sim) {
  if (!sim) return;
  cudaSetDevice(sim->device);
  cudaDeviceSynchronize();
  free_graph(sim);
  for (cudaEvent_t &ev : sim->ev)
    if (ev) cudaEventDestroy(ev);
  if (sim->cap) cudaStreamDestroy(sim->cap);
  for (void *p : sim->allocs) cudaFree(p);
  for (void *p : sim->ad.allocs) cudaFree(p);
  for (float *t : sim->traj)
    if (t) cudaFree(t);
  for (float *g : sim->grids)
    if (g) cudaFree(g);
  if (sim->staging) cudaFree(sim->staging);
  if (sim->ctrl_host) cudaFreeHost(sim->ctrl_host);
  if (sim->render_img) cudaFree(sim->render_img);
  if (sim->render_out) cudaFree(sim->render_out);
  if (sim->render_rays) cudaFree(sim->render_rays);
  delete sim;
}

gg_status gg_create_batch(const gg_params *params, uint32_t n_envs, const uint32_t *env_offsets,
                          const float *pos_radius, const float *vel, const float *mass, int inputs_on_device,
                          gg_sim **out) {
  if (!out) return GG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params || params->struct_size != sizeof(gg_params)) return GG_ERR_INVALID_ARG;
  if (n_envs == 0 || !env_offsets) return GG_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return GG_ERR_NO_DEVICE;
  }
  gg_sim *s = new (std::nothrow) gg_sim();
  if (!s) return GG_ERR_OOM;
  gg_status rc = GG_OK;
  auto bail = [&](gg_status st) {
    gg_destroy(s);
    return st;
  };
  cudaGetDevice(&s->device);
  const gg_params &P = *params;
  s->p = P;
  std::vector<uint32_t> offs(env_offsets, env_offsets + n_envs + 1);
  if (offs[0] != 0) return bail(GG_ERR_INVALID_ARG);
  for (uint32_t e = 0; e < n_envs; ++e)
    if (offs[e + 1] < offs[e]) return bail(GG_ERR_INVALID_ARG);
  const uint32_t n = offs[n_envs];
  if (n && !pos_radius) return bail(GG_ERR_INVALID_ARG);
  if (!(P.dt > 0.f) || !std::isfinite(P.dt) || !(P.mu >= 0.f) || !(P.alpha >= 0.f) || P.pja_iters == 0 ||
      P.pja_iters > 100000 || !(P.cell_size >= 0.f) || !(P.density >= 0.f) ||
      !std::isfinite(P.gravity[0]) || !std::isfinite(P.gravity[1]) || !std::isfinite(P.gravity[2]))
    return bail(GG_ERR_INVALID_ARG);
  s->K = P.max_contacts ? P.max_contacts : 16;
  s->Kb = P.max_body_contacts ? P.max_body_contacts : 4;
  s->maxb = P.max_bodies ? P.max_bodies : 8;
  s->H = P.wrench_history ? P.wrench_history : 1;
  if (s->K > (uint32_t)gg::kMaxK || s->Kb > (uint32_t)gg::kMaxKb || s->maxb > 64 || s->H > (1u << 20))
    return bail(GG_ERR_INVALID_ARG);
  if (P.tuning > kNumShapes) return bail(GG_ERR_INVALID_ARG);
  if (P.binning > 2 || !std::isfinite(P.cyclic_z[0]) || !std::isfinite(P.cyclic_z[1]) ||
      (P.cyclic_z[1] < P.cyclic_z[0]))
    return bail(GG_ERR_INVALID_ARG);
  if (P.pja_weight > 1) return bail(GG_ERR_INVALID_ARG);
  if (P.pja_weight && P.max_free_bodies)
    return bail(fail(s, GG_ERR_UNSUPPORTED, "pja_weight = 1 (Alg. 1 as printed) does not support free bodies"));
  s->F = P.max_free_bodies;
  s->Lcap = P.free_contact_capacity ? P.free_contact_capacity : 4096;
  if (s->F > 4096 || s->Lcap > 8192) return bail(GG_ERR_INVALID_ARG);
  s->n = n;
  s->n_envs = n_envs;

  // host copies of the inputs
  std::vector<float> hp((size_t)n * 4), hv((size_t)n * 3, 0.f), hm;
  auto fetch = [&](const float *src, float *dst, size_t count) -> gg_status {
    if (!count) return GG_OK;
    if (inputs_on_device) {
      cudaError_t e = cudaMemcpy(dst, src, count * sizeof(float), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(s, e, "reading input arrays");
    } else {
      std::memcpy(dst, src, count * sizeof(float));
    }
    return GG_OK;
  };
  if ((rc = fetch(pos_radius, hp.data(), (size_t)n * 4)) != GG_OK) return bail(rc);
  if (vel && (rc = fetch(vel, hv.data(), (size_t)n * 3)) != GG_OK) return bail(rc);
  if (mass) {
    hm.resize(n);
    if ((rc = fetch(mass, hm.data(), n)) != GG_OK) return bail(rc);
  }
  const double rho = P.density > 0.f ? P.density : 2500.0;
  std::vector<float4> h_pos(n), h_vel(n);
  std::vector<uint32_t> h_env(n);
  for (uint32_t i = 0; i < n; ++i) {
    const float *q = &hp[(size_t)4 * i];
    if (!finite_pos(q[0]) || !finite_pos(q[1]) || !finite_pos(q[2]) || !(q[3] > 0.f) || !std::isfinite(q[3]))
      return bail(fail(s, GG_ERR_INVALID_ARG, "particle " + std::to_string(i) + ": bad position or radius"));
    const float m = mass ? hm[i] : (float)(rho * (4.0 / 3.0) * 3.14159265358979323846 * (double)q[3] * q[3] * q[3]);
    if (!(m > 0.f) || !std::isfinite(m))
      return bail(fail(s, GG_ERR_INVALID_ARG, "particle " + std::to_string(i) + ": bad mass"));
    h_pos[i] = make_float4(q[0], q[1], q[2], q[3]);
    h_vel[i] = make_float4(hv[3 * i], hv[3 * i + 1], hv[3 * i + 2], 1.0f / m);
  }
  // environments: cell size, hash range, wrench chunks
  s->envs.resize(n_envs);
  uint32_t chunks = 0;
  for (uint32_t e = 0; e < n_envs; ++e) {
    DevEnv &E = s->envs[e];
    E.off = offs[e];
    E.n = offs[e + 1] - offs[e];
    float rmax = 0.f;
    for (uint32_t i = E.off; i < E.off + E.n; ++i) {
      rmax = std::max(rmax, h_pos[i].w);
      h_env[i] = e;
    }
    s->rmax.push_back(rmax);
    float c = P.cell_size > 0.f ? P.cell_size : (float)(2.002 * (double)rmax);
    if (E.n && !(c >= 2.0f * rmax))
      return bail(fail(s, GG_ERR_INVALID_ARG, "cell_size must be >= 2 r_max of every environment"));
    if (!(c > 0.f)) c = 1.0f;
    E.inv_cell = (float)(1.0 / (double)c);
    E.nbodies = 0;
    E.chunk0 = chunks;
    E.nchunks = (E.n + gg::kWrenchChunk - 1) / gg::kWrenchChunk;
    chunks += E.nchunks;
  }
  const uint32_t hf0 = P.hash_factor ? P.hash_factor : 2;
  const bool tune_nh = P.hash_tune && !P.hash_size && !P.hash_factor;
  if (P.hash_tune > 1) return bail(GG_ERR_INVALID_ARG);
  if ((rc = layout_hash(s, tune_nh ? kHashFactors[kNumHashFactors - 1] : hf0)) != GG_OK) return bail(rc);
  s->nh_cap = s->nh_pad;  // allocation for the largest factor; then the factor in use
  if ((rc = layout_hash(s, hf0)) != GG_OK) return bail(rc);
  s->n_chunks = chunks;
  const uint32_t nbt = n_envs * s->maxb;
  s->nbodies.assign(n_envs, 0);
  s->traj.assign(nbt, nullptr);
  s->grids.assign(nbt, nullptr);

  // device buffers, all at capacity
  StepArgs &a = s->a;
  a.n = n;
  a.n_envs = n_envs;
  a.nh_total = s->nh_total;
  a.nh_pad = s->nh_pad;
  a.maxb = s->maxb;
  a.K = s->K;
  a.Kb = s->Kb;
  a.n_chunks = chunks;
  a.wrench_hist = s->H;
  a.dt = P.dt;
  a.mu = P.mu;
  a.ab = P.alpha / P.dt;
  a.lit = P.pja_weight;
  {
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, s->device) != cudaSuccess || khz <= 0) khz = 2000000;
    const double us = P.wait_limit_us ? (double)P.wait_limit_us : 500000.0;
    a.wait_cycles = (long long)(us * (double)khz / 1000.0);
  }
  a.cyc_lo = P.cyclic_z[0];
  a.cyc_h = P.cyclic_z[1] > P.cyclic_z[0] ? P.cyclic_z[1] - P.cyclic_z[0] : 0.f;
  for (int k = 0; k < 3; ++k) a.g[k] = P.gravity[k];
  const size_t nK = (size_t)n * s->K, nKb = (size_t)n * s->Kb;
  if ((rc = dalloc(s, &a.pos_id, n)) || (rc = dalloc(s, &a.vel_id, n)) || (rc = dalloc(s, &a.env_of, n)) ||
      (rc = dalloc(s, &a.key_id, n)) || (rc = dalloc(s, &a.cnt, s->nh_cap)) ||
      (rc = dalloc(s, &a.start, (size_t)s->nh_cap + 4)) || (rc = dalloc(s, &a.range, s->nh_cap)) || (rc = dalloc(s, &a.bsum, s->nh_cap / gg::kScanTile)) ||
      (rc = dalloc(s, &a.sid_tmp, n)) || (rc = dalloc(s, &a.sid, n)) || (rc = dalloc(s, &a.pos_s, n)) || (rc = dalloc(s, &a.U[0], n)) ||
      (rc = dalloc(s, &a.U[1], n)) || (rc = dalloc(s, &a.ccount, n)) || (rc = dalloc(s, &a.cj, nK)) ||
      (rc = dalloc(s, &a.cn, nK)) || (rc = dalloc(s, &a.clam, 3 * nK)) || (rc = dalloc(s, &a.bj, nKb)) ||
      (rc = dalloc(s, &a.bn, nKb)) || (rc = dalloc(s, &a.bxc, nKb)) || (rc = dalloc(s, &a.blam, 3 * nKb)) ||
      (rc = dalloc(s, &a.envs, n_envs)) || (rc = dalloc(s, &a.bodies, nbt)) ||
      (rc = dalloc(s, &a.chunk_env, chunks)) || (rc = dalloc(s, &a.wpart, (size_t)std::max(chunks, 1u) * s->maxb * 6)) ||
      (rc = dalloc(s, &a.wrench, (size_t)s->H * nbt * 6)) || (rc = dalloc(s, &a.ctrl, 1)) ||
      (rc = dalloc(s, &s->vel3, (size_t)n * 3)) || (rc = dalloc(s, &a.ncb, nbt)) ||
      (rc = dalloc(s, &a.fcount, s->F)) || (rc = dalloc(s, &a.flist, (size_t)s->F * s->Lcap)) ||
      (rc = dalloc(s, &a.fgb, s->F)) || (rc = dalloc(s, &a.fcc, (size_t)s->F * 8 * s->maxb)))
    return bail(rc);
  if ((rc = dalloc(s, &a.head, s->nh_cap)) || (rc = dalloc(s, &a.next, n)) || (rc = dalloc(s, &a.pcnt, n)) ||
      (rc = dalloc(s, &a.pscr, (size_t)2 * s->K * n)))
    return bail(rc);
  a.F = s->F;
  a.Lcap = s->Lcap;
  s->fgb.assign(s->F, 0xffffffffu);
  std::vector<uint32_t> h_chunk_env(std::max(chunks, 1u), 0);
  for (uint32_t e = 0; e < n_envs; ++e)
    for (uint32_t c = 0; c < s->envs[e].nchunks; ++c) h_chunk_env[s->envs[e].chunk0 + c] = e;
  cudaError_t e;
#define GG_UP(dst, src, bytes)                                                        \
  if ((e = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice)) != cudaSuccess) \
    return bail(cuda_fail(s, e, "upload"));
  if (n) {
    GG_UP(a.pos_id, h_pos.data(), sizeof(float4) * n);
    GG_UP(a.vel_id, h_vel.data(), sizeof(float4) * n);
    GG_UP(a.env_of, h_env.data(), sizeof(uint32_t) * n);
  }
  GG_UP(a.envs, s->envs.data(), sizeof(DevEnv) * n_envs);
  GG_UP(a.chunk_env, h_chunk_env.data(), sizeof(uint32_t) * h_chunk_env.size());
#undef GG_UP
  if ((e = cudaMemset(a.cnt, 0, sizeof(uint32_t) * s->nh_cap)) != cudaSuccess ||
      (e = cudaMemset(a.start, 0, sizeof(uint32_t) * ((size_t)s->nh_cap + 4))) != cudaSuccess ||
      (e = cudaMemset(a.bodies, 0, sizeof(DevBody) * nbt)) != cudaSuccess ||
      (e = cudaMemset(a.wrench, 0, sizeof(float) * s->H * nbt * 6)) != cudaSuccess ||
      (e = cudaMemset(a.ccount, 0, sizeof(uint32_t) * std::max(n, 1u))) != cudaSuccess ||
      (e = cudaMemset(a.pcnt, 0, sizeof(uint32_t) * std::max(n, 1u))) != cudaSuccess ||
      (e = cudaMemset(a.head, 0xff, sizeof(uint32_t) * s->nh_cap)) != cudaSuccess ||  // every list empty
      (e = cudaMemset(a.sid, 0, sizeof(uint32_t) * std::max(n, 1u))) != cudaSuccess ||
      (e = cudaMemset(a.key_id, 0, sizeof(uint32_t) * std::max(n, 1u))) != cudaSuccess ||
      (e = cudaMemset(a.ctrl, 0, sizeof(DevCtrl))) != cudaSuccess ||
      (e = cudaMemset(a.ncb, 0, sizeof(uint32_t) * nbt)) != cudaSuccess ||
      (e = cudaMemset(a.fgb, 0xff, sizeof(uint32_t) * std::max(s->F, 1u))) != cudaSuccess ||
      (e = cudaMemset(a.fcount, 0, sizeof(uint32_t) * std::max(s->F, 1u))) != cudaSuccess ||
      (e = cudaMemset(a.fcc, 0, sizeof(gg::CornerContact) * std::max<size_t>((size_t)s->F * 8 * s->maxb, 1))) !=
          cudaSuccess)
    return bail(cuda_fail(s, e, "initialising buffers"));
  if ((e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(s, e, "cudaStreamCreate"));
  if (P.barrier_test_phantoms) {
    const uint32_t ph = P.barrier_test_phantoms;
    if ((e = cudaMemcpy(&a.ctrl->bar_extra, &ph, sizeof(ph), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(cuda_fail(s, e, "initialising the control word"));
  }
  s->tuning_sel = P.tuning ? P.tuning : (P.binning == 2 ? 7u : 1u);
  if (!shape_allowed(s, s->tuning_sel)) return bail(fail(s, GG_ERR_INVALID_ARG, "tuning set and binning disagree"));
  if ((rc = set_shape(s, s->tuning_sel)) != GG_OK) return bail(rc);
  *out = s;
  return GG_OK;
}

gg_status gg_create(const gg_params *params, uint32_t n, const float *pos_radius, const float *vel, const float *mass,
                    int inputs_on_device, gg_sim **out) {
  uint32_t offs[2] = {0, n};
  return gg_create_batch(params, 1, offs, pos_radius, vel, mass, inputs_on_device, out);
}

gg_status gg_set_bodies(gg_sim *s, uint32_t env, uint32_t n_bodies, const gg_body *bodies) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (env >= s->n_envs || n_bodies > s->maxb || (n_bodies && !bodies))
    return fail(s, GG_ERR_INVALID_ARG, "gg_set_bodies: bad environment, count or pointer");
  std::vector<DevBody> hb(s->maxb);
  std::memset(hb.data(), 0, sizeof(DevBody) * s->maxb);
  for (uint32_t b = 0; b < n_bodies; ++b) {
    const gg_body &in = bodies[b];
    DevBody &o = hb[b];
    if (in.kind > GG_BODY_TUBE) return fail(s, GG_ERR_INVALID_ARG, "unknown body kind");
    if (in.kind == GG_BODY_GRID && in.is_free)
      return fail(s, GG_ERR_UNSUPPORTED, "GRID bodies are kinematic (free bodies are boxes)");
    if (in.is_free && !(in.mass > 0.f && in.inertia[0] > 0.f && in.inertia[1] > 0.f && in.inertia[2] > 0.f))
      return fail(s, GG_ERR_INVALID_ARG, "a free body needs a positive mass and inertia");
    double qn = std::sqrt((double)in.quat[0] * in.quat[0] + (double)in.quat[1] * in.quat[1] +
                          (double)in.quat[2] * in.quat[2] + (double)in.quat[3] * in.quat[3]);
    if (!(qn > 0.0) || !std::isfinite(qn)) return fail(s, GG_ERR_INVALID_ARG, "body quaternion must be non-zero");
    o.kind = in.kind;
    o.is_free = in.is_free;
    for (int k = 0; k < 12; ++k) o.shape[k] = in.shape[k];
    for (int k = 0; k < 3; ++k) {
      o.p[k] = in.pos[k];
      o.own_v[k] = o.v[k] = in.lin_vel[k];
      o.own_w[k] = o.w[k] = in.ang_vel[k];
      o.inertia[k] = in.inertia[k];
    }
    // keep the caller's float quaternion when it is already unit length to FP32 precision
    const bool unit = std::fabs(qn - 1.0) < 1e-6;
    for (int k = 0; k < 4; ++k) o.q[k] = unit ? in.quat[k] : (float)(in.quat[k] / qn);
    rot_from_quat(o.q, o.R);  // valid before the first step (gg_render); each step recomputes it
    if (in.kind == GG_BODY_BOX || in.kind == GG_BODY_BOX_MINUS_BOX)  // the solid lies inside box A
      o.bound_r = (float)std::sqrt((double)in.shape[0] * in.shape[0] + (double)in.shape[1] * in.shape[1] +
                                   (double)in.shape[2] * in.shape[2]);
    o.mass = in.mass;
    o.env = env;
    o.active = 1;
    o.fid = 0xffffffffu;
  }
  // free-body slots: release this environment's, then assign in body order
  std::vector<uint32_t> fgb = s->fgb;
  for (uint32_t &g : fgb)
    if (g != 0xffffffffu && g / s->maxb == env) g = 0xffffffffu;
  for (uint32_t b = 0; b < n_bodies; ++b) {
    if (!bodies[b].is_free) continue;
    uint32_t f = 0;
    while (f < s->F && fgb[f] != 0xffffffffu) ++f;
    if (f == s->F) return fail(s, GG_ERR_INVALID_ARG, "more free bodies than gg_params.max_free_bodies");
    fgb[f] = env * s->maxb + b;
    hb[b].fid = f;
  }
  GG_CUDA(s, cudaDeviceSynchronize());
  s->fgb = fgb;
  if (s->F) GG_CUDA(s, cudaMemcpy(s->a.fgb, fgb.data(), sizeof(uint32_t) * s->F, cudaMemcpyHostToDevice));
  for (uint32_t b = 0; b < s->maxb; ++b) {
    float *&t = s->traj[env * s->maxb + b];
    if (t) cudaFree(t);
    t = nullptr;
    float *&g = s->grids[env * s->maxb + b];
    if (g) cudaFree(g);
    g = nullptr;
  }
  GG_CUDA(s, cudaMemcpy(s->a.bodies + (size_t)env * s->maxb, hb.data(), sizeof(DevBody) * s->maxb,
                        cudaMemcpyHostToDevice));
  s->nbodies[env] = n_bodies;
  s->envs[env].nbodies = n_bodies;
  GG_CUDA(s, cudaMemcpy(&s->a.envs[env].nbodies, &n_bodies, sizeof(uint32_t), cudaMemcpyHostToDevice));
  return GG_OK;
}

gg_status gg_set_trajectory(gg_sim *s, uint32_t env, uint32_t body, uint32_t n_steps, const float *twist,
                            int twist_on_device) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (env >= s->n_envs || body >= s->nbodies[env] || (n_steps && !twist))
    return fail(s, GG_ERR_INVALID_ARG, "gg_set_trajectory: bad environment, body or pointer");
  GG_CUDA(s, cudaDeviceSynchronize());
  const uint32_t gb = env * s->maxb + body;
  float *&t = s->traj[gb];
  if (t) cudaFree(t);
  t = nullptr;
  if (n_steps) {
    cudaError_t e = cudaMalloc(&t, sizeof(float) * 6 * n_steps);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      t = nullptr;
      return fail(s, GG_ERR_OOM, "trajectory allocation failed");
    }
    GG_CUDA(s, cudaMemcpy(t, twist, sizeof(float) * 6 * n_steps,
                          twist_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  }
  DevCtrl c{};
  GG_CUDA(s, cudaMemcpy(&c, s->a.ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost));
  DevBody *db = s->a.bodies + gb;
  const float *tp = t;
  GG_CUDA(s, cudaMemcpy(&db->traj, &tp, sizeof(tp), cudaMemcpyHostToDevice));
  GG_CUDA(s, cudaMemcpy(&db->traj_len, &n_steps, sizeof(uint32_t), cudaMemcpyHostToDevice));
  GG_CUDA(s, cudaMemcpy(&db->traj_start, &c.step, sizeof(uint32_t), cudaMemcpyHostToDevice));
  return GG_OK;
}

gg_status gg_set_body_grid(gg_sim *s, uint32_t env, uint32_t body, const uint32_t dims[3], const float origin[3],
                           float spacing, const float *values, int on_device) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (env >= s->n_envs || body >= s->nbodies[env] || !dims || !origin || !values)
    return fail(s, GG_ERR_INVALID_ARG, "gg_set_body_grid: bad environment, body or pointer");
  if (dims[0] < 2 || dims[1] < 2 || dims[2] < 2 || !(spacing > 0.f) || !std::isfinite(spacing) ||
      !std::isfinite(origin[0]) || !std::isfinite(origin[1]) || !std::isfinite(origin[2]))
    return fail(s, GG_ERR_INVALID_ARG, "gg_set_body_grid: dims must be >= 2 and spacing > 0");
  const size_t count = (size_t)dims[0] * dims[1] * dims[2];
  if (count > ((size_t)1 << 31)) return fail(s, GG_ERR_INVALID_ARG, "gg_set_body_grid: more than 2^31 samples");
  const uint32_t gb = env * s->maxb + body;
  GG_CUDA(s, cudaDeviceSynchronize());
  DevBody hb;
  GG_CUDA(s, cudaMemcpy(&hb, s->a.bodies + gb, sizeof(DevBody), cudaMemcpyDeviceToHost));
  if (hb.kind != GG_BODY_GRID) return fail(s, GG_ERR_INVALID_ARG, "gg_set_body_grid: the body is not GG_BODY_GRID");
  float *&g = s->grids[gb];
  if (g) cudaFree(g);
  g = nullptr;
  cudaError_t e = cudaMalloc(&g, sizeof(float) * count);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    g = nullptr;
    return fail(s, GG_ERR_OOM, "grid allocation failed");
  }
  GG_CUDA(s, cudaMemcpy(g, values, sizeof(float) * count, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  for (int k = 0; k < 3; ++k) {
    hb.shape[k] = origin[k];
    hb.gn[k] = dims[k];
  }
  hb.shape[3] = spacing;
  hb.shape[4] = (float)(1.0 / (double)spacing);
  hb.grid = g;
  double far2 = 0.0;  // the sampled box's farthest corner from the body origin (no contact beyond the box)
  for (int k = 0; k < 3; ++k) {
    const double lo = origin[k], hi = origin[k] + (double)spacing * (dims[k] - 1);
    far2 += std::max(lo * lo, hi * hi);
  }
  hb.bound_r = (float)std::sqrt(far2);
  GG_CUDA(s, cudaMemcpy(s->a.bodies + gb, &hb, sizeof(DevBody), cudaMemcpyHostToDevice));
  return GG_OK;
}

gg_status gg_render(gg_sim *s, uint32_t env, const gg_camera *cam, float *out, int out_on_device, void *stream) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (!cam || !out || cam->struct_size != sizeof(gg_camera) || env >= s->n_envs)
    return fail(s, GG_ERR_INVALID_ARG, "gg_render: bad camera, output or environment");
  const gg_camera &C = *cam;
  if (C.kind > GG_CAMERA_DEPTH || C.width == 0 || C.height == 0 || C.width > 4096 || C.height > 4096)
    return fail(s, GG_ERR_INVALID_ARG, "gg_render: bad camera kind or size");
  gg::RenderArgs r{};
  r.kind = C.kind;
  r.W = C.width;
  r.H = C.height;
  if (C.kind == GG_CAMERA_HEIGHT) {
    if (!(C.extent[0] > 0.f) || !(C.extent[1] > 0.f) || !std::isfinite(C.extent[0]) || !std::isfinite(C.extent[1]))
      return fail(s, GG_ERR_INVALID_ARG, "gg_render: extents must be positive");
    // the oracle's order: step = extent / W; corner = centre - extent / 2
    r.sx = C.extent[0] / (float)C.width;
    r.sy = C.extent[1] / (float)C.height;
    r.bx = C.pos[0] - 0.5f * C.extent[0];
    r.by = C.pos[1] - 0.5f * C.extent[1];
    r.empty = C.empty;
  } else {
    if (!(C.fov_y > 0.f && C.fov_y < 3.14159f) || !(C.near_clip > 0.f) || !(C.far_clip > C.near_clip) ||
        !std::isfinite(C.far_clip))
      return fail(s, GG_ERR_INVALID_ARG, "gg_render: bad field of view or clip range");
    r.f = (float)(0.5 * (double)C.height / std::tan(0.5 * (double)C.fov_y));
    rot_from_quat(C.quat, r.R);
    for (int k = 0; k < 3; ++k) r.o[k] = C.pos[k];
    r.near = C.near_clip;
    r.far = C.far_clip;
    r.eps = C.march_eps > 0.f ? C.march_eps : 1e-4f;
    r.steps = C.march_steps ? C.march_steps : 64;
    r.mask = C.body_mask;
  }
  const size_t np = (size_t)C.width * C.height;
  if (np > s->render_px) {
    if (s->render_img) cudaFree(s->render_img);
    if (s->render_out) cudaFree(s->render_out);
    if (s->render_rays) cudaFree(s->render_rays);
    s->render_img = nullptr;
    s->render_out = nullptr;
    s->render_rays = nullptr;
    s->render_px = 0;
    if (cudaMalloc(&s->render_img, np * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&s->render_out, np * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s->render_rays, np * sizeof(float4)) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(s, GG_ERR_OOM, "gg_render: scratch allocation failed");
    }
    s->render_px = np;
  }
  r.rays = s->render_rays;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const gg::DevEnv &E = s->envs[env];
  float *dst = out_on_device ? out : s->render_out;
  GG_CUDA(s, gg::enqueue_render(s->a, E.off, E.n, env * s->maxb, s->nbodies[env], r, s->render_img, dst, st));
  if (!out_on_device) {
    GG_CUDA(s, cudaMemcpyAsync(out, dst, np * sizeof(float), cudaMemcpyDeviceToHost, st));
    GG_CUDA(s, cudaStreamSynchronize(st));
  }
  return GG_OK;
}

gg_status gg_set_particles(gg_sim *s, const float *pos_radius, const float *vel, int on_device, void *stream) {
  if (!s || !pos_radius) return s ? fail(s, GG_ERR_INVALID_ARG, "gg_set_particles: null positions") : GG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!s->n) return GG_OK;
  if (!on_device) {  // pinned host buffers: one kernel reads them over the host link
    const void *dp = pinned_device_ptr(pos_radius);
    const void *dv = vel ? pinned_device_ptr(vel) : nullptr;
    if (dp && (!vel || dv) && (reinterpret_cast<uintptr_t>(dp) & 15u) == 0) {
      GG_CUDA(s, gg::enqueue_state_in(s->a.pos_id, s->a.vel_id, static_cast<const float *>(dp),
                                      static_cast<const float *>(dv), s->n, st));
      return GG_OK;
    }
  }
  GG_CUDA(s, cudaMemcpyAsync(s->a.pos_id, pos_radius, sizeof(float4) * s->n, kind, st));
  if (vel) {
    const float *src = vel;
    if (!on_device) {
      GG_CUDA(s, cudaMemcpyAsync(s->vel3, vel, sizeof(float) * 3 * s->n, cudaMemcpyHostToDevice, st));
      src = s->vel3;
    }
    GG_CUDA(s, gg::enqueue_vel3_to_vel4(s->a.vel_id, src, s->n, st));
  }
  return GG_OK;
}

gg_status gg_step(gg_sim *s, uint32_t n_steps, void *stream) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (!s->tuned && n_steps) {
    gg_status rc = autotune(s, static_cast<cudaStream_t>(stream));
    if (rc != GG_OK) return rc;
  }
  if (!s->exec[s->timing]) {
    gg_status rc = capture(s);
    if (rc != GG_OK) return rc;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (uint32_t k = 0; k < n_steps; ++k) GG_CUDA(s, cudaGraphLaunch(s->exec[s->timing], st));
  s->steps += n_steps;
  return GG_OK;
}

gg_status gg_step_io(gg_sim *s, const float *pos_radius, const float *vel, float *out, void *stream) {
  if (!s || !pos_radius || !out) return s ? fail(s, GG_ERR_INVALID_ARG, "gg_step_io: null buffer") : GG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const void *dp = pinned_device_ptr(pos_radius);
  const void *dv = vel ? pinned_device_ptr(vel) : nullptr;
  void *dout = pinned_device_ptr(out);
  const bool one_graph = s->n && !s->timing && dp && (!vel || dv) && dout &&
                         (reinterpret_cast<uintptr_t>(dp) & 15u) == 0 && (reinterpret_cast<uintptr_t>(dout) & 15u) == 0;
  gg_status rc;
  if (!one_graph) {
    if ((rc = gg_set_particles(s, pos_radius, vel, 0, stream)) != GG_OK) return rc;
    if ((rc = gg_step(s, 1, stream)) != GG_OK) return rc;
    return gg_readback(s, GG_FIELD_POS_VEL, out, gg_field_bytes(s, GG_FIELD_POS_VEL), 0, stream);
  }
  if (!s->tuned && (rc = autotune(s, st)) != GG_OK) return rc;  // (may drop the graphs)
  if (!s->ctrl_host) GG_CUDA(s, cudaHostAlloc(reinterpret_cast<void **>(&s->ctrl_host), sizeof(DevCtrl), 0));
  DevCtrl *cd = static_cast<DevCtrl *>(pinned_device_ptr(s->ctrl_host));
  if (!cd) return fail(s, GG_ERR_INTERNAL, "gg_step_io: status mirror not mapped");
  if (!s->io_exec || s->io_ptr[0] != dp || s->io_ptr[1] != dv || s->io_ptr[2] != dout) {
    if (s->io_exec) cudaGraphExecDestroy(s->io_exec);
    s->io_exec = nullptr;
    const size_t n = s->n;
    GG_CUDA(s, cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = gg::enqueue_state_in(s->a.pos_id, s->a.vel_id, static_cast<const float *>(dp),
                                          static_cast<const float *>(dv), s->n, s->cap);
    if (e1 == cudaSuccess) e1 = gg::enqueue_step(s->a, s->ls, s->cap, nullptr);
    if (e1 == cudaSuccess)
      e1 = gg::enqueue_state_out(s->a.pos_id, s->a.vel_id, static_cast<float *>(dout),
                                 reinterpret_cast<float *>(static_cast<char *>(dout) + n * 16), s->n, s->a.ctrl, cd,
                                 s->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s->cap, &g);
    if (e1 == cudaSuccess && e2 == cudaSuccess) e1 = cudaGraphInstantiate(&s->io_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(s, e1 != cudaSuccess ? e1 : e2, "gg_step_io capture");
    s->io_ptr[0] = dp;
    s->io_ptr[1] = dv;
    s->io_ptr[2] = dout;
  }
  GG_CUDA(s, cudaGraphLaunch(s->io_exec, st));
  s->steps += 1;
  GG_CUDA(s, cudaStreamSynchronize(st));
  return status_from_flags(s, s->ctrl_host->status);
}

gg_status gg_sync(gg_sim *s, void *stream) {
  if (!s) return GG_ERR_INVALID_ARG;
  DevCtrl c{};
  gg_status rc = read_ctrl(s, &c, static_cast<cudaStream_t>(stream));
  if (rc != GG_OK) return rc;
  return status_from_flags(s, c.status);
}

size_t gg_field_bytes(const gg_sim *s, gg_field f) {
  if (!s) return 0;
  const size_t n = s->n, nbt = (size_t)s->n_envs * s->maxb;
  switch (f) {
  case GG_FIELD_POS: return n * 16;
  case GG_FIELD_VEL: return n * 12;
  case GG_FIELD_BODY_STATE: return nbt * 16 * 4;
  case GG_FIELD_BODY_WRENCH: return (size_t)s->H * nbt * 6 * 4;
  case GG_FIELD_CELL_KEY: return n * 4;
  case GG_FIELD_SORT_PERM: return n * 4;
  case GG_FIELD_CELL_START: return ((size_t)s->nh_total + 1) * 4;
  case GG_FIELD_CONTACTS: return n * (2 + s->K + s->Kb) * 4;
  case GG_FIELD_CONTACT_GEOM: return n * s->K * 16;
  case GG_FIELD_CONTACT_IMPULSE: return n * s->K * 12;
  case GG_FIELD_BODY_CONTACT_GEOM: return n * s->Kb * 32;
  case GG_FIELD_BODY_CONTACT_IMPULSE: return n * s->Kb * 12;
  case GG_FIELD_STATS: return sizeof(gg_stats);
  case GG_FIELD_STATE: return sizeof(StateHeader) + n * 32 + nbt * 16 * 4;
  case GG_FIELD_POS_VEL: return n * 28;
  }
  return 0;
}

gg_status gg_readback(gg_sim *s, gg_field f, void *dst, size_t bytes, int dst_on_device, void *stream) {
  if (!s) return GG_ERR_INVALID_ARG;
  const size_t need = gg_field_bytes(s, f);
  if (need == 0 || bytes != need || !dst) return fail(s, GG_ERR_INVALID_ARG, "gg_readback: bad field, size or pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind d2x = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n = s->n, nbt = (size_t)s->n_envs * s->maxb;
  // device-side producer: write straight into dst when it is device memory, else into staging
  auto target = [&](size_t b, void **t) -> gg_status {
    if (dst_on_device) {
      *t = dst;
      return GG_OK;
    }
    gg_status rc = ensure_staging(s, b);
    *t = s->staging;
    return rc;
  };
  gg_status rc = GG_OK;
  void *t = nullptr;
  bool ctrl_done = false;  // the control word already came back with the data (pinned path)
  switch (f) {
  case GG_FIELD_POS:
    if (n) GG_CUDA(s, cudaMemcpyAsync(dst, s->a.pos_id, need, d2x, st));
    break;
  case GG_FIELD_VEL:
    if ((rc = target(need, &t)) != GG_OK) return rc;
    GG_CUDA(s, gg::enqueue_vel4_to_vel3(s->a.vel_id, static_cast<float *>(t), s->n, st));
    if (!dst_on_device && n) GG_CUDA(s, cudaMemcpyAsync(dst, t, need, cudaMemcpyDeviceToHost, st));
    break;
  case GG_FIELD_POS_VEL:
    if (!n) break;
    if (!dst_on_device) {  // a pinned host buffer: one kernel writes it over the host link
      char *dd = static_cast<char *>(pinned_device_ptr(dst));
      if (dd && (reinterpret_cast<uintptr_t>(dd) & 15u) == 0) {
        if (!s->ctrl_host) GG_CUDA(s, cudaHostAlloc(reinterpret_cast<void **>(&s->ctrl_host), sizeof(DevCtrl), 0));
        DevCtrl *cd = static_cast<DevCtrl *>(pinned_device_ptr(s->ctrl_host));
        GG_CUDA(s, gg::enqueue_state_out(s->a.pos_id, s->a.vel_id, reinterpret_cast<float *>(dd),
                                         reinterpret_cast<float *>(dd + n * 16), s->n, s->a.ctrl, cd, st));
        if (cd) {
          GG_CUDA(s, cudaStreamSynchronize(st));
          ctrl_done = true;
        }
        break;
      }
    }
    if ((rc = target(need, &t)) != GG_OK) return rc;
    GG_CUDA(s, cudaMemcpyAsync(t, s->a.pos_id, n * 16, cudaMemcpyDeviceToDevice, st));
    GG_CUDA(s, gg::enqueue_vel4_to_vel3(s->a.vel_id, reinterpret_cast<float *>(static_cast<char *>(t) + n * 16),
                                        s->n, st));
    if (!dst_on_device) GG_CUDA(s, cudaMemcpyAsync(dst, t, need, cudaMemcpyDeviceToHost, st));
    break;
  case GG_FIELD_BODY_STATE:
    if ((rc = target(need, &t)) != GG_OK) return rc;
    GG_CUDA(s, gg::enqueue_body_state(s->a.bodies, (uint32_t)nbt, static_cast<float *>(t), st));
    if (!dst_on_device) GG_CUDA(s, cudaMemcpyAsync(dst, t, need, cudaMemcpyDeviceToHost, st));
    break;
  case GG_FIELD_BODY_WRENCH: {
    const size_t row = nbt * 6 * sizeof(float);
    const uint64_t H = s->H;
    const uint64_t oldest = s->steps >= H ? s->steps % H : 0;
    char *d = static_cast<char *>(dst);
    const char *src = reinterpret_cast<const char *>(s->a.wrench);
    if (s->steps < H) {  // newest step in the last row: zero rows, then steps 0 .. steps-1
      const size_t z = (H - s->steps) * row;
      if (dst_on_device)
        GG_CUDA(s, cudaMemsetAsync(d, 0, z, st));
      else
        std::memset(d, 0, z);
      if (s->steps) GG_CUDA(s, cudaMemcpyAsync(d + z, src, s->steps * row, d2x, st));
    } else if (oldest) {  // ring has wrapped: rows [oldest, H) then [0, oldest)
      GG_CUDA(s, cudaMemcpyAsync(d, src + oldest * row, (H - oldest) * row, d2x, st));
      GG_CUDA(s, cudaMemcpyAsync(d + (H - oldest) * row, src, oldest * row, d2x, st));
    } else {
      GG_CUDA(s, cudaMemcpyAsync(d, src, H * row, d2x, st));
    }
    break;
  }
  case GG_FIELD_CELL_KEY:
    if (n) GG_CUDA(s, cudaMemcpyAsync(dst, s->a.key_id, need, d2x, st));
    break;
  case GG_FIELD_SORT_PERM:
    if (s->a.lists) GG_CUDA(s, gg::enqueue_sort_from_keys(s->a, st));  // binned by lists: sort on demand
    if (n) GG_CUDA(s, cudaMemcpyAsync(dst, s->a.sid, need, d2x, st));
    break;
  case GG_FIELD_CELL_START:
    if (s->a.lists) GG_CUDA(s, gg::enqueue_sort_from_keys(s->a, st));
    GG_CUDA(s, cudaMemcpyAsync(dst, s->a.start, need, d2x, st));
    break;
  case GG_FIELD_CONTACTS:
  case GG_FIELD_CONTACT_GEOM:
  case GG_FIELD_CONTACT_IMPULSE:
  case GG_FIELD_BODY_CONTACT_GEOM:
  case GG_FIELD_BODY_CONTACT_IMPULSE: {
    if ((rc = target(need, &t)) != GG_OK) return rc;
    uint32_t *rows = f == GG_FIELD_CONTACTS ? static_cast<uint32_t *>(t) : nullptr;
    float *geom = f == GG_FIELD_CONTACT_GEOM ? static_cast<float *>(t) : nullptr;
    float *lam = f == GG_FIELD_CONTACT_IMPULSE ? static_cast<float *>(t) : nullptr;
    float *bgeom = f == GG_FIELD_BODY_CONTACT_GEOM ? static_cast<float *>(t) : nullptr;
    float *blam = f == GG_FIELD_BODY_CONTACT_IMPULSE ? static_cast<float *>(t) : nullptr;
    GG_CUDA(s, gg::enqueue_export_contacts(s->a, rows, geom, lam, bgeom, blam, st));
    if (!dst_on_device && n) GG_CUDA(s, cudaMemcpyAsync(dst, t, need, cudaMemcpyDeviceToHost, st));
    break;
  }
  case GG_FIELD_STATS: {
    if (dst_on_device) return fail(s, GG_ERR_UNSUPPORTED, "GG_FIELD_STATS is host-only");
    DevCtrl c{};
    if ((rc = read_ctrl(s, &c, st)) != GG_OK) return rc;
    gg_stats out{};
    out.steps = s->steps;
    out.n_pp = c.n_pp;
    out.n_body = c.n_body;
    out.max_pp = c.max_pp;
    out.max_body = c.max_body;
    out.status_flags = c.status;
    out.n_active = c.n_active;
    uint32_t bits = c.max_psi_bits;
    std::memcpy(&out.max_psi, &bits, 4);
    std::memcpy(dst, &out, sizeof(out));
    return status_from_flags(s, c.status);
  }
  case GG_FIELD_STATE: {
    if ((rc = target(need, &t)) != GG_OK) return rc;
    StateHeader h{kStateMagic, s->n, s->n_envs, s->maxb, s->steps, {0, 0}};
    char *d = static_cast<char *>(t);
    GG_CUDA(s, cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    GG_CUDA(s, cudaStreamSynchronize(st));  // h lives on this stack frame
    if (n) {
      GG_CUDA(s, cudaMemcpyAsync(d + sizeof(h), s->a.pos_id, n * 16, cudaMemcpyDeviceToDevice, st));
      GG_CUDA(s, cudaMemcpyAsync(d + sizeof(h) + n * 16, s->a.vel_id, n * 16, cudaMemcpyDeviceToDevice, st));
    }
    GG_CUDA(s, gg::enqueue_body_state(s->a.bodies, (uint32_t)nbt, reinterpret_cast<float *>(d + sizeof(h) + n * 32), st));
    if (!dst_on_device) GG_CUDA(s, cudaMemcpyAsync(dst, t, need, cudaMemcpyDeviceToHost, st));
    break;
  }
  default:
    return fail(s, GG_ERR_INVALID_ARG, "unknown field");
  }
  if (dst_on_device) return GG_OK;
  DevCtrl c{};
  if (ctrl_done)
    c = *s->ctrl_host;
  else if ((rc = read_ctrl(s, &c, st)) != GG_OK)
    return rc;
  return status_from_flags(s, c.status);
}

gg_status gg_set_state(gg_sim *s, const void *state, size_t bytes, int on_device, void *stream) {
  if (!s || !state) return s ? fail(s, GG_ERR_INVALID_ARG, "gg_set_state: null state") : GG_ERR_INVALID_ARG;
  if (bytes != gg_field_bytes(s, GG_FIELD_STATE)) return fail(s, GG_ERR_INVALID_ARG, "gg_set_state: size mismatch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GG_CUDA(s, cudaStreamSynchronize(st));
  GG_CUDA(s, cudaDeviceSynchronize());
  std::vector<char> h(bytes);
  GG_CUDA(s, cudaMemcpy(h.data(), state, bytes, on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  StateHeader hd;
  std::memcpy(&hd, h.data(), sizeof(hd));
  if (hd.magic != kStateMagic || hd.n != s->n || hd.n_envs != s->n_envs || hd.maxb != s->maxb)
    return fail(s, GG_ERR_INVALID_ARG, "gg_set_state: checkpoint from a different simulation");
  const size_t n = s->n, nbt = (size_t)s->n_envs * s->maxb;
  if (n) {
    GG_CUDA(s, cudaMemcpy(s->a.pos_id, h.data() + sizeof(hd), n * 16, cudaMemcpyHostToDevice));
    GG_CUDA(s, cudaMemcpy(s->a.vel_id, h.data() + sizeof(hd) + n * 16, n * 16, cudaMemcpyHostToDevice));
  }
  std::vector<DevBody> bd(nbt);
  GG_CUDA(s, cudaMemcpy(bd.data(), s->a.bodies, sizeof(DevBody) * nbt, cudaMemcpyDeviceToHost));
  const float *bs = reinterpret_cast<const float *>(h.data() + sizeof(hd) + n * 32);
  for (size_t b = 0; b < nbt; ++b) {
    const float *q = bs + 16 * b;
    for (int k = 0; k < 3; ++k) bd[b].p[k] = q[k];
    for (int k = 0; k < 4; ++k) bd[b].q[k] = q[3 + k];
    for (int k = 0; k < 3; ++k) bd[b].own_v[k] = q[7 + k];
    for (int k = 0; k < 3; ++k) bd[b].own_w[k] = q[10 + k];
  }
  GG_CUDA(s, cudaMemcpy(s->a.bodies, bd.data(), sizeof(DevBody) * nbt, cudaMemcpyHostToDevice));
  DevCtrl c{};
  GG_CUDA(s, cudaMemcpy(&c, s->a.ctrl, sizeof(c), cudaMemcpyDeviceToHost));
  c.step = (uint32_t)hd.steps;
  GG_CUDA(s, cudaMemcpy(s->a.ctrl, &c, sizeof(c), cudaMemcpyHostToDevice));
  s->steps = hd.steps;
  return GG_OK;
}

gg_status gg_tape_reserve(gg_sim *s, uint32_t n_steps, uint32_t K) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (s->n_envs != 1) return fail(s, GG_ERR_UNSUPPORTED, "differentiation needs a single environment");
  if (s->F) return fail(s, GG_ERR_UNSUPPORTED, "differentiation of free rigid bodies is not supported");
  if (s->a.lit) return fail(s, GG_ERR_UNSUPPORTED, "differentiation with pja_weight = 1 is not supported");
  if (n_steps == 0 || K == 0) return fail(s, GG_ERR_INVALID_ARG, "gg_tape_reserve: n_steps and K must be > 0");
  GG_CUDA(s, cudaDeviceSynchronize());
  for (void *p : s->ad.allocs) cudaFree(p);
  s->ad.allocs.clear();
  s->ad.taped = 0;
  const size_t n = s->n, I = s->ls.iters, KN = (size_t)s->K * n, KbN = (size_t)s->Kb * n;
  const uint32_t nblk = gg::adjoint_blocks(s->n);
  s->ad.state_bytes = (state_bytes(s) + 255) / 256 * 256;
  const size_t nck = (n_steps + K - 1) / K;
  const size_t slots = std::min(K, n_steps);  // steps of a segment, each with its own tape
  gg::Tape &tp = s->ad.tp;
  gg::AdjArgs &d = s->ad.d;
  gg_status rc;
  if ((rc = ad_alloc(s, &s->ad.ckpt, nck * s->ad.state_bytes)) || (rc = ad_alloc(s, &s->ad.seg, (size_t)K * s->ad.state_bytes)) ||
      (rc = ad_alloc(s, &s->ad.fin, s->ad.state_bytes)) || (rc = ad_alloc(s, &tp.Uh, slots * (I + 1) * n)) ||
      (rc = ad_alloc(s, &tp.lamh, slots * (I + 1) * 3 * KN)) || (rc = ad_alloc(s, &tp.blamh, slots * (I + 1) * 3 * KbN)) ||
      (rc = ad_alloc(s, &s->ad.ccount, slots * n)) || (rc = ad_alloc(s, &s->ad.cj, slots * KN)) ||
      (rc = ad_alloc(s, &s->ad.cn, slots * KN)) || (rc = ad_alloc(s, &s->ad.bj, slots * KbN)) ||
      (rc = ad_alloc(s, &s->ad.bn, slots * KbN)) || (rc = ad_alloc(s, &s->ad.bxc, slots * KbN)) ||
      (rc = ad_alloc(s, &d.twin, KN)) || (rc = ad_alloc(s, &d.Ubar[0], n)) || (rc = ad_alloc(s, &d.Ubar[1], n)) ||
      (rc = ad_alloc(s, &d.ubar[0], 3 * KN)) || (rc = ad_alloc(s, &d.ubar[1], 3 * KN)) || (rc = ad_alloc(s, &d.Lbar, 3 * KN)) || (rc = ad_alloc(s, &d.bLbar, 3 * KbN)) ||
      (rc = ad_alloc(s, &d.psibar, KN)) || (rc = ad_alloc(s, &d.nbar, 3 * KN)) || (rc = ad_alloc(s, &d.bpsibar, KbN)) ||
      (rc = ad_alloc(s, &d.bnbar, 3 * KbN)) || (rc = ad_alloc(s, &d.bxcbar, 3 * KbN)) ||
      (rc = ad_alloc(s, &d.basebar, n)) || (rc = ad_alloc(s, &d.xbar_s, n)) || (rc = ad_alloc(s, &d.xbar, n)) ||
      (rc = ad_alloc(s, &d.vbar, n)) || (rc = ad_alloc(s, &d.part, (I + 1) * nblk * 10)) ||
      (rc = ad_alloc(s, &d.pose_bar, 6)) || (rc = ad_alloc(s, &d.dtwist, (size_t)n_steps * 6)) ||
      (rc = ad_alloc(s, &d.mubar, 1)))
    return rc;
  d.tp = tp;
  d.I = (uint32_t)I;
  d.nblk = nblk;
  d.tool = 0xffffffffu;
  s->ad.n_steps = n_steps;
  s->ad.K = K;
  s->ad.slots = (uint32_t)slots;
  return GG_OK;
}

gg_status gg_step_taped(gg_sim *s, uint32_t tool_body, uint32_t n_steps, void *stream) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (!s->ad.ckpt || n_steps == 0 || n_steps > s->ad.n_steps)
    return fail(s, GG_ERR_INVALID_ARG, "gg_step_taped: reserve at least n_steps with gg_tape_reserve first");
  if (tool_body >= s->nbodies[0]) return fail(s, GG_ERR_INVALID_ARG, "gg_step_taped: no such body");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (uint32_t k = 0; k < n_steps; ++k) {
    if (k % s->ad.K == 0) {
      gg_status rc = save_state(s, s->ad.ckpt + (size_t)(k / s->ad.K) * s->ad.state_bytes, st);
      if (rc != GG_OK) return rc;
    }
    gg_status rc = gg_step(s, 1, stream);
    if (rc != GG_OK) return rc;
  }
  gg_status rc = save_state(s, s->ad.fin, st);
  if (rc != GG_OK) return rc;
  s->ad.taped = n_steps;
  s->ad.tool = tool_body;
  s->ad.d.tool = tool_body;  // environment 0: global index = local index
  return GG_OK;
}

gg_status gg_backward(gg_sim *s, const float *dL_dpos, const float *dL_dvel, const float *dL_dpose, float *dL_dtwist,
                      float *dL_dmu, int on_device, void *stream) {
  if (!s) return GG_ERR_INVALID_ARG;
  if (!s->ad.taped) return fail(s, GG_ERR_INVALID_ARG, "gg_backward: no taped run (gg_step_taped)");
  if (!dL_dpos || !dL_dtwist || !dL_dmu) return fail(s, GG_ERR_INVALID_ARG, "gg_backward: null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gg::AdjArgs &d = s->ad.d;
  const uint32_t N = s->ad.taped, K = s->ad.K, n = s->n;
  const cudaMemcpyKind h2x = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind x2h = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // seeds: dL/dx_N, dL/dv_N (float3 -> float4, id order)
  const float *src = dL_dpos;
  if (!on_device && n) {
    GG_CUDA(s, cudaMemcpyAsync(s->vel3, dL_dpos, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
    src = s->vel3;
  }
  GG_CUDA(s, gg::enqueue_pack3(d.xbar, src, n, st));
  src = dL_dvel;
  if (dL_dvel && !on_device && n) {
    GG_CUDA(s, cudaMemcpyAsync(s->vel3, dL_dvel, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
    src = s->vel3;
  }
  GG_CUDA(s, gg::enqueue_pack3(d.vbar, src, n, st));
  // seed of the tool pose: dL/dp, and dL/dq turned into a world-frame rotation adjoint
  // (q' = exp(dtheta / 2) q:  rbar_k = 1/2 <(0, e_k) q, dL/dq>)
  float pose6[6] = {0, 0, 0, 0, 0, 0};
  if (dL_dpose) {
    float g7[7];
    GG_CUDA(s, cudaMemcpyAsync(g7, dL_dpose, sizeof(g7), h2x == cudaMemcpyHostToDevice ? cudaMemcpyHostToHost
                                                                                     : cudaMemcpyDeviceToHost, st));
    DevBody tb;  // the tool's final pose, from the final state (bodies follow the 32 n bytes of particles)
    GG_CUDA(s, cudaMemcpyAsync(&tb, s->ad.fin + (size_t)n * 32 + (size_t)s->ad.tool * sizeof(DevBody), sizeof(DevBody),
                               cudaMemcpyDeviceToHost, st));
    GG_CUDA(s, cudaStreamSynchronize(st));
    const float w = tb.q[0], x = tb.q[1], y = tb.q[2], z = tb.q[3];
    const float *gq = g7 + 3;
    pose6[0] = g7[0];
    pose6[1] = g7[1];
    pose6[2] = g7[2];
    pose6[3] = 0.5f * (-x * gq[0] + w * gq[1] - z * gq[2] + y * gq[3]);
    pose6[4] = 0.5f * (-y * gq[0] + z * gq[1] + w * gq[2] - x * gq[3]);
    pose6[5] = 0.5f * (-z * gq[0] - y * gq[1] + x * gq[2] + w * gq[3]);
  }
  GG_CUDA(s, cudaMemcpyAsync(d.pose_bar, pose6, sizeof(pose6), cudaMemcpyHostToDevice, st));
  GG_CUDA(s, cudaMemsetAsync(d.mubar, 0, sizeof(double), st));
  GG_CUDA(s, cudaStreamSynchronize(st));  // pose6 lives on this stack frame
  // Each checkpoint segment is recomputed with taped full steps, every step keeping its
  // contact arrays and its sweeps' iterates in a slot of its own, and then reversed from
  // its last step: the body frames of the step restored, then its adjoint.  One graph
  // per slot and direction (the slot's arrays are baked in; the adjoint reads the step
  // index from the step counter restored with the state), captured when first needed,
  // so that the host captures the next graph while the device runs the previous one.
  const uint32_t slots = s->ad.slots;
  std::vector<cudaGraphExec_t> fwd(slots, nullptr), adj(slots, nullptr);
  struct ExecGuard {  // the graphs are destroyed on every return below, after their launches
    std::vector<cudaGraphExec_t> *v[2];
    cudaStream_t st;
    ~ExecGuard() {
      cudaStreamSynchronize(st);
      for (auto *x : v)
        for (cudaGraphExec_t g : *x)
          if (g) cudaGraphExecDestroy(g);
    }
  } guard{{&fwd, &adj}, st};
  const gg::DevCtrl *ctrl0 = reinterpret_cast<const gg::DevCtrl *>(
      s->ad.ckpt + (size_t)n * 32 + (size_t)s->n_envs * s->maxb * sizeof(DevBody));
  auto launch_slot = [&](bool reverse, uint32_t slot) -> gg_status {
    cudaGraphExec_t &x = reverse ? adj[slot] : fwd[slot];
    if (!x) {
      const gg::StepArgs ak = slot_args(s, slot);
      gg::AdjArgs dk = d;
      dk.tp = slot_tape(s, slot);
      // the forward graph first saves the step's start state into the slot, the reverse
      // graph first restores it
      const gg::CopyRegions cr = state_regions(s, s->ad.seg + (size_t)slot * s->ad.state_bytes, !reverse);
      GG_CUDA(s, cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
      cudaError_t e1 = gg::enqueue_copy_regions(cr, s->cap);
      if (e1 == cudaSuccess && !reverse) {
        e1 = gg::enqueue_step(ak, s->ls, s->cap, nullptr, &dk.tp, true);
      } else if (e1 == cudaSuccess) {
        e1 = gg::enqueue_prep_bodies(ak, s->cap);
        if (e1 == cudaSuccess) e1 = gg::enqueue_adjoint_step(ak, dk, ctrl0, N, s->cap);
      }
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(s->cap, &g);
      if (e1 == cudaSuccess && e2 == cudaSuccess) e1 = cudaGraphInstantiate(&x, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e1 != cudaSuccess || e2 != cudaSuccess)
        return cuda_fail(s, e1 != cudaSuccess ? e1 : e2, "capturing the reverse pass");
    }
    GG_CUDA(s, cudaGraphLaunch(x, st));
    return GG_OK;
  };
  // An error inside the segment loop would leave the simulation at an intermediate
  // checkpoint: put the end state of the taped run back on every return before the
  // loop completes (destroyed before `guard`, so the copy is queued before its wait).
  struct FinGuard {
    gg_sim *s;
    cudaStream_t st;
    bool done;
    ~FinGuard() {
      if (!done) (void)restore_state(s, s->ad.fin, st);
    }
  } fin_guard{s, st, false};
  const uint32_t nseg = (N + K - 1) / K;
  for (int seg = (int)nseg - 1; seg >= 0; --seg) {
    const uint32_t k0 = (uint32_t)seg * K, k1 = std::min(k0 + K, N);
    gg_status rc = restore_state(s, s->ad.ckpt + (size_t)seg * s->ad.state_bytes, st);
    if (rc != GG_OK) return rc;
    for (uint32_t k = k0; k < k1; ++k)  // taped recompute, each step's start state kept
      if ((rc = launch_slot(false, k - k0)) != GG_OK) return rc;
    for (int k = (int)k1 - 1; k >= (int)k0; --k)  // the steps' adjoints, last first
      if ((rc = launch_slot(true, (uint32_t)(k - k0))) != GG_OK) return rc;
  }

  fin_guard.done = true;
  gg_status rc = restore_state(s, s->ad.fin, st);
  if (rc != GG_OK) return rc;
  GG_CUDA(s, cudaMemcpyAsync(dL_dtwist, d.dtwist, sizeof(float) * 6 * N, x2h, st));
  double mu = 0.0;
  GG_CUDA(s, cudaMemcpyAsync(&mu, d.mubar, sizeof(double), cudaMemcpyDeviceToHost, st));
  GG_CUDA(s, cudaStreamSynchronize(st));
  const float muf = (float)mu;
  GG_CUDA(s, cudaMemcpy(dL_dmu, &muf, sizeof(float), on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
  DevCtrl c{};
  rc = read_ctrl(s, &c, st);
  if (rc != GG_OK) return rc;
  return status_from_flags(s, c.status);
}

}  // extern "C"
