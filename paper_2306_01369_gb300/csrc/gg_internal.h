// gg_internal.h -- launchers shared by the C ABI and the kernels (not installed).
#pragma once
#include <cuda_runtime.h>

#include "gg_device.cuh"

namespace gg {

// One kernel launch.  With `pdl` the launch asks for programmatic serialization with
// the stream's previous kernel; the kernel must begin with pdl_enter (it then still
// waits for that kernel's completion before touching memory; what overlaps is its
// launch and the predecessor's tail).  Only kernels follow kernels with pdl set.
template <typename... P, typename... A>
inline cudaError_t launch(bool pdl, void (*k)(P...), dim3 grid, unsigned block, size_t smem, cudaStream_t st,
                          A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Launch shape of the step; any choice gives bit-identical results.
struct LaunchShape {
  uint32_t iters;       // projected-Jacobi iterations
  int pja_block;        // threads per block of k_pja (one launch per sweep)
  int fused_block;      // > 0: all sweeps in one cooperative launch of this block size ...
  uint32_t fused_grid;  // ... and this many blocks (all resident); 0: one launch per sweep
  uint32_t lists;       // binning: 0 counting sort, 1 linked list per bucket (Alg. 2)
  uint32_t lean;        // per-launch sweeps capped at 40 registers (more resident warps: pays
                        // when the working set spills out of L2, costs when it fits)
  uint32_t half;        // pair search over half the stencil in two passes instead of k_contacts
  uint32_t detect;      // detection and all sweeps in one cooperative launch (fused_grid blocks)
  uint32_t serp;        // serpentine sweeps: every other per-launch sweep runs its blocks in reverse
  uint32_t pre;         // per-launch sweeps load the first round's records with the counts
  uint32_t one;         // OneLoop: every iteration re-walks the cells and computes the responses
};
int fused_pja_blocks_per_sm(int block);
int detect_sweeps_blocks_per_sm(bool lists, uint32_t K);

// ev (optional): 5 events recorded at the stage boundaries of the step.
// tape (optional): keep every sweep's iterates; unless `whole`, stop after the sweeps
// (no integration, wrench or pose update).  With `whole` the taped step is a full step.
cudaError_t enqueue_step(const StepArgs &a, const LaunchShape &ls, cudaStream_t st, cudaEvent_t *ev = nullptr,
                         const Tape *tape = nullptr, bool whole = false);
// the body frames and velocities of the step in the device step counter (as the step's
// binning kernel sets them), for an adjoint run on a restored state
cudaError_t enqueue_prep_bodies(const StepArgs &a, cudaStream_t st);
uint32_t kernels_per_step(const StepArgs &a, const LaunchShape &ls);
// the counting sort of the keys of the last binning (for the sort-order readbacks when
// the step bins by linked lists)
cudaError_t enqueue_sort_from_keys(const StepArgs &a, cudaStream_t st);
// The adjoint of one step, on that step's start state with its body frames set
// (enqueue_prep_bodies) and with the contact arrays and tape its taped forward left;
// the step index is the device step counter less ctrl0->step (the counter saved with
// the taped run's first checkpoint), so the enqueued work does not depend on it.
cudaError_t enqueue_adjoint_step(const StepArgs &a, const AdjArgs &d, const DevCtrl *ctrl0, uint32_t n_taped,
                                 cudaStream_t st);
uint32_t adjoint_blocks(uint32_t n);
// up to four regions of 32-bit words (unused ones with zero words), copied in one launch
struct CopyRegions {
  uint32_t *dst[4];
  const uint32_t *src[4];
  size_t words[4];
};
cudaError_t enqueue_copy_regions(const CopyRegions &c, cudaStream_t st);
// Depth observation (gg_render): everything the kernels need, precomputed on the host.
struct RenderArgs {
  uint32_t kind, W, H;
  float bx, by, sx, sy, empty;  // height camera: first pixel centre's corner, pixel steps, empty value
  float o[3], R[9], f;          // depth camera: origin, rotation camera -> world, focal length (pixels)
  float near, far, eps;
  uint32_t mask, steps;
  float4 *rays;                 // depth camera: per-pixel unit ray (scratch, W * H)
};
cudaError_t enqueue_render(const StepArgs &a, uint32_t env_off, uint32_t env_n, uint32_t gb0, uint32_t nb,
                           const RenderArgs &c, uint32_t *img, float *out, cudaStream_t st);
cudaError_t enqueue_pack3(float4 *dst, const float *src3, uint32_t n, cudaStream_t st);
cudaError_t enqueue_export_contacts(const StepArgs &a, uint32_t *rows, float *geom, float *lam, float *bgeom,
                                    float *blam, cudaStream_t st);
cudaError_t enqueue_vel3_to_vel4(float4 *vel_id, const float *vel3, uint32_t n, cudaStream_t st);
// pos: float[n][4] (16-byte aligned), vel: float[n][3]; device-accessible host memory;
// ctrl_out (optional, device-accessible host memory): receives a copy of *ctrl
cudaError_t enqueue_state_out(const float4 *pos_id, const float4 *vel_id, float *pos, float *vel, uint32_t n,
                              const DevCtrl *ctrl, DevCtrl *ctrl_out, cudaStream_t st);
cudaError_t enqueue_state_in(float4 *pos_id, float4 *vel_id, const float *pos, const float *vel, uint32_t n,
                             cudaStream_t st);
cudaError_t enqueue_vel4_to_vel3(const float4 *vel_id, float *vel3, uint32_t n, cudaStream_t st);
cudaError_t enqueue_body_state(const DevBody *bodies, uint32_t nbt, float *out, cudaStream_t st);

}  // namespace gg
