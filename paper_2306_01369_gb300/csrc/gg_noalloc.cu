// gg_noalloc.cu -- binning and bucket sort of one particle set with no device
// allocation, for callers that cannot call cudaMalloc themselves or let a library
// do it: code that runs inside a framework's memory pool or an allocator-free
// real-time loop, hosts where every device byte is budgeted up front, and
// plug-ins that are handed device pointers but not allowed to allocate.
//
// The caller passes device pointers to its inputs and outputs only.  The scratch
// the sort needs (bucket histogram, scan block sums, unsorted slot list) lives in
// the file-scope array g_noalloc_scratch below, which every GPU that loads this
// library holds until the process exits.  Sizes are limited by that array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/gg.h"
#include "gg_device.cuh"

namespace {

constexpr uint32_t kNAThreads = 256;
constexpr uint32_t kNAItems = 16;
constexpr uint32_t kNATile = kNAThreads * kNAItems;
constexpr uint32_t kNABuckets = GG_NOALLOC_MAX_BUCKETS;                   // histogram capacity
constexpr uint32_t kNABlocks = kNABuckets / kNATile;                      // scan blocks at capacity
constexpr uint32_t kNAWords = kNABuckets + kNABlocks + GG_NOALLOC_MAX_PARTICLES;

static_assert(kNABuckets % kNATile == 0, "bucket capacity must be a whole number of scan tiles");
static_assert(kNABlocks <= 1024, "block sums are scanned by one block");

// Scratch shared by every call on a device: [histogram | block sums | unsorted slots].
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNAWords];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
uint32_t *g_scratch_ptr[kMaxDevices] = {};

__global__ void na_clear(uint32_t *cnt, uint32_t words) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) cnt[i] = 0u;
}

__global__ void na_key(const float4 *pos, uint32_t n, float inv_cell, uint32_t nh, uint32_t *key, uint32_t *cnt) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = pos[i];
  const uint32_t k = gg::hash_cell(gg::cell_of(p.x, inv_cell), gg::cell_of(p.y, inv_cell), gg::cell_of(p.z, inv_cell), nh);
  key[i] = k;
  atomicAdd(&cnt[k], 1u);
}

__device__ __forceinline__ uint32_t na_warp_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive block scan; returns this thread's offset and the block total in *total.
__device__ __forceinline__ uint32_t na_block_scan(uint32_t v, uint32_t *total) {
  __shared__ uint32_t ws[32];
  __shared__ uint32_t tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t inc = na_warp_scan(v);
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const uint32_t s = lane < nw ? ws[lane] : 0u;
    const uint32_t si = na_warp_scan(s);
    if (lane < nw) ws[lane] = si - s;
    if (lane == 31) tot = si;
  }
  __syncthreads();
  const uint32_t r = ws[wid] + inc - v;
  *total = tot;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kNAThreads) na_reduce(const uint32_t *cnt, uint32_t *bsum) {
  const uint32_t base = blockIdx.x * kNATile + threadIdx.x * kNAItems;
  uint32_t s = 0;
#pragma unroll
  for (uint32_t k = 0; k < kNAItems; ++k) s += cnt[base + k];
  uint32_t total;
  (void)na_block_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) na_top(uint32_t *bsum, uint32_t nblk, uint32_t *start, uint32_t nh) {
  const uint32_t v = threadIdx.x < nblk ? bsum[threadIdx.x] : 0u;
  uint32_t total;
  const uint32_t ex = na_block_scan(v, &total);
  if (threadIdx.x < nblk) bsum[threadIdx.x] = ex;
  if (threadIdx.x == 0) start[nh] = total;
}

__global__ void __launch_bounds__(kNAThreads) na_down(const uint32_t *cnt, const uint32_t *bsum, uint32_t *start,
                                                      uint32_t nh) {
  const uint32_t base = blockIdx.x * kNATile + threadIdx.x * kNAItems;
  uint32_t v[kNAItems], s = 0;
#pragma unroll
  for (uint32_t k = 0; k < kNAItems; ++k) {
    v[k] = cnt[base + k];
    s += v[k];
  }
  uint32_t total;
  uint32_t run = bsum[blockIdx.x] + na_block_scan(s, &total);
#pragma unroll
  for (uint32_t k = 0; k < kNAItems; ++k) {
    if (base + k < nh) start[base + k] = run;
    run += v[k];
  }
}

__global__ void na_scatter(const uint32_t *key, uint32_t n, const uint32_t *start, uint32_t *cnt, uint32_t *slots) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = key[i];
  slots[start[k] + atomicSub(&cnt[k], 1u) - 1u] = i;
}

// ascending id inside each bucket; a bucket above GG_NOALLOC_MAX_OCCUPANCY keeps the
// scatter's order (the rank would cost its occupancy per member)
__global__ void na_rank(const uint32_t *key, uint32_t n, const uint32_t *start, const uint32_t *slots, uint32_t *perm) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t id = slots[s];
  const uint32_t k = key[id];
  const uint32_t b0 = start[k], b1 = start[k + 1];
  uint32_t r = s - b0;
  if (b1 - b0 <= GG_NOALLOC_MAX_OCCUPANCY) {
    r = 0;
    for (uint32_t t = b0; t < b1; ++t) r += slots[t] < id ? 1u : 0u;
  }
  perm[b0 + r] = id;
}

uint32_t *scratch_for_current_device(gg_status *st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    *st = GG_ERR_NO_DEVICE;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      *st = GG_ERR_CUDA;
      return nullptr;
    }
    g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
  }
  *st = GG_OK;
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" gg_status gg_bin_sort_noalloc(const float *pos_radius, uint32_t n, float cell_size, uint32_t n_h,
                                         uint32_t *keys, uint32_t *perm, uint32_t *cell_start, void *stream) {
  if (n > GG_NOALLOC_MAX_PARTICLES || n_h == 0 || n_h > GG_NOALLOC_MAX_BUCKETS) return GG_ERR_INVALID_ARG;
  if (!(cell_size > 0.f) || !cell_start || (n && (!pos_radius || !keys || !perm))) return GG_ERR_INVALID_ARG;
  gg_status st;
  uint32_t *scratch = scratch_for_current_device(&st);
  if (!scratch) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float inv_cell = (float)(1.0 / (double)cell_size);
  const uint32_t nblk = (n_h + kNATile - 1) / kNATile;
  const uint32_t hist_words = nblk * kNATile;  // whole tiles: the scan reads them all
  uint32_t *cnt = scratch, *bsum = scratch + kNABuckets, *slots = bsum + kNABlocks;
  const uint32_t gp = (n + 255) / 256;
  na_clear<<<(hist_words + 1023) / 1024, 1024, 0, s>>>(cnt, hist_words);
  if (n) na_key<<<gp, 256, 0, s>>>(reinterpret_cast<const float4 *>(pos_radius), n, inv_cell, n_h, keys, cnt);
  na_reduce<<<nblk, kNAThreads, 0, s>>>(cnt, bsum);
  na_top<<<1, 1024, 0, s>>>(bsum, nblk, cell_start, n_h);
  na_down<<<nblk, kNAThreads, 0, s>>>(cnt, bsum, cell_start, n_h);
  if (n) {
    na_scatter<<<gp, 256, 0, s>>>(keys, n, cell_start, cnt, slots);
    na_rank<<<gp, 256, 0, s>>>(keys, n, cell_start, slots, perm);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GG_OK : GG_ERR_CUDA;
}
