// gg_kernels.cu -- sm_103a kernels of the granular contact step.
//
// One time step = the launches below, in this order (captured once into a CUDA
// graph and replayed):
//   k_key            bucket of every particle (Eq. 6), body prep; then either
//                    a push onto the bucket's linked list (Alg. 2), or
//                    the bucket histogram for the counting sort:
//   k_scan_*         exclusive scan of the histogram (tile sums, their scan, down-sweep)
//                    -> bucket start table and (start, end) ranges
//   k_scatter        counting-sort scatter (returns the histogram to zero)
//   k_reorder        stable order inside each bucket (ascending id), positions in slot order
//   k_contacts       27-cell bucket walk, sphere test, SDF tests (Sec. II-B, II-C), or
//   k_pairs_half     the forward half of the walk, hits mirrored into scratch, and
//   k_pairs_finish   the partner lists sorted and deduplicated, SDF tests
//   k_free_prep      (free bodies) sorted contact lists, box-corner contacts
//   k_pja  x I       projected-Jacobi sweeps (Alg. 1), one launch per iteration,
//   k_free_update    each followed (free bodies) by the bodies' twist update
//   k_integrate_wrench  symplectic Euler (Eq. 4-5) in place, per-body impulse sums
//                    over fixed chunks of particles (deterministic), the lists emptied
//   k_wrench_bodies  per-body sums over chunks into the wrench readback ring, body
//                    poses, step counter
// Contacts, sweeps and integration run over particles in the caller's order (their
// storage order); the bucket table is only walked, so spatially ordered inputs keep
// neighbours' data in nearby cache lines.
// Detection and impulse computation are separate launches, the split the paper
// finds fastest (Sec. II-D).
#include <algorithm>

#include "gg_device.cuh"
#include "gg_internal.h"

namespace gg {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Fixed-order sum of 6 floats over the block, result valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum6(float v[6]) {
  __shared__ float sm[NT / 32][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) sm[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float s = sm[0][k];
      for (int w = 1; w < NT / 32; ++w) s += sm[w][k];
      v[k] = s;
    }
  }
}

__device__ __forceinline__ void flag(DevCtrl *c, uint32_t f) { atomicOr(&c->status, f); }

// v + dt g (the velocity before contact impulses), with 1/m in w
__device__ __forceinline__ float4 base_velocity(const StepArgs &a, float4 v) {
  return make_float4(v.x + a.dt * a.g[0], v.y + a.dt * a.g[1], v.z + a.dt * a.g[2], v.w);
}

// ---------------------------------------------------------------------------
// 1. bucket keys + histogram; body pose/twist for this step
// ---------------------------------------------------------------------------

__device__ void prep_body(const StepArgs &a, uint32_t gb) {
  DevBody &B = a.bodies[gb];
  if (!B.active) return;
  quat_to_R(B.q, B.R);
  const uint32_t step = a.ctrl->step;
  if (B.is_free) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      B.v[k] = B.own_v[k] + a.dt * a.g[k];
      B.w[k] = B.own_w[k];
    }
    return;
  }
  const float *tw = nullptr;
  if (B.traj && step >= B.traj_start && step - B.traj_start < B.traj_len) tw = B.traj + 6u * (step - B.traj_start);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    B.v[k] = tw ? tw[k] : B.own_v[k];
    B.w[k] = tw ? tw[3 + k] : B.own_w[k];
  }
}

// The body frames and velocities of the step in the device step counter (prep_body)
// alone: the reverse pass runs it on the state restored for a step, before its adjoint.
__global__ void k_prep_bodies(StepArgs a) {
  const uint32_t gb = blockIdx.x * blockDim.x + threadIdx.x;
  if (gb < a.n_envs * a.maxb) prep_body(a, gb);
}

// Histogram of the stored keys (the sort-order readbacks of a step that binned by lists).
__global__ void k_hist_keys(StepArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) atomicAdd(&a.cnt[a.key_id[i]], 1u);
}

// Linked-list binning: every bucket's list emptied (after a taped step, which ends
// with its sweeps; a full step does this in k_integrate_wrench).
__global__ void k_list_clear(StepArgs a) {
  pdl_enter();
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < a.nh_total; b += gridDim.x * blockDim.x)
    a.head[b] = kListEnd;
}

__global__ void k_key(StepArgs a) {
  pdl_enter();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    float4 p = a.pos_id[i];
    const DevEnv &E = a.envs[a.env_of[i]];
    int32_t k0 = cell_of(p.x, E.inv_cell), k1 = cell_of(p.y, E.inv_cell), k2 = cell_of(p.z, E.inv_cell);
    uint32_t key = E.hbase + hash_cell_fm(k0, k1, k2, E);
    // checked build: a key outside the environment's range is replaced by an in-range
    // one before it is stored, so the scatter, reorder and walks that index with the
    // stored key stay in bounds while the failed check is latched
    if (!GG_GUARD(a.ctrl, key - E.hbase < E.nh && key < a.nh_total)) key = E.hbase < a.nh_total ? E.hbase : 0u;
    a.key_id[i] = key;
    if (a.lists)
      a.next[i] = atomicExch(&a.head[key], i);  // lock-free push onto the bucket's list (Alg. 2)
    else
      atomicAdd(&a.cnt[key], 1u);
  }
  if (i < a.n_envs * a.maxb) {
    prep_body(a, i);
    a.ncb[i] = 0;
  }
  if (i < a.F) a.fcount[i] = 0;
  if (i == 0) {
    a.ctrl->bar_count = 0;
    a.ctrl->bar_abort = 0;
    a.ctrl->n_pp = 0;
    a.ctrl->n_body = 0;
    a.ctrl->max_pp = 0;
    a.ctrl->max_body = 0;
    a.ctrl->max_psi_bits = 0;
    a.ctrl->n_active = 0;
  }
}

// ---------------------------------------------------------------------------
// 2. exclusive scan of the bucket histogram (reduce, scan block sums, down-sweep)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(StepArgs a) {
  pdl_enter();
  const uint4 *c4 = reinterpret_cast<const uint4 *>(a.cnt + (size_t)blockIdx.x * kScanTile +
                                                     (size_t)threadIdx.x * kScanItems);
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems / 4; ++k) {
    uint4 v = c4[k];
    s += v.x + v.y + v.z + v.w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ uint32_t ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    a.bsum[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of the block sums in place; start[nh_pad] = total.
__global__ void __launch_bounds__(1024) k_scan_top(StepArgs a, uint32_t nblk) {
  pdl_enter();
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nblk; base += 1024) {
    uint32_t idx = base + threadIdx.x;
    uint32_t v = idx < nblk ? a.bsum[idx] : 0u;
    // block scan of 1024 values
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint32_t s = ws[lane];
      uint32_t si = warp_incl_scan(s);
      ws[lane] = si - s;
    }
    __syncthreads();
    uint32_t excl = carry + ws[wid] + inc - v;
    if (idx < nblk) a.bsum[idx] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.start[a.nh_pad] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(StepArgs a) {
  pdl_enter();
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  const uint4 *c4 = reinterpret_cast<const uint4 *>(a.cnt + base);
  uint32_t v[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems / 4; ++k) {
    uint4 q = c4[k];
    v[4 * k] = q.x;
    v[4 * k + 1] = q.y;
    v[4 * k + 2] = q.z;
    v[4 * k + 3] = q.w;
  }
  uint32_t tsum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) tsum += v[k];
  __shared__ uint32_t ws[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = warp_incl_scan(tsum);
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < kScanThreads / 32 ? ws[lane] : 0u;
    uint32_t si = warp_incl_scan(s);
    if (lane < kScanThreads / 32) ws[lane] = si - s;
  }
  __syncthreads();
  uint32_t run = a.bsum[blockIdx.x] + ws[wid] + inc - tsum;
  uint4 *s4 = reinterpret_cast<uint4 *>(a.start + base);
  uint4 *r4 = reinterpret_cast<uint4 *>(a.range + base);  // two (start, end) pairs per uint4
#pragma unroll
  for (int k = 0; k < kScanItems / 4; ++k) {
    uint32_t b[5];
    b[0] = run;
#pragma unroll
    for (int m = 0; m < 4; ++m) b[m + 1] = b[m] + v[4 * k + m];
    run = b[4];
    s4[k] = make_uint4(b[0], b[1], b[2], b[3]);
    r4[2 * k] = make_uint4(b[0], b[1], b[1], b[2]);
    r4[2 * k + 1] = make_uint4(b[2], b[3], b[3], b[4]);
  }
}

// ---------------------------------------------------------------------------
// 3. scatter into buckets; 4. stable order inside buckets + gather
// ---------------------------------------------------------------------------

__global__ void k_scatter(StepArgs a) {
  pdl_enter();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint32_t key = a.key_id[i];
  const uint32_t r = atomicSub(&a.cnt[key], 1u) - 1u;  // leaves the histogram at zero
  a.sid_tmp[a.start[key] + r] = i;
}

__global__ void k_reorder(StepArgs a) {
  pdl_enter();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const uint32_t id = a.sid_tmp[s];
  const uint32_t key = a.key_id[id];
  const uint2 rg = a.range[key];
  const uint32_t b0 = rg.x, b1 = rg.y;
  uint32_t rank = 0;
  if (b1 - b0 > kMaxBucket) {  // too crowded to rank: keep the scatter's order, report
    flag(a.ctrl, kFlagBucketBound);
    rank = s - b0;
  } else {
    for (uint32_t t = b0; t < b1; ++t) rank += (a.sid_tmp[t] < id) ? 1u : 0u;
  }
  a.sid[b0 + rank] = id;
  a.pos_s[b0 + rank] = a.pos_id[id];
}

// ---------------------------------------------------------------------------
// 5. contacts: particle-particle (27 buckets) and particle-body (SDF)
// ---------------------------------------------------------------------------

// Inserts partner jid into the thread's list (shared memory, stride S) kept in
// ascending id order; a bucket reached twice yields the same id, which is skipped.
// v[q] for a q known only at run time, without putting v in local memory.  Measured on
// the column collapse (contact stage, us per step): the half-stencil pass 51.1 with
// indexed arrays, 47.4 with this, 46.5 with this and a 56-register cap; k_contacts
// keeps its indexed arrays (55.0, against 55.2 with this and 58.0 with the cap).
template <typename T>
__device__ __forceinline__ T pick3(const T (&v)[3], int q) {
  return q == 0 ? v[0] : (q == 1 ? v[1] : v[2]);
}

__device__ __forceinline__ void insert_partner(uint32_t *fid, uint32_t S, uint32_t K, uint32_t jid, uint32_t &npp,
                                               bool &ovf) {
  uint32_t p = 0;
  while (p < npp && fid[p * S] < jid) ++p;
  if (p < npp && fid[p * S] == jid) return;
  if (npp == K) {
    ovf = true;
    if (p == K) return;
  } else {
    ++npp;
  }
  for (uint32_t q2 = npp - 1; q2 > p; --q2) fid[q2 * S] = fid[(q2 - 1) * S];
  fid[p * S] = jid;
}

// A bucket's (start, end), cut to kMaxBucket entries (the cut is reported).
__device__ __forceinline__ uint2 bounded_range(const StepArgs &a, uint2 rg) {
  if (rg.y - rg.x > kMaxBucket) {
    flag(a.ctrl, kFlagBucketBound);
    rg.y = rg.x + kMaxBucket;
  }
  return rg;
}

constexpr int kWalkGroup = 3;       // buckets of a row (dx = -1, 0, 1), walked together
constexpr int kContactsBlock = 128;  // threads per block of k_contacts

// Contact normal (from j towards i) and penetration psi = r_i + r_j - |x_i - x_j| of a
// pair that passed the hit test; coincident centres get +-z by id order.  Every
// product is rounded on its own (no contraction), so the result is the same wherever
// the helper is inlined.
__device__ __forceinline__ float4 pair_geometry(const float4 &pi, const float4 &pj, uint32_t i, uint32_t j) {
  float d2;
  float3 d;
  sphere_hit(pi, pj, &d2, &d);
  const float dist = __fsqrt_rn(d2);
  float3 nn;
  if (dist > 0.f) {
    const float id = __frcp_rn(dist);
    nn = make_float3(__fmul_rn(d.x, id), __fmul_rn(d.y, id), __fmul_rn(d.z, id));
  } else {
    nn = make_float3(0.f, 0.f, i > j ? 1.f : -1.f);
  }
  return make_float4(nn.x, nn.y, nn.z, __fsub_rn(__fadd_rn(pi.w, pj.w), dist));
}

// Particle-body contact test (Sec. II-C, Eq. 7): culled by the body's bounding sphere
// (with a margin far above rounding), then the SDF at the centre in the body frame;
// true when f <= r_i (y, f and the SDF branch returned for body_geometry).
__device__ __forceinline__ bool body_touch(const DevBody &B, const float3 &xi, float ri, float3 *y, float *f,
                                           int *br) {
  if (B.bound_r > 0.f) {
    const float dx = xi.x - B.p[0], dy = xi.y - B.p[1], dz = xi.z - B.p[2];
    const float rb = B.bound_r + ri;
    if (dx * dx + dy * dy + dz * dz > 1.0001f * rb * rb) return false;
  }
  *y = world_to_body(B, xi);
  *f = body_sdf(B, *y, br);
  return *f <= ri;
}

// World normal and psi = r_i - f of a touching body, and the contact point x_i - f n.
__device__ __forceinline__ void body_geometry(const DevBody &B, const float3 &xi, float ri, const float3 &y, float f,
                                              int br, float4 *bn, float4 *bxc) {
  const float3 nn = rot_apply(B.R, body_grad(B, y, br));
  *bn = make_float4(nn.x, nn.y, nn.z, ri - f);
  *bxc = make_float4(xi.x - f * nn.x, xi.y - f * nn.y, xi.z - f * nn.z, 0.f);
}

// Contact records of particle i from its partner list (ascending ids, shared memory,
// stride S), then its body contacts in ascending body index; counts and U^0.
__device__ __forceinline__ void contact_records(const StepArgs &a, uint32_t i, float4 pi, float4 vi, uint32_t e,
                                                const DevEnv &E, const uint32_t *fid, uint32_t S, uint32_t K,
                                                uint32_t npp, bool ovf, uint32_t &nbc, float &psi_max) {
    const size_t n = a.n;
    // the partners' positions are gathered four at a time, all four loads in flight
    // before any record of the group is computed and stored
    constexpr uint32_t kGroup = 4;
    for (uint32_t c0 = 0; c0 < npp; c0 += kGroup) {
      uint32_t jg[kGroup];
      float4 pg[kGroup];
#pragma unroll
      for (uint32_t q = 0; q < kGroup; ++q) {
        jg[q] = c0 + q < npp ? fid[(c0 + q) * S] : i;
        pg[q] = a.pos_id[jg[q]];
      }
#pragma unroll
      for (uint32_t q = 0; q < kGroup; ++q) {
        const uint32_t c = c0 + q;
        if (c >= npp) break;
        const uint32_t j = jg[q];
        const float4 g = pair_geometry(pi, pg[q], i, j);
        psi_max = fmaxf(psi_max, g.w);
        const size_t o = (size_t)c * n + i;
        a.cj[o] = j;
        a.cn[o] = g;
        a.clam[o] = 0.f;
        a.clam[o + (size_t)K * n] = 0.f;
        a.clam[o + 2 * (size_t)K * n] = 0.f;
      }
    }
    // particle-body contacts, bodies in ascending index
    const float3 xi = make_float3(pi.x, pi.y, pi.z);
    for (uint32_t b = 0; b < E.nbodies; ++b) {
      const uint32_t gb = e * a.maxb + b;
      const DevBody &B = a.bodies[gb];
      float3 y;
      float f;
      int br;
      if (!body_touch(B, xi, pi.w, &y, &f, &br)) continue;
      if (nbc == a.Kb) {
        flag(a.ctrl, kFlagBodyOverflow);
        continue;
      }
      float4 bn, bxc;
      body_geometry(B, xi, pi.w, y, f, br, &bn, &bxc);
      psi_max = fmaxf(psi_max, bn.w);
      const size_t o = (size_t)nbc * n + i;
      if (B.is_free) {
        atomicAdd(&a.ncb[gb], 1u);
        const uint32_t pos = atomicAdd(&a.fcount[B.fid], 1u);
        if (pos < a.Lcap)
          a.flist[(size_t)B.fid * a.Lcap + pos] = i * a.Kb + nbc;
        else
          flag(a.ctrl, kFlagBodyOverflow);
      }
      a.bj[o] = gb;
      a.bn[o] = bn;
      a.bxc[o] = bxc;
      a.blam[o] = 0.f;
      a.blam[o + (size_t)a.Kb * n] = 0.f;
      a.blam[o + 2 * (size_t)a.Kb * n] = 0.f;
      ++nbc;
    }
    if (ovf) flag(a.ctrl, kFlagPPOverflow);
    a.ccount[i] = npp | (nbc << 8);
    const float4 sb = base_velocity(a, vi);
    a.U[0][i] = make_float4(sb.x, sb.y, sb.z, (float)(a.lit ? 1u : npp + nbc) * sb.w);
  }

// Per-step statistics (integer atomics: order-independent); every thread of the warp calls.
__device__ __forceinline__ void contact_stats(const StepArgs &a, uint32_t npp, uint32_t nbc, float psi_max) {
  uint32_t s_pp = npp, s_b = nbc, m_pp = npp, m_b = nbc;
  const uint32_t act = __popc(__ballot_sync(0xffffffffu, npp + nbc > 0));
  float m_psi = psi_max;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s_pp += __shfl_xor_sync(0xffffffffu, s_pp, o);
    s_b += __shfl_xor_sync(0xffffffffu, s_b, o);
    m_pp = max(m_pp, __shfl_xor_sync(0xffffffffu, m_pp, o));
    m_b = max(m_b, __shfl_xor_sync(0xffffffffu, m_b, o));
    m_psi = fmaxf(m_psi, __shfl_xor_sync(0xffffffffu, m_psi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (s_pp) atomicAdd(&a.ctrl->n_pp, s_pp);
    if (s_b) atomicAdd(&a.ctrl->n_body, s_b);
    if (act) atomicAdd(&a.ctrl->n_active, act);
    if (m_pp) atomicMax(&a.ctrl->max_pp, m_pp);
    if (m_b) atomicMax(&a.ctrl->max_body, m_b);
    if (m_psi > 0.f) atomicMax(&a.ctrl->max_psi_bits, __float_as_uint(m_psi));
  }
}

// The partner list of a thread, kept sorted by id while the buckets are walked, lives
// in shared memory, slot p of thread t at [p * blockDim.x + t] (conflict-free): an
// array indexed at run time in registers would go to local memory, which at full
// occupancy does not fit in L1.  Dynamic shared memory: K * blockDim.x words.
// The partner list of particle i (Sec. II-B 27-cell query): ascending ids in the
// thread's shared-memory column fid (stride S), the K smallest kept (ovf set if more).
template <bool LISTS>
__device__ __forceinline__ void walk_partners(const StepArgs &a, uint32_t i, const float4 &pi, const DevEnv &E,
                                              uint32_t *fid, uint32_t S, uint32_t &npp, bool &ovf) {
  {
    const int32_t k0 = cell_of(pi.x, E.inv_cell), k1 = cell_of(pi.y, E.inv_cell), k2 = cell_of(pi.z, E.inv_cell);
    const uint32_t K = a.K;
    // Eq. 6 terms of the three cells along each axis, combined 27 ways below
    uint32_t hx[3], hy[3], hz[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      hx[q] = ((uint32_t)(k0 + q - 1) - kHashQ) * kHashP1;
      hy[q] = ((uint32_t)(k1 + q - 1) - kHashQ) * kHashP2;
      hz[q] = ((uint32_t)(k2 + q - 1) - kHashQ) * kHashP3;
    }
    // Neighbour cells that cannot hold a partner are not walked.  In cell units
    // (u = x inv_c, cell k spans [k - 1/2, k + 1/2)) the gap from u_i to the cell
    // at offset d along an axis is 0 for d = 0 and 1/2 -+ f for d = -+1, f = u_i - k_i.
    // A partner j has |x_i - x_j| <= r_i + r_j <= r_i + c/2 (c >= 2 r_max is checked
    // at creation), so a cell whose gap vector is longer than r_i inv_c + 1/2 plus a
    // margin (float32 rounding of u and of the cell assignment: 2^-10 cells plus
    // four ulps of |u|) is skipped.  A bucket shared with a nearer cell is still
    // walked for that cell, so the contact set is exactly the 27-cell one.
    float g2x[3], g2y[3], g2z[3];
    {
      const float ux = __fmul_rn(pi.x, E.inv_cell), uy = __fmul_rn(pi.y, E.inv_cell), uz = __fmul_rn(pi.z, E.inv_cell);
      const float fx = __fsub_rn(ux, (float)k0), fy = __fsub_rn(uy, (float)k1), fz = __fsub_rn(uz, (float)k2);
      const float lo_x = fmaxf(0.5f + fx, 0.f), hi_x = fmaxf(0.5f - fx, 0.f);
      const float lo_y = fmaxf(0.5f + fy, 0.f), hi_y = fmaxf(0.5f - fy, 0.f);
      const float lo_z = fmaxf(0.5f + fz, 0.f), hi_z = fmaxf(0.5f - fz, 0.f);
      g2x[0] = lo_x * lo_x; g2x[1] = 0.f; g2x[2] = hi_x * hi_x;
      g2y[0] = lo_y * lo_y; g2y[1] = 0.f; g2y[2] = hi_y * hi_y;
      g2z[0] = lo_z * lo_z; g2z[1] = 0.f; g2z[2] = hi_z * hi_z;
    }
    float reach;
    {
      const float um = fabsf(__fmul_rn(pi.x, E.inv_cell)) + fabsf(__fmul_rn(pi.y, E.inv_cell)) +
                       fabsf(__fmul_rn(pi.z, E.inv_cell));
      const float rr = pi.w * E.inv_cell + 0.5f + 0.0009765625f + um * 4.76837158203125e-7f;  // 2^-10, 2^-21
      reach = rr * rr;
    }
    if constexpr (!LISTS) {
    // The 27 buckets are walked as nine rows of three (dx = -1, 0, 1 at fixed dy, dz).
    // A row's three ranges are loaded while the previous row is walked; within a row
    // the walk takes one candidate from every non-empty bucket per round, so the
    // position loads of a round, and the id loads of its hits, are independent.
    uint32_t n0[kWalkGroup], n1[kWalkGroup];
#pragma unroll
    for (int q = 0; q < kWalkGroup; ++q) {
      n0[q] = n1[q] = 0u;
      if (g2x[q] + g2y[0] + g2z[0] <= reach) {
        const uint2 rg = bounded_range(a, a.range[E.hbase + mod_nh(hx[q] ^ hy[0] ^ hz[0], E)]);
        n0[q] = rg.x;
        n1[q] = rg.y;
      }
    }
#pragma unroll 1
    for (int row = 0; row < 9; ++row) {
      uint32_t r0[kWalkGroup], r1[kWalkGroup];
#pragma unroll
      for (int q = 0; q < kWalkGroup; ++q) {
        r0[q] = n0[q];
        r1[q] = n1[q];
      }
      if (row < 8) {
        const int ny = (row + 1) % 3, nz = (row + 1) / 3;
        // selects keep the per-axis terms in registers (run-time indexing would not)
        const uint32_t hyz = hy[ny] ^ hz[nz];
        const float g2yz = g2y[ny] + g2z[nz];
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q) {
          n0[q] = n1[q] = 0u;
          if (g2x[q] + g2yz <= reach) {
            const uint2 rg = bounded_range(a, a.range[E.hbase + mod_nh(hx[q] ^ hyz, E)]);
            n0[q] = rg.x;
            n1[q] = rg.y;
          }
        }
      }
      for (;;) {
        float4 pc[kWalkGroup];
        uint32_t live = 0;
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q)
          if (r0[q] < r1[q]) {
            live |= 1u << q;
            pc[q] = a.pos_s[r0[q]];
          }
        if (!live) break;
        uint32_t hit = 0;
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q) {
          float d2;
          float3 d;
          if (((live >> q) & 1u) && sphere_hit(pi, pc[q], &d2, &d)) hit |= 1u << q;
        }
        uint32_t jc[kWalkGroup];
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q)
          if ((hit >> q) & 1u) jc[q] = a.sid[r0[q]];
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q) {
          r0[q] += (live >> q) & 1u;
          if (!((hit >> q) & 1u)) continue;
          const uint32_t jid = jc[q];
          if (jid != i) insert_partner(fid, S, K, jid, npp, ovf);
        }
      }
    }
    } else {
    // Linked lists (Alg. 2): the three buckets of a row are walked together, one link
    // of each per round (each link is a load that depends on the previous one).
#pragma unroll 1
    for (int row = 0; row < 9; ++row) {
      const uint32_t hyz = hy[row % 3] ^ hz[row / 3];
      const float g2yz = g2y[row % 3] + g2z[row / 3];
      uint32_t jn[kWalkGroup];
#pragma unroll
      for (int q = 0; q < kWalkGroup; ++q)
        jn[q] = (g2x[q] + g2yz <= reach) ? a.head[E.hbase + mod_nh(hx[q] ^ hyz, E)] : kListEnd;
      // an intact list has at most n links: past that the lists were not emptied
      // before this step's pushes (a cycle), so the walk stops and the step reports it
      for (uint32_t round = 0;; ++round) {
        float4 pc[kWalkGroup];
        uint32_t nx[kWalkGroup];
        bool any = false;
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q)
          if (jn[q] != kListEnd && GG_GUARD(a.ctrl, jn[q] < a.n)) {
            any = true;
            pc[q] = a.pos_id[jn[q]];
            nx[q] = a.next[jn[q]];
          } else {
            jn[q] = kListEnd;
          }
        if (!any) break;
        if (round >= a.n) {
          flag(a.ctrl, kFlagListBound);
          break;
        }
        if (round >= kMaxBucket) {
          flag(a.ctrl, kFlagBucketBound);
          break;
        }
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q) {
          if (jn[q] == kListEnd) continue;
          float d2;
          float3 d;
          if (jn[q] != i && sphere_hit(pi, pc[q], &d2, &d)) insert_partner(fid, S, K, jn[q], npp, ovf);
          jn[q] = nx[q];
        }
      }
    }
    }
  }
}

// Detection of particle i (Sec. II-B 27-cell query, Sec. II-C SDF tests): its partner
// list, then its contact records.
template <bool LISTS>
__device__ __forceinline__ void detect_particle(const StepArgs &a, uint32_t i, uint32_t *fid, uint32_t S,
                                                uint32_t &npp, uint32_t &nbc, float &psi_max) {
  const float4 pi = a.pos_id[i];
  const uint32_t e = a.env_of[i];
  const DevEnv E = a.envs[e];
  bool ovf = false;
  walk_partners<LISTS>(a, i, pi, E, fid, S, npp, ovf);
  contact_records(a, i, pi, a.vel_id[i], e, E, fid, S, a.K, npp, ovf, nbc, psi_max);
}

template <bool LISTS>
__global__ void __launch_bounds__(kContactsBlock, 8) k_contacts(StepArgs a) {
  pdl_enter();
  extern __shared__ uint32_t s_fid[];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t npp = 0, nbc = 0;
  float psi_max = 0.f;
  if (i < a.n) detect_particle<LISTS>(a, i, s_fid + threadIdx.x, blockDim.x, npp, nbc, psi_max);
  contact_stats(a, npp, nbc, psi_max);
}

// Half-stencil pair search, two passes (the autotuner's alternative to k_contacts).
// Pass 1 walks the particle's own cell and the 13 neighbour cells of the forward half
// (offset (dx, dy, dz) > 0 in (dz, dy, dx) order; in its own cell only partners with a
// larger id).  Scratch rows 0..K-1 of particle i hold the partners i found (written by
// i alone), rows K..2K-1 the particles that found i (appended with one atomic per pair
// on the low half of pcnt[i]); i adds its own count to the high half at the end.  The
// hit test is symmetric in FP32, so each pair is found once, or twice when two of the
// walked cells share a bucket.  Pass 2 sorts and deduplicates the entries and writes
// the same records as k_contacts.
// The partner half of a hit needs the slot an atomic returns.  The first kDeferPairs
// hits of a thread keep their partner in shared memory (slot q of thread t at
// [q][t]) and take their atomics together after the walk (mirror_deferred), so the
// walk does not wait for an atomic at every hit; later hits take theirs at once.  The
// partner rows are sorted by pass 2, so the order in which the atomics land changes
// nothing.
constexpr uint32_t kDeferPairs = 4;

__device__ __forceinline__ void mirror_pair(const StepArgs &a, uint32_t i, uint32_t j) {
  const uint32_t aj = atomicAdd(&a.pcnt[j], 1u) & 0xffffu;
  if (aj < a.K) a.pscr[(size_t)(a.K + aj) * a.n + j] = i;
}

__device__ __forceinline__ void record_pair(const StepArgs &a, uint32_t i, uint32_t j, uint32_t &nf, uint32_t *jd) {
  if (nf < a.K) a.pscr[(size_t)nf * a.n + i] = j;
  if (nf < kDeferPairs)
    jd[nf * kContactsBlock] = j;
  else
    mirror_pair(a, i, j);
  ++nf;
}

// The deferred hits' atomics, all issued before any of their slots is used.
__device__ __forceinline__ void mirror_deferred(const StepArgs &a, uint32_t i, uint32_t nf, const uint32_t *jd) {
  uint32_t j[kDeferPairs], aj[kDeferPairs];
#pragma unroll
  for (uint32_t q = 0; q < kDeferPairs; ++q) j[q] = q < nf ? jd[q * kContactsBlock] : 0u;
#pragma unroll
  for (uint32_t q = 0; q < kDeferPairs; ++q) aj[q] = q < nf ? atomicAdd(&a.pcnt[j[q]], 1u) & 0xffffu : a.K;
#pragma unroll
  for (uint32_t q = 0; q < kDeferPairs; ++q)
    if (aj[q] < a.K) a.pscr[(size_t)(a.K + aj[q]) * a.n + j[q]] = i;
}

template <bool LISTS>
__global__ void __launch_bounds__(kContactsBlock, 9) k_pairs_half(StepArgs a) {
  pdl_enter();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const float4 pi = a.pos_id[i];
  const uint32_t e = a.env_of[i];
  const DevEnv E = a.envs[e];
  const int32_t k0 = cell_of(pi.x, E.inv_cell), k1 = cell_of(pi.y, E.inv_cell), k2 = cell_of(pi.z, E.inv_cell);
  uint32_t nf = 0;  // partners found by i
  __shared__ uint32_t s_jd[kDeferPairs * kContactsBlock];  // the first kDeferPairs of them
  uint32_t *jd = s_jd + threadIdx.x;
    // Eq. 6 terms of the three cells along each axis, combined 27 ways below
    uint32_t hx[3], hy[3], hz[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      hx[q] = ((uint32_t)(k0 + q - 1) - kHashQ) * kHashP1;
      hy[q] = ((uint32_t)(k1 + q - 1) - kHashQ) * kHashP2;
      hz[q] = ((uint32_t)(k2 + q - 1) - kHashQ) * kHashP3;
    }
    // Neighbour cells that cannot hold a partner are not walked.  In cell units
    // (u = x inv_c, cell k spans [k - 1/2, k + 1/2)) the gap from u_i to the cell
    // at offset d along an axis is 0 for d = 0 and 1/2 -+ f for d = -+1, f = u_i - k_i.
    // A partner j has |x_i - x_j| <= r_i + r_j <= r_i + c/2 (c >= 2 r_max is checked
    // at creation), so a cell whose gap vector is longer than r_i inv_c + 1/2 plus a
    // margin (float32 rounding of u and of the cell assignment: 2^-10 cells plus
    // four ulps of |u|) is skipped.  A bucket shared with a nearer cell is still
    // walked for that cell, so the contact set is exactly the 27-cell one.
    float g2x[3], g2y[3], g2z[3];
    {
      const float ux = __fmul_rn(pi.x, E.inv_cell), uy = __fmul_rn(pi.y, E.inv_cell), uz = __fmul_rn(pi.z, E.inv_cell);
      const float fx = __fsub_rn(ux, (float)k0), fy = __fsub_rn(uy, (float)k1), fz = __fsub_rn(uz, (float)k2);
      const float lo_x = fmaxf(0.5f + fx, 0.f), hi_x = fmaxf(0.5f - fx, 0.f);
      const float lo_y = fmaxf(0.5f + fy, 0.f), hi_y = fmaxf(0.5f - fy, 0.f);
      const float lo_z = fmaxf(0.5f + fz, 0.f), hi_z = fmaxf(0.5f - fz, 0.f);
      g2x[0] = lo_x * lo_x; g2x[1] = 0.f; g2x[2] = hi_x * hi_x;
      g2y[0] = lo_y * lo_y; g2y[1] = 0.f; g2y[2] = hi_y * hi_y;
      g2z[0] = lo_z * lo_z; g2z[1] = 0.f; g2z[2] = hi_z * hi_z;
    }
    float reach;
    {
      const float um = fabsf(__fmul_rn(pi.x, E.inv_cell)) + fabsf(__fmul_rn(pi.y, E.inv_cell)) +
                       fabsf(__fmul_rn(pi.z, E.inv_cell));
      const float rr = pi.w * E.inv_cell + 0.5f + 0.0009765625f + um * 4.76837158203125e-7f;  // 2^-10, 2^-21
      reach = rr * rr;
    }
  // rows (qy, qz) of the forward half, index 1 = offset 0: (0..2, 2) whole, (2, 1) whole,
  // (1, 1) with qx = 1 (the own cell) and 2
#pragma unroll 1
  for (int row = 0; row < 5; ++row) {
    const int qz = row < 3 ? 2 : 1;
    const int qy = row < 3 ? row : (row == 3 ? 2 : 1);
    const uint32_t mask = row == 4 ? 6u : 7u;
    const uint32_t hyz = pick3(hy, qy) ^ pick3(hz, qz);
    const float g2yz = pick3(g2y, qy) + pick3(g2z, qz);
    if constexpr (LISTS) {
      uint32_t jn[kWalkGroup];
#pragma unroll
      for (int q = 0; q < kWalkGroup; ++q)
        jn[q] = (((mask >> q) & 1u) && g2x[q] + g2yz <= reach) ? a.head[E.hbase + mod_nh(hx[q] ^ hyz, E)]
                                                                : kListEnd;
      // an intact list has at most n links: past that the lists were not emptied
      // before this step's pushes (a cycle), so the walk stops and the step reports it
      for (uint32_t round = 0;; ++round) {
        float4 pc[kWalkGroup];
        uint32_t nx[kWalkGroup];
        bool any = false;
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q)
          if (jn[q] != kListEnd && GG_GUARD(a.ctrl, jn[q] < a.n)) {
            any = true;
            pc[q] = a.pos_id[jn[q]];
            nx[q] = a.next[jn[q]];
          } else {
            jn[q] = kListEnd;
          }
        if (!any) break;
        if (round >= a.n) {
          flag(a.ctrl, kFlagListBound);
          break;
        }
        if (round >= kMaxBucket) {
          flag(a.ctrl, kFlagBucketBound);
          break;
        }
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q) {
          if (jn[q] == kListEnd) continue;
          const uint32_t j = jn[q];
          float d2;
          float3 d;
          const bool own = row == 4 && q == 1;
          if ((own ? j > i : j != i) && sphere_hit(pi, pc[q], &d2, &d)) record_pair(a, i, j, nf, jd);
          jn[q] = nx[q];
        }
      }
    } else {
      uint32_t r0[kWalkGroup], r1[kWalkGroup];
#pragma unroll
      for (int q = 0; q < kWalkGroup; ++q) {
        r0[q] = r1[q] = 0u;
        if (((mask >> q) & 1u) && g2x[q] + g2yz <= reach) {
          const uint2 rg = bounded_range(a, a.range[E.hbase + mod_nh(hx[q] ^ hyz, E)]);
          r0[q] = rg.x;
          r1[q] = rg.y;
        }
      }
      for (;;) {
        float4 pc[kWalkGroup];
        uint32_t live = 0;
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q)
          if (r0[q] < r1[q]) {
            live |= 1u << q;
            pc[q] = a.pos_s[r0[q]];
          }
        if (!live) break;
        uint32_t hit = 0;
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q) {
          float d2;
          float3 d;
          if (((live >> q) & 1u) && sphere_hit(pi, pc[q], &d2, &d)) hit |= 1u << q;
        }
        uint32_t jc[kWalkGroup];
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q)
          if ((hit >> q) & 1u) jc[q] = a.sid[r0[q]];
#pragma unroll
        for (int q = 0; q < kWalkGroup; ++q) {
          r0[q] += (live >> q) & 1u;
          if (!((hit >> q) & 1u)) continue;
          const bool own = row == 4 && q == 1;
          if (own ? jc[q] > i : jc[q] != i) record_pair(a, i, jc[q], nf, jd);
        }
      }
    }
  }
  mirror_deferred(a, i, nf, jd);
  if (nf) atomicAdd(&a.pcnt[i], min(nf, a.K + 1u) << 16);
}

// Pass 2: the partner list of particle i from its scratch entries (sorted, duplicates
// dropped, the K smallest ids kept as in k_contacts), then the same records.
// Loads are issued in batches, each batch before any of its values is used: the counts
// with the particle's position, velocity and environment; then the first kFinishPre
// entries of both scratch halves together (only entries below the counts are read).
// The entries are inserted in the order they are stored (finder half, then partner
// half), so the lists do not depend on the batching.
constexpr uint32_t kFinishPre = 4;

__global__ void __launch_bounds__(kContactsBlock, 8) k_pairs_finish(StepArgs a) {
  pdl_enter();
  extern __shared__ uint32_t s_fid[];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t npp = 0, nbc = 0;
  float psi_max = 0.f;
  if (i < a.n) {
    const size_t n = a.n;
    const uint32_t K = a.K;
    const uint32_t cnt = a.pcnt[i];
    const float4 pi = a.pos_id[i];
    const float4 vi = a.vel_id[i];
    const uint32_t e = a.env_of[i];
    const uint32_t nfw = cnt >> 16, nbw = cnt & 0xffffu;
    bool ovf = nfw > K || nbw > K;  // entries were lost: the list may be incomplete
    const uint32_t mf = min(nfw, K), mb = min(nbw, K);
    uint32_t jf[kFinishPre], jb[kFinishPre];
#pragma unroll
    for (uint32_t p = 0; p < kFinishPre; ++p) {
      jf[p] = p < mf ? a.pscr[(size_t)p * n + i] : 0u;
      jb[p] = p < mb ? a.pscr[(size_t)(K + p) * n + i] : 0u;
    }
    const DevEnv E = a.envs[e];
    uint32_t *fid = s_fid + threadIdx.x;
    const uint32_t S = blockDim.x;
#pragma unroll
    for (uint32_t p = 0; p < kFinishPre; ++p)
      if (p < mf && GG_GUARD(a.ctrl, jf[p] < a.n && jf[p] != i)) insert_partner(fid, S, K, jf[p], npp, ovf);
    for (uint32_t p = kFinishPre; p < mf; ++p) {
      const uint32_t j = a.pscr[(size_t)p * n + i];
      if (GG_GUARD(a.ctrl, j < a.n && j != i)) insert_partner(fid, S, K, j, npp, ovf);
    }
#pragma unroll
    for (uint32_t p = 0; p < kFinishPre; ++p)
      if (p < mb && GG_GUARD(a.ctrl, jb[p] < a.n && jb[p] != i)) insert_partner(fid, S, K, jb[p], npp, ovf);
    for (uint32_t p = kFinishPre; p < mb; ++p) {
      const uint32_t j = a.pscr[(size_t)(K + p) * n + i];
      if (GG_GUARD(a.ctrl, j < a.n && j != i)) insert_partner(fid, S, K, j, npp, ovf);
    }
    a.pcnt[i] = 0;  // ready for the next step
    contact_records(a, i, pi, vi, e, E, fid, S, K, npp, ovf, nbc, psi_max);
  }
  contact_stats(a, npp, nbc, psi_max);
}

// ---------------------------------------------------------------------------
// 6. one projected-Jacobi sweep: U[s] -> U[s^1]
// ---------------------------------------------------------------------------

// One Jacobi update of particle i: U[s] -> U[s^1] (s: double-buffer index).
// TAPE: also keep the iterates in tape slot it + 1 (it = iteration number).
// LDCG: read the velocity estimates through L2 only (the fused kernel reads, within
// one launch, estimates that other SMs wrote in the previous iteration).
// PRE: load the records of slots 0 and 1 together with the counts (below).
template <bool TAPE, bool LDCG, bool PRE = false>
__device__ __forceinline__ void pja_particle(const StepArgs &a, uint32_t i, int s, const Tape &tp, int it) {
  const float4 *__restrict__ Uin = a.U[s];
  const uint32_t *__restrict__ cj = a.cj;
  const float4 *__restrict__ cn = a.cn;
  float *__restrict__ clam = a.clam;
  const size_t n = a.n;
  const uint32_t cc = a.ccount[i];
  const uint32_t npp = cc & 0xffu, nbc = (cc >> 8) & 0xffu;
  const float4 ui = LDCG ? __ldcg(Uin + i) : Uin[i];
  const float4 base = base_velocity(a, a.vel_id[i]);
  float sx = 0.f, sy = 0.f, sz = 0.f;
  const size_t KN = (size_t)a.K * n;
  const float mu = a.mu, ab = a.ab;
  const float pw = a.lit ? 0.f : 1.f;  // partner's share of the effective mass (exact 0 or 1)
  // one contact update (Alg. 1 with the accumulated clamp): new impulse stored (and taped)
  auto update = [&](size_t o, const float4 &nn, const float3 &la, const float4 &uj) {
    const float3 l = pja_project(la, make_float3(ui.x - uj.x, ui.y - uj.y, ui.z - uj.z), make_float3(nn.x, nn.y, nn.z),
                                 ab * nn.w, 1.0f / (ui.w + pw * uj.w), mu);
    clam[o] = l.x;
    clam[o + KN] = l.y;
    clam[o + 2 * KN] = l.z;
    if (TAPE) {
      float *h = tp.lamh + (size_t)(it + 1) * 3 * KN;
      h[o] = l.x;
      h[o + KN] = l.y;
      h[o + 2 * KN] = l.z;
    }
    return l;
  };
  auto gather = [&](uint32_t j) { return LDCG ? __ldcg(Uin + j) : Uin[j]; };
  // PRE: the records of slots 0 and 1 are loaded together with the counts (those rows
  // exist for every particle; a particle with fewer contacts does not use them), so for
  // most particles the partner gathers are the second dependent load, not the third.
  // That pays on settled beds streaming from DRAM (1M spheres: 35.1 -> 33.6 us per
  // sweep) and costs where most spheres have no contact (the collapsing column: their
  // unused records are 64 bytes of extra reads each, 3.2 -> 3.6 us), so the serpentine
  // launch shapes, which the autotuner picks for the former, use it.
  // (Loading only the partner ids of slots 0 and 1 early was measured too: slower on
  // every workload, 64 registers with spills.)
  const bool two = PRE && a.K > 1;
  uint32_t pj0 = 0u, pj1 = 0u;
  float4 pn0 = make_float4(0.f, 0.f, 0.f, 0.f), pn1 = pn0;
  float3 pl0 = make_float3(0.f, 0.f, 0.f), pl1 = pl0;
  if (PRE) {
    pj0 = cj[i];
    pn0 = cn[i];
    pl0 = make_float3(clam[i], clam[i + KN], clam[i + 2 * KN]);
    if (two) {
      pj1 = cj[n + i];
      pn1 = cn[n + i];
      pl1 = make_float3(clam[n + i], clam[n + i + KN], clam[n + i + 2 * KN]);
    }
  }
  // two contacts per round: both rounds' loads issue before either update is stored;
  // the impulses are still added in contact order
  uint32_t c = 0;
  if (two && npp >= 2) {
    uint32_t j0 = pj0, j1 = pj1;
    if (!GG_GUARD(a.ctrl, j0 < a.n && j1 < a.n)) j0 = j1 = i;  // debug build: never gather out of range
    const float4 u0 = gather(j0), u1 = gather(j1);
    const float3 l0 = update(i, pn0, pl0, u0);
    const float3 l1 = update(n + i, pn1, pl1, u1);
    sx += l0.x;
    sy += l0.y;
    sz += l0.z;
    sx += l1.x;
    sy += l1.y;
    sz += l1.z;
    c = 2;
  }
  for (; c + 1 < npp; c += 2) {
    const size_t o0 = (size_t)c * n + i, o1 = o0 + n;
    uint32_t j0 = cj[o0], j1 = cj[o1];
    if (!GG_GUARD(a.ctrl, j0 < a.n && j1 < a.n)) j0 = j1 = i;  // debug build: never gather out of range
    const float4 n0 = cn[o0], n1 = cn[o1];
    const float3 la0 = make_float3(clam[o0], clam[o0 + KN], clam[o0 + 2 * KN]);
    const float3 la1 = make_float3(clam[o1], clam[o1 + KN], clam[o1 + 2 * KN]);
    const float4 u0 = gather(j0), u1 = gather(j1);
    const float3 l0 = update(o0, n0, la0, u0);
    const float3 l1 = update(o1, n1, la1, u1);
    sx += l0.x;
    sy += l0.y;
    sz += l0.z;
    sx += l1.x;
    sy += l1.y;
    sz += l1.z;
  }
  if (c < npp) {
    const size_t o = (size_t)c * n + i;
    const bool pre = PRE && c == 0;
    uint32_t j = pre ? pj0 : cj[o];
    if (!GG_GUARD(a.ctrl, j < a.n)) j = i;
    const float4 nn = pre ? pn0 : cn[o];
    const float3 lam = pre ? pl0 : make_float3(clam[o], clam[o + KN], clam[o + 2 * KN]);
    const float3 l = update(o, nn, lam, gather(j));
    sx += l.x;
    sy += l.y;
    sz += l.z;
  }
  const size_t KbN = (size_t)a.Kb * n;
  for (uint32_t c = 0; c < nbc; ++c) {
    const size_t o = (size_t)c * n + i;
    const uint32_t gbo = a.bj[o];
    if (!GG_GUARD(a.ctrl, gbo < a.n_envs * a.maxb)) continue;
    const DevBody &B = a.bodies[gbo];
    const float4 nn = a.bn[o];
    const float4 xc = a.bxc[o];
    const float3 lam = make_float3(a.blam[o], a.blam[o + KbN], a.blam[o + 2 * KbN]);
    const float rx = xc.x - B.p[0], ry = xc.y - B.p[1], rz = xc.z - B.p[2];
    const float ubx = B.v[0] + (B.w[1] * rz - B.w[2] * ry);
    const float uby = B.v[1] + (B.w[2] * rx - B.w[0] * rz);
    const float ubz = B.v[2] + (B.w[0] * ry - B.w[1] * rx);
    float invb = 0.f;
    if (B.is_free) {  // n_b (1/M + (a x n) . I_w^-1 (a x n)), mass split over the body's contacts
      const float cx = ry * nn.z - rz * nn.y, cy = rz * nn.x - rx * nn.z, cz = rx * nn.y - ry * nn.x;
      const float t0 = B.R[0] * cx + B.R[3] * cy + B.R[6] * cz;
      const float t1 = B.R[1] * cx + B.R[4] * cy + B.R[7] * cz;
      const float t2 = B.R[2] * cx + B.R[5] * cy + B.R[8] * cz;
      invb = (float)a.ncb[gbo] * (1.0f / B.mass + t0 * t0 / B.inertia[0] + t1 * t1 / B.inertia[1] +
                                      t2 * t2 / B.inertia[2]);
    }
    const float w = 1.0f / (ui.w + invb);
    const float3 u = make_float3(ui.x - ubx, ui.y - uby, ui.z - ubz);
    const float3 l = pja_project(lam, u, make_float3(nn.x, nn.y, nn.z), a.ab * nn.w, w, a.mu);
    a.blam[o] = l.x;
    a.blam[o + KbN] = l.y;
    a.blam[o + 2 * KbN] = l.z;
    if (TAPE) {
      float *h = tp.blamh + (size_t)(it + 1) * 3 * KbN;
      h[o] = l.x;
      h[o + KbN] = l.y;
      h[o + 2 * KbN] = l.z;
    }
    sx += l.x;
    sy += l.y;
    sz += l.z;
  }
  const float4 un = make_float4(base.x + base.w * sx, base.y + base.w * sy, base.z + base.w * sz, ui.w);
  a.U[s ^ 1][i] = un;
  if (TAPE) tp.Uh[(size_t)(it + 1) * n + i] = un;
}

// Blocks are dispatched in index order, and the caches keep what was touched last.
// With rev set, a sweep runs over the particles from the last block to the first: the
// serpentine launch shapes reverse every other sweep, starting with the first, so that
// each sweep starts on the particles whose data the stage before it (the contact
// build, or the previous sweep) touched last, while they are still in L2.  That pays
// when the sweep's working set is larger than L2 (a 1M-sphere bed: 41.7 -> 35.1 us per
// sweep) and costs when it fits and the work is uneven (the collapsing column, whose
// contacts sit in its low ids: a reversed sweep dispatches its heavy blocks last, 3.3
// -> 3.7 us), so it is a launch shape the autotuner chooses.  A sweep's order does not
// change its results (Jacobi).
__device__ __forceinline__ uint32_t sweep_particle(int rev) {
  const uint32_t blk = rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
  return blk * blockDim.x + threadIdx.x;
}

// One sweep per launch.
template <bool TAPE, bool PRE = false>
__global__ void __launch_bounds__(512) k_pja(StepArgs a, int s, Tape tp, int it, int rev) {
  pdl_enter();
  const uint32_t i = sweep_particle(rev);
  if (i < a.n) pja_particle<TAPE, false, PRE>(a, i, s, tp, it);
}

// One sweep per launch with at most 40 registers per thread (62.5 % -> 75 % occupancy
// at 256-thread blocks, at the price of a few spilled values): the autotuner's choice
// when the sweep's working set streams from DRAM.
__global__ void __maxnreg__(40) k_pja_lean(StepArgs a, int s, int it, int rev) {
  pdl_enter();
  const uint32_t i = sweep_particle(rev);
  const Tape none{};
  if (i < a.n) pja_particle<false, false>(a, i, s, none, it);
}


// OneLoop, the third form of the paper's loop-structure ablation (Sec. II-D, Fig.
// warp-divergence-performance): every impulse iteration walks the neighbour cells
// again and computes each contact's response as it finds it, instead of reading the
// records that detection stored once per step.  The detection launch still runs
// first, for the contact counts behind the mass-splitting weights, U^0 and the zeroed
// impulses.  The walk yields the same ascending partner list, the geometry comes from
// the same helpers (pair_geometry, body_touch, body_geometry) and the impulses keep
// their ELL slots, so the iterates are bit-identical to the split form (tested).  Not
// with free bodies (their updates run between sweeps) nor taped steps.
template <bool LISTS>
__global__ void __launch_bounds__(kContactsBlock) k_oneloop(StepArgs a, int s) {
  pdl_enter();
  extern __shared__ uint32_t s_fid[];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const float4 pi = a.pos_id[i];
  const uint32_t e = a.env_of[i];
  const DevEnv E = a.envs[e];
  uint32_t *fid = s_fid + threadIdx.x;
  const uint32_t S = blockDim.x;
  uint32_t npp = 0;
  bool ovf = false;
  walk_partners<LISTS>(a, i, pi, E, fid, S, npp, ovf);
  const float4 *__restrict__ Uin = a.U[s];
  float *__restrict__ clam = a.clam;
  const size_t n = a.n, KN = (size_t)a.K * n, KbN = (size_t)a.Kb * n;
  const float4 ui = Uin[i];
  const float4 base = base_velocity(a, a.vel_id[i]);
  const float pw = a.lit ? 0.f : 1.f;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (uint32_t c = 0; c < npp; ++c) {
    const uint32_t j = fid[c * S];
    const float4 g = pair_geometry(pi, a.pos_id[j], i, j);
    const float4 uj = Uin[j];
    const size_t o = (size_t)c * n + i;
    const float3 l = pja_project(make_float3(clam[o], clam[o + KN], clam[o + 2 * KN]),
                                 make_float3(ui.x - uj.x, ui.y - uj.y, ui.z - uj.z), make_float3(g.x, g.y, g.z),
                                 a.ab * g.w, 1.0f / (ui.w + pw * uj.w), a.mu);
    clam[o] = l.x;
    clam[o + KN] = l.y;
    clam[o + 2 * KN] = l.z;
    sx += l.x;
    sy += l.y;
    sz += l.z;
  }
  const float3 xi = make_float3(pi.x, pi.y, pi.z);
  uint32_t nbc = 0;
  for (uint32_t b = 0; b < E.nbodies && nbc < a.Kb; ++b) {
    const DevBody &B = a.bodies[e * a.maxb + b];
    float3 y;
    float f;
    int br;
    if (!body_touch(B, xi, pi.w, &y, &f, &br)) continue;
    float4 bn, bxc;
    body_geometry(B, xi, pi.w, y, f, br, &bn, &bxc);
    const size_t o = (size_t)nbc * n + i;
    const float rx = bxc.x - B.p[0], ry = bxc.y - B.p[1], rz = bxc.z - B.p[2];
    const float ubx = B.v[0] + (B.w[1] * rz - B.w[2] * ry);
    const float uby = B.v[1] + (B.w[2] * rx - B.w[0] * rz);
    const float ubz = B.v[2] + (B.w[0] * ry - B.w[1] * rx);
    const float3 l = pja_project(make_float3(a.blam[o], a.blam[o + KbN], a.blam[o + 2 * KbN]),
                                 make_float3(ui.x - ubx, ui.y - uby, ui.z - ubz), make_float3(bn.x, bn.y, bn.z),
                                 a.ab * bn.w, 1.0f / (ui.w + 0.f), a.mu);
    a.blam[o] = l.x;
    a.blam[o + KbN] = l.y;
    a.blam[o + 2 * KbN] = l.z;
    sx += l.x;
    sy += l.y;
    sz += l.z;
    ++nbc;
  }
  a.U[s ^ 1][i] = make_float4(base.x + base.w * sx, base.y + base.w * sy, base.z + base.w * sz, ui.w);
}

// Grid-wide barrier of a cooperative launch (all blocks resident).  The wait is
// bounded: past `limit` SM cycles it latches kFlagTimeout and sets bar_abort, after
// which every later barrier returns at once, so the kernel always finishes.
__device__ __forceinline__ void grid_barrier(DevCtrl *c, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t *vgen = &c->bar_gen;
    volatile uint32_t *vab = &c->bar_abort;
    const uint32_t gen = *vgen;
    __threadfence();
    const uint32_t arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1 + c->bar_extra) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else if (!*vab) {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*vab) break;
        if (clock64() - t0 > limit) {
          atomicOr(&c->status, kFlagTimeout);
          atomicExch(&c->bar_abort, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// All I sweeps in one persistent cooperative launch (no free bodies): a grid-stride
// loop over particles per sweep, a grid barrier between sweeps.  Same per-particle
// arithmetic as k_pja, so results are bit-identical.
__global__ void __launch_bounds__(1024) k_pja_fused(StepArgs a, uint32_t iters) {
  pdl_enter();
  const Tape none{};
  for (uint32_t it = 0; it < iters; ++it) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x)
      pja_particle<false, true>(a, i, (int)(it & 1), none, (int)it);
    if (it + 1 < iters) grid_barrier(a.ctrl, a.wait_cycles);
  }
}

// Detection and all I sweeps in one persistent cooperative launch (no free bodies):
// the paper's TwoLoopsFused (Sec. II-D, Fig. warp-divergence-performance), the
// collision loop and the impulse loop kept as two loops of one kernel.  A sweep needs
// the contact count of every partner (the mass-splitting weight) and the partner's
// first velocity estimate, so a grid barrier separates detection from the first sweep,
// and each sweep from the next.  Each thread handles the same particles in both loops
// (grid-stride), so its own contact records are read back by the SM that wrote them;
// partners' estimates are read through L2.  Same per-particle arithmetic as
// k_contacts + k_pja, so results are bit-identical to the split launches.
constexpr int kDetectSweepBlock = 256;

template <bool LISTS>
__global__ void __launch_bounds__(kDetectSweepBlock) k_detect_sweeps(StepArgs a, uint32_t iters) {
  pdl_enter();
  extern __shared__ uint32_t s_fid[];
  const Tape none{};
  const uint32_t stride = gridDim.x * blockDim.x;
  // every thread of a block runs the same rounds, so the warp-level statistics see all lanes
  for (uint32_t base = blockIdx.x * blockDim.x; base < a.n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    uint32_t npp = 0, nbc = 0;
    float psi_max = 0.f;
    if (i < a.n) detect_particle<LISTS>(a, i, s_fid + threadIdx.x, blockDim.x, npp, nbc, psi_max);
    contact_stats(a, npp, nbc, psi_max);
  }
  grid_barrier(a.ctrl, a.wait_cycles);
  for (uint32_t it = 0; it < iters; ++it) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
      pja_particle<false, true>(a, i, (int)(it & 1), none, (int)it);
    if (it + 1 < iters) grid_barrier(a.ctrl, a.wait_cycles);
  }
}

// ---------------------------------------------------------------------------
// 6b. free rigid bodies: contact list order, corner contacts, per-iteration update
// ---------------------------------------------------------------------------

constexpr int kFreeSortMax = 8192;  // contact-list capacity limit (shared-memory sort)

// One block per free body: sort its contact list (bitonic, ascending), then find
// its box corners touching the environment's non-free bodies (FP32 decision).
__global__ void __launch_bounds__(1024) k_free_prep(StepArgs a) {
  pdl_enter();
  __shared__ uint32_t sk[kFreeSortMax];
  const uint32_t fid = blockIdx.x;
  const uint32_t gb = a.fgb[fid];
  if (gb == 0xffffffffu) return;
  const uint32_t cnt = min(a.fcount[fid], a.Lcap);
  uint32_t P = 1;
  while (P < cnt) P <<= 1;
  uint32_t *lst = a.flist + (size_t)fid * a.Lcap;
  for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) sk[t] = t < cnt ? lst[t] : 0xffffffffu;
  __syncthreads();
  for (uint32_t k = 2; k <= P; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) {
        const uint32_t p = t ^ j;
        if (p > t) {
          const bool up = (t & k) == 0;
          const uint32_t x = sk[t], y = sk[p];
          if ((x > y) == up) {
            sk[t] = y;
            sk[p] = x;
          }
        }
      }
      __syncthreads();
    }
  for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) lst[t] = sk[t];
  // corners of a free box against the non-free bodies of its environment
  const DevBody &B = a.bodies[gb];
  const uint32_t e = gb / a.maxb;
  CornerContact *cc = a.fcc + (size_t)fid * 8 * a.maxb;
  for (uint32_t t = threadIdx.x; t < 8 * a.maxb; t += blockDim.x) {
    const uint32_t corner = t / a.maxb, ob = t % a.maxb;
    CornerContact c{};
    c.o = ob;
    const DevBody &O = a.bodies[e * a.maxb + ob];
    if (B.kind == 1 && e * a.maxb + ob != gb && O.active && !O.is_free) {
      float cw[3];
      const float cf[3] = {(corner & 1) ? B.shape[0] : -B.shape[0], (corner & 2) ? B.shape[1] : -B.shape[1],
                           (corner & 4) ? B.shape[2] : -B.shape[2]};
#pragma unroll
      for (int q = 0; q < 3; ++q)
        cw[q] = __fadd_rn(B.p[q], __fadd_rn(__fadd_rn(__fmul_rn(B.R[3 * q], cf[0]), __fmul_rn(B.R[3 * q + 1], cf[1])),
                                            __fmul_rn(B.R[3 * q + 2], cf[2])));
      const float3 xw = make_float3(cw[0], cw[1], cw[2]);
      const float3 y = world_to_body(O, xw);
      int br;
      const float f = body_sdf(O, y, &br);
      if (f <= 0.0f) {
        const float3 nn = rot_apply(O.R, body_grad(O, y, br));
        c.valid = 1;
        c.n[0] = nn.x;
        c.n[1] = nn.y;
        c.n[2] = nn.z;
        c.psi = -f;
        c.xc[0] = xw.x - f * nn.x;
        c.xc[1] = xw.y - f * nn.y;
        c.xc[2] = xw.z - f * nn.z;
        atomicAdd(&a.ncb[gb], 1u);
      }
    }
    cc[t] = c;
  }
}

__device__ __forceinline__ float free_inv_mass(const DevBody &B, float3 r, float3 n) {
  const float cx = r.y * n.z - r.z * n.y, cy = r.z * n.x - r.x * n.z, cz = r.x * n.y - r.y * n.x;
  const float t0 = B.R[0] * cx + B.R[3] * cy + B.R[6] * cz;
  const float t1 = B.R[1] * cx + B.R[4] * cy + B.R[7] * cz;
  const float t2 = B.R[2] * cx + B.R[5] * cy + B.R[8] * cz;
  return 1.0f / B.mass + t0 * t0 / B.inertia[0] + t1 * t1 / B.inertia[1] + t2 * t2 / B.inertia[2];
}

// After each sweep, one block per free body: update its corner contacts (against
// the twist of this iteration), sum every impulse it received in a fixed order,
// and set its twist for the next iteration (Newton-Euler, gyroscopic term dropped).
__global__ void __launch_bounds__(256) k_free_update(StepArgs a) {
  pdl_enter();
  const uint32_t fid = blockIdx.x;
  const uint32_t gb = a.fgb[fid];
  if (gb == 0xffffffffu) return;
  DevBody &B = a.bodies[gb];
  const uint32_t e = gb / a.maxb;
  const float nb = (float)a.ncb[gb];
  const float3 V = make_float3(B.v[0], B.v[1], B.v[2]), W = make_float3(B.w[0], B.w[1], B.w[2]);
  float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  CornerContact *cc = a.fcc + (size_t)fid * 8 * a.maxb;
  for (uint32_t t = threadIdx.x; t < 8 * a.maxb; t += blockDim.x) {
    CornerContact c = cc[t];
    if (!c.valid) continue;
    const DevBody &O = a.bodies[e * a.maxb + c.o];
    const float3 r = make_float3(c.xc[0] - B.p[0], c.xc[1] - B.p[1], c.xc[2] - B.p[2]);
    const float3 ro = make_float3(c.xc[0] - O.p[0], c.xc[1] - O.p[1], c.xc[2] - O.p[2]);
    const float3 ub = make_float3(V.x + W.y * r.z - W.z * r.y, V.y + W.z * r.x - W.x * r.z, V.z + W.x * r.y - W.y * r.x);
    const float3 uo = make_float3(O.v[0] + O.w[1] * ro.z - O.w[2] * ro.y, O.v[1] + O.w[2] * ro.x - O.w[0] * ro.z,
                                  O.v[2] + O.w[0] * ro.y - O.w[1] * ro.x);
    const float3 nn = make_float3(c.n[0], c.n[1], c.n[2]);
    const float w = 1.0f / (nb * free_inv_mass(B, r, nn));
    const float3 l = pja_project(make_float3(c.lam[0], c.lam[1], c.lam[2]),
                                 make_float3(ub.x - uo.x, ub.y - uo.y, ub.z - uo.z), nn, a.ab * c.psi, w, a.mu);
    cc[t].lam[0] = l.x;
    cc[t].lam[1] = l.y;
    cc[t].lam[2] = l.z;
    v[0] += l.x;
    v[1] += l.y;
    v[2] += l.z;
    v[3] += r.y * l.z - r.z * l.y;
    v[4] += r.z * l.x - r.x * l.z;
    v[5] += r.x * l.y - r.y * l.x;
  }
  const size_t n = a.n, KbN = (size_t)a.Kb * n;
  const uint32_t cnt = min(a.fcount[fid], a.Lcap);
  const uint32_t *lst = a.flist + (size_t)fid * a.Lcap;
  for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
    const uint32_t code = lst[t];
    const size_t o = (size_t)(code % a.Kb) * n + code / a.Kb;
    const float fx = -a.blam[o], fy = -a.blam[o + KbN], fz = -a.blam[o + 2 * KbN];
    const float4 xc = a.bxc[o];
    const float rx = xc.x - B.p[0], ry = xc.y - B.p[1], rz = xc.z - B.p[2];
    v[0] += fx;
    v[1] += fy;
    v[2] += fz;
    v[3] += ry * fz - rz * fy;
    v[4] += rz * fx - rx * fz;
    v[5] += rx * fy - ry * fx;
  }
  block_sum6<256>(v);
  if (threadIdx.x == 0) {
    const float im = 1.0f / B.mass;
    // I_w^-1 L = R diag(1/I) R^T L
    const float t0 = (B.R[0] * v[3] + B.R[3] * v[4] + B.R[6] * v[5]) / B.inertia[0];
    const float t1 = (B.R[1] * v[3] + B.R[4] * v[4] + B.R[7] * v[5]) / B.inertia[1];
    const float t2 = (B.R[2] * v[3] + B.R[5] * v[4] + B.R[8] * v[5]) / B.inertia[2];
    B.v[0] = B.own_v[0] + a.dt * a.g[0] + im * v[0];
    B.v[1] = B.own_v[1] + a.dt * a.g[1] + im * v[1];
    B.v[2] = B.own_v[2] + a.dt * a.g[2] + im * v[2];
    B.w[0] = B.own_w[0] + (B.R[0] * t0 + B.R[1] * t1 + B.R[2] * t2);
    B.w[1] = B.own_w[1] + (B.R[3] * t0 + B.R[4] * t1 + B.R[5] * t2);
    B.w[2] = B.own_w[2] + (B.R[6] * t0 + B.R[7] * t1 + B.R[8] * t2);
  }
}

// ---------------------------------------------------------------------------
// 7. symplectic Euler back into particle-id order
// ---------------------------------------------------------------------------

// Euler update of one particle, in place (Eq. 4-5).
__device__ __forceinline__ void integrate_particle(const StepArgs &a, int s, uint32_t i) {
  const float4 u = a.U[s][i];
  const float4 p = a.pos_id[i];
  const float invm = a.vel_id[i].w;
  const float x = p.x + a.dt * u.x, y = p.y + a.dt * u.y;
  float z = p.z + a.dt * u.z;
  if (a.cyc_h > 0.f && z < a.cyc_lo) z += a.cyc_h;  // cyclic vertical boundary (gear tower)
  if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(u.x) && isfinite(u.y) && isfinite(u.z)))
    flag(a.ctrl, kFlagNonFinite);
  a.pos_id[i] = make_float4(x, y, z, p.w);
  a.vel_id[i] = make_float4(u.x, u.y, u.z, invm);
}

// ---------------------------------------------------------------------------
// 7-8. integration and the wrench partials: one block per chunk of kWrenchChunk
//      particles of one environment; the block integrates its particles, then sums
//      each body's contact forces and torques over them in a fixed order
// ---------------------------------------------------------------------------

// One particle of the chunk per thread.  (Two per thread in 512-thread blocks, so that
// a 262,144-sphere step's 256 chunks fit one wave of two blocks per SM, measured
// slower: 16.0 against 14.3 us for the stage on the column.)
constexpr int kIntegrateThreads = kWrenchChunk;

__global__ void __launch_bounds__(kIntegrateThreads) k_integrate_wrench(StepArgs a, int s, int rev) {
  pdl_enter();
  // rev: the last sweep ran forward in a serpentine launch shape, so start from the last
  // chunk, on the estimates still in L2 (the partials are per chunk: order changes nothing)
  const uint32_t c = rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
  const uint32_t e = a.chunk_env[c];
  const DevEnv &E = a.envs[e];
  const uint32_t s0 = E.off + (c - E.chunk0) * kWrenchChunk;
  const uint32_t s1 = min(s0 + kWrenchChunk, E.off + E.n);
  // one particle per thread (the chunk is the block)
  const uint32_t i = s0 + threadIdx.x;
  const bool own = i < s1;
  const uint32_t nbc = own ? (a.ccount[i] >> 8) & 0xffu : 0u;
  if (own) integrate_particle(a, s, i);
  // linked-list binning: the step's lists have been walked, so empty every bucket for
  // the next step's pushes here instead of in a launch of its own (created empty); the
  // table is padded to a multiple of kScanTile buckets, so it is cleared four at a time
  if (a.lists) {
    uint4 *h4 = reinterpret_cast<uint4 *>(a.head);
    const uint4 empty = make_uint4(kListEnd, kListEnd, kListEnd, kListEnd);
    for (uint32_t b = blockIdx.x * kIntegrateThreads + threadIdx.x; b < a.nh_pad / 4u; b += gridDim.x * kIntegrateThreads)
      h4[b] = empty;
  }
  // no body contact in the chunk (most chunks): every partial of the environment's
  // bodies is zero, written at once (the partials of slot c are contiguous)
  if (!__syncthreads_or(nbc != 0u)) {
    for (uint32_t t = threadIdx.x; t < 6u * E.nbodies; t += kIntegrateThreads)
      a.wpart[(size_t)c * a.maxb * 6 + t] = 0.f;
    return;
  }
  const size_t n = a.n, KbN = (size_t)a.Kb * n;
  const float inv_dt = 1.0f / a.dt;
  for (uint32_t lb = 0; lb < E.nbodies; ++lb) {
    const uint32_t gb = e * a.maxb + lb;
    const DevBody &B = a.bodies[gb];
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int hit = 0;
    for (uint32_t k = 0; k < nbc; ++k) {
      const size_t o = (size_t)k * n + i;
      if (a.bj[o] != gb) continue;
      hit = 1;
      const float fx = -a.blam[o] * inv_dt, fy = -a.blam[o + KbN] * inv_dt, fz = -a.blam[o + 2 * KbN] * inv_dt;
      const float4 xc = a.bxc[o];
      const float rx = xc.x - B.p[0], ry = xc.y - B.p[1], rz = xc.z - B.p[2];
      v[0] += fx;
      v[1] += fy;
      v[2] += fz;
      v[3] += ry * fz - rz * fy;
      v[4] += rz * fx - rx * fz;
      v[5] += rx * fy - ry * fx;
    }
    if (!__syncthreads_or(hit)) {  // no contact with this body in the chunk: zero partial
      if (threadIdx.x < 6) a.wpart[((size_t)c * a.maxb + lb) * 6 + threadIdx.x] = 0.f;
      continue;
    }
    block_sum6<kIntegrateThreads>(v);
    if (threadIdx.x == 0) {
      float *dst = a.wpart + ((size_t)c * a.maxb + lb) * 6;
#pragma unroll
      for (int k = 0; k < 6; ++k) dst[k] = v[k];
    }
    __syncthreads();  // block_sum6's shared slots are reused by the next body
  }
}

// Pose of a body after the step: p += dt v, q <- exp(dt w / 2) q (in registers).
__device__ __forceinline__ void advance_pose(float dt, float p[3], float q[4], const float v[3], const float w[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) p[k] += dt * v[k];
  const float tx = dt * w[0], ty = dt * w[1], tz = dt * w[2];
  const float ang = sqrtf(tx * tx + ty * ty + tz * tz);
  if (ang > 0.f) {
    float sh, ch;
    sincosf(0.5f * ang, &sh, &ch);
    const float sc = sh / ang;
    const float dw = ch, dx = tx * sc, dy = ty * sc, dz = tz * sc;
    const float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    const float rw = dw * qw - dx * qx - dy * qy - dz * qz;
    const float rx = dw * qx + dx * qw + dy * qz - dz * qy;
    const float ry = dw * qy - dx * qz + dy * qw + dz * qx;
    const float rz = dw * qz + dx * qy - dy * qx + dz * qw;
    const float inv = rsqrtf(rw * rw + rx * rx + ry * ry + rz * rz);
    q[0] = rw * inv;
    q[1] = rx * inv;
    q[2] = ry * inv;
    q[3] = rz * inv;
  }
}

// One block per body slot: sum its environment's chunk partials in a fixed order (a
// thread per chunk, strided, then the block's fixed tree) into the wrench ring, then
// advance the body's pose (no block reads another body's pose); a free body keeps the
// twist of its last sweep as its own.  A block's loads are all issued before any is
// used, so the kernel is one memory round trip deep (a warp per body walking the
// chunks in turn was eight round trips deep on a 256-chunk environment: 10 us).  The
// last block to finish advances the step counter (every block read it first; no block
// waits for another).
constexpr int kWrenchBodyThreads = 256;

__global__ void __launch_bounds__(kWrenchBodyThreads) k_wrench_bodies(StepArgs a) {
  pdl_enter();
  const uint32_t gb = blockIdx.x;
  const uint32_t nbt = a.n_envs * a.maxb;
  const uint32_t step = a.ctrl->step;
  DevBody &B = a.bodies[gb];
  const uint32_t e = gb / a.maxb, lb = gb % a.maxb;
  const uint32_t c0 = a.envs[e].chunk0, c1 = c0 + a.envs[e].nchunks;
  const uint32_t active = B.active, is_free = B.is_free;
  float p[3], q[4], bv[3], bw[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p[k] = B.p[k];
    bv[k] = B.v[k];
    bw[k] = B.w[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = B.q[k];
  float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (active) {  // the partials of an inactive slot are never written
#pragma unroll 4
    for (uint32_t c = c0 + threadIdx.x; c < c1; c += kWrenchBodyThreads) {
      const float *src = a.wpart + ((size_t)c * a.maxb + lb) * 6;
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] += src[k];
    }
  }
  block_sum6<kWrenchBodyThreads>(v);
  if (threadIdx.x == 0) {
    if (active && a.F) {  // free-box corners: +lambda on the box, -lambda on the other body
      const float inv_dt = 1.0f / a.dt;
      for (uint32_t ob = 0; ob < a.maxb; ++ob) {
        const DevBody &Fb = a.bodies[e * a.maxb + ob];
        if (!Fb.active || !Fb.is_free) continue;
        const CornerContact *cc = a.fcc + (size_t)Fb.fid * 8 * a.maxb;
        for (uint32_t t = 0; t < 8 * a.maxb; ++t) {
          if (!cc[t].valid) continue;
          const float sg = (e * a.maxb + ob == gb) ? inv_dt : ((e * a.maxb + cc[t].o == gb) ? -inv_dt : 0.f);
          if (sg == 0.f) continue;
          const float fx = sg * cc[t].lam[0], fy = sg * cc[t].lam[1], fz = sg * cc[t].lam[2];
          const float rx = cc[t].xc[0] - p[0], ry = cc[t].xc[1] - p[1], rz = cc[t].xc[2] - p[2];
          v[0] += fx;
          v[1] += fy;
          v[2] += fz;
          v[3] += ry * fz - rz * fy;
          v[4] += rz * fx - rx * fz;
          v[5] += rx * fy - ry * fx;
        }
      }
    }
    float *dst = a.wrench + ((size_t)(step % a.wrench_hist) * nbt + gb) * 6;
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[k] = v[k];
    if (active) {
      advance_pose(a.dt, p, q, bv, bw);
#pragma unroll
      for (int k = 0; k < 3; ++k) B.p[k] = p[k];
#pragma unroll
      for (int k = 0; k < 4; ++k) B.q[k] = q[k];
      if (is_free) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          B.own_v[k] = bv[k];
          B.own_w[k] = bw[k];
        }
      }
    }
    // every thread of this block read the counter before block_sum6's barrier
    if (gridDim.x == 1) {
      a.ctrl->step = step + 1;
    } else {
      __threadfence();
      if (atomicAdd(&a.ctrl->blocks_done, 1u) == gridDim.x - 1) {
        a.ctrl->blocks_done = 0;
        a.ctrl->step = step + 1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// readback helpers (outside the step)
// ---------------------------------------------------------------------------

__global__ void k_export_contacts(StepArgs a, uint32_t *rows, float *geom, float *lam, float *bgeom, float *blam) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const uint32_t id = s;
  const uint32_t K = a.K, Kb = a.Kb, W = 2 + K + Kb;
  const size_t n = a.n;
  const uint32_t cc = a.ccount[s];
  const uint32_t npp = cc & 0xffu, nbc = (cc >> 8) & 0xffu;
  if (rows) {
    uint32_t *r = rows + (size_t)id * W;
    r[0] = npp;
    r[1] = nbc;
    for (uint32_t c = 0; c < K; ++c) r[2 + c] = c < npp ? a.cj[(size_t)c * n + s] : 0xffffffffu;
    for (uint32_t c = 0; c < Kb; ++c) r[2 + K + c] = c < nbc ? a.bj[(size_t)c * n + s] % a.maxb : 0xffffffffu;
  }
  for (uint32_t c = 0; c < K; ++c) {
    const size_t o = (size_t)c * n + s;
    const bool on = c < npp;
    if (geom) {
      float4 g = on ? a.cn[o] : make_float4(0.f, 0.f, 0.f, 0.f);
      float *d = geom + ((size_t)id * K + c) * 4;
      d[0] = g.x;
      d[1] = g.y;
      d[2] = g.z;
      d[3] = g.w;
    }
    if (lam) {
      float *d = lam + ((size_t)id * K + c) * 3;
      d[0] = on ? a.clam[o] : 0.f;
      d[1] = on ? a.clam[o + (size_t)K * n] : 0.f;
      d[2] = on ? a.clam[o + 2 * (size_t)K * n] : 0.f;
    }
  }
  for (uint32_t c = 0; c < Kb; ++c) {
    const size_t o = (size_t)c * n + s;
    const bool on = c < nbc;
    if (bgeom) {
      float4 g = on ? a.bn[o] : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 x = on ? a.bxc[o] : make_float4(0.f, 0.f, 0.f, 0.f);
      float *d = bgeom + ((size_t)id * Kb + c) * 8;
      d[0] = g.x;
      d[1] = g.y;
      d[2] = g.z;
      d[3] = g.w;
      d[4] = x.x;
      d[5] = x.y;
      d[6] = x.z;
      d[7] = 0.f;
    }
    if (blam) {
      float *d = blam + ((size_t)id * Kb + c) * 3;
      d[0] = on ? a.blam[o] : 0.f;
      d[1] = on ? a.blam[o + (size_t)Kb * n] : 0.f;
      d[2] = on ? a.blam[o + 2 * (size_t)Kb * n] : 0.f;
    }
  }
}

// float[n][4] / float[n][3] conversions for user-facing particle arrays
__global__ void k_vel3_to_vel4(float4 *vel_id, const float *vel3, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 v = vel_id[i];
  vel_id[i] = make_float4(vel3[3 * i], vel3[3 * i + 1], vel3[3 * i + 2], v.w);
}

__global__ void k_pack3(float4 *dst, const float *src3, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = src3 ? make_float4(src3[3 * i], src3[3 * i + 1], src3[3 * i + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_vel4_to_vel3(const float4 *vel_id, float *vel3, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 v = vel_id[i];
  vel3[3 * i] = v.x;
  vel3[3 * i + 1] = v.y;
  vel3[3 * i + 2] = v.z;
}

__global__ void k_body_state(const DevBody *bodies, uint32_t nbt, float *out) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbt) return;
  const DevBody &B = bodies[b];
  float *d = out + (size_t)b * 16;
  for (int k = 0; k < 3; ++k) d[k] = B.p[k];
  for (int k = 0; k < 4; ++k) d[3 + k] = B.q[k];
  for (int k = 0; k < 3; ++k) d[7 + k] = B.own_v[k];
  for (int k = 0; k < 3; ++k) d[10 + k] = B.own_w[k];
  d[13] = d[14] = d[15] = 0.f;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static inline unsigned grid_for(uint32_t n, int bs) { return (n + bs - 1) / bs > 0 ? (n + bs - 1) / bs : 1; }

static inline cudaError_t mark(cudaEvent_t *ev, int k, cudaStream_t st) {
  return ev ? cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal) : cudaSuccess;
}

uint32_t kernels_per_step(const StepArgs &a, const LaunchShape &ls) {
  uint32_t k = a.lists ? 2 : 5;  // key (+ scan x3), wrench sums + body poses
  if (a.n && ls.detect && ls.fused_grid && !a.F)
    k += (a.lists ? 0 : 2) + 1;  // (scatter, reorder,) detection + sweeps
  else if (a.n)
    k += (a.lists ? 1 : 3) + (ls.half ? 1 : 0) + ((ls.fused_grid && !a.F) ? 1 : ls.iters);  // (scatter, reorder,) contacts, pja
  if (a.n_chunks) k += 1;  // integrate + wrench partials
  if (a.F) k += 1 + ls.iters;  // free_prep, free_update x I
  return k;
}

cudaError_t enqueue_step(const StepArgs &a, const LaunchShape &ls, cudaStream_t st, cudaEvent_t *ev, const Tape *tp,
                         bool whole) {
  cudaError_t e;
  const uint32_t nbt = a.n_envs * a.maxb;
  const uint32_t nk = a.n > nbt ? a.n : nbt;
  // Programmatic launches chain the kernels of the step; the first kernel after an
  // event record, a copy or the previous step is launched normally.
  const bool allow_pdl = true;
  bool after_kernel = false;
#define GG_LAUNCH(kern, grid, block, smem, ...)                                                       \
  do {                                                                                                \
    if ((e = launch(allow_pdl && after_kernel, kern, grid, block, smem, st, __VA_ARGS__)) != cudaSuccess) \
      return e;                                                                                       \
    after_kernel = true;                                                                              \
  } while (0)
#define GG_MARK(k)                                             \
  do {                                                         \
    if (ev) {                                                  \
      if ((e = mark(ev, k, st)) != cudaSuccess) return e;      \
      after_kernel = false;                                    \
    }                                                          \
  } while (0)
  GG_MARK(0);
  if (a.lists) {
    GG_LAUNCH(k_key, dim3(grid_for(nk, 256)), 256, 0, a);  // the lists were emptied by the last step
  } else {
    GG_LAUNCH(k_key, dim3(grid_for(nk, 256)), 256, 0, a);
    const uint32_t nblk = a.nh_pad / kScanTile;
    GG_LAUNCH(k_scan_reduce, dim3(nblk), kScanThreads, 0, a);
    GG_LAUNCH(k_scan_top, dim3(1), 1024, 0, a, nblk);
    GG_LAUNCH(k_scan_down, dim3(nblk), kScanThreads, 0, a);
    if (a.n) {
      GG_LAUNCH(k_scatter, dim3(grid_for(a.n, 256)), 256, 0, a);
      GG_LAUNCH(k_reorder, dim3(grid_for(a.n, 256)), 256, 0, a);
    }
  }
  GG_MARK(1);
  // detection and the sweeps in one cooperative launch (not with free bodies, whose
  // updates run between sweeps, nor taped)
  const bool detect_fused = ls.detect && ls.fused_grid && !a.F && !tp && a.n;
  if (detect_fused) {
    GG_MARK(2);  // the contact stage is inside the sweeps' launch: its interval stays empty
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ls.fused_grid);
    cfg.blockDim = dim3(kDetectSweepBlock);
    cfg.dynamicSmemBytes = (size_t)a.K * kDetectSweepBlock * sizeof(uint32_t);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if ((e = cudaLaunchKernelEx(&cfg, a.lists ? k_detect_sweeps<true> : k_detect_sweeps<false>, a, ls.iters)) !=
        cudaSuccess)
      return e;
    after_kernel = true;
  } else if (a.n) {
    const size_t smem = (size_t)a.K * kContactsBlock * sizeof(uint32_t);
    const dim3 g(grid_for(a.n, kContactsBlock));
    if (ls.half) {
      if (a.lists)
        GG_LAUNCH(k_pairs_half<true>, g, kContactsBlock, 0, a);
      else
        GG_LAUNCH(k_pairs_half<false>, g, kContactsBlock, 0, a);
      GG_LAUNCH(k_pairs_finish, g, kContactsBlock, smem, a);
    } else if (a.lists) {
      GG_LAUNCH(k_contacts<true>, g, kContactsBlock, smem, a);
    } else {
      GG_LAUNCH(k_contacts<false>, g, kContactsBlock, smem, a);
    }
  }
  if (a.F) GG_LAUNCH(k_free_prep, dim3(a.F), 1024, 0, a);
  if (!detect_fused) GG_MARK(2);
  if (tp && a.n) {  // U^0 and lambda^0 = 0 open the tape
    if ((e = cudaMemcpyAsync(tp->Uh, a.U[0], sizeof(float4) * a.n, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(tp->lamh, 0, sizeof(float) * 3 * (size_t)a.K * a.n, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(tp->blamh, 0, sizeof(float) * 3 * (size_t)a.Kb * a.n, st)) != cudaSuccess) return e;
    after_kernel = false;
  }
  const Tape none{};
  if (detect_fused) {
    // the sweeps ran in the detection launch
  } else if (!tp && ls.fused_grid && !ls.detect && !a.F && a.n) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ls.fused_grid);
    cfg.blockDim = dim3(ls.fused_block);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if ((e = cudaLaunchKernelEx(&cfg, k_pja_fused, a, ls.iters)) != cudaSuccess) return e;
    after_kernel = true;
  } else if (ls.one && !tp && !a.F && a.n) {
    const size_t smem = (size_t)a.K * kContactsBlock * sizeof(uint32_t);
    for (uint32_t it = 0; it < ls.iters; ++it)
      if (a.lists)
        GG_LAUNCH(k_oneloop<true>, dim3(grid_for(a.n, kContactsBlock)), kContactsBlock, smem, a, (int)(it & 1));
      else
        GG_LAUNCH(k_oneloop<false>, dim3(grid_for(a.n, kContactsBlock)), kContactsBlock, smem, a, (int)(it & 1));
  } else
  for (uint32_t it = 0; it < ls.iters; ++it) {
    const int rev = (ls.serp && !tp && it % 2 == 0) ? 1 : 0;  // serpentine: reverse sweeps 0, 2, 4, ...
    if (a.n) {
      if (tp)
        GG_LAUNCH(k_pja<true>, dim3(grid_for(a.n, ls.pja_block)), ls.pja_block, 0, a, (int)(it & 1), *tp, (int)it, 0);
      else if (ls.lean)
        GG_LAUNCH(k_pja_lean, dim3(grid_for(a.n, ls.pja_block)), ls.pja_block, 0, a, (int)(it & 1), (int)it, rev);
      else if (ls.pre)  // the first round's records preloaded (see pja_particle)
        GG_LAUNCH((k_pja<false, true>), dim3(grid_for(a.n, ls.pja_block)), ls.pja_block, 0, a, (int)(it & 1), none,
                  (int)it, rev);
      else
        GG_LAUNCH(k_pja<false>, dim3(grid_for(a.n, ls.pja_block)), ls.pja_block, 0, a, (int)(it & 1), none, (int)it,
                  rev);
    }
    if (a.F) GG_LAUNCH(k_free_update, dim3(a.F), 256, 0, a);
  }
  if (tp && !whole) {  // the taped step ends here; empty the lists it filled
    if (a.lists) GG_LAUNCH(k_list_clear, dim3(std::min<uint32_t>(grid_for(a.nh_total, 256), 4096u)), 256, 0, a);
    return cudaGetLastError();
  }
  GG_MARK(3);
  if (a.n_chunks)
    GG_LAUNCH(k_integrate_wrench, dim3(a.n_chunks), kIntegrateThreads, 0, a, (int)(ls.iters & 1),
              (int)(ls.serp && !tp && ls.iters % 2 == 0));
  GG_LAUNCH(k_wrench_bodies, dim3(nbt), kWrenchBodyThreads, 0, a);
  GG_MARK(4);
#undef GG_LAUNCH
#undef GG_MARK
  return cudaGetLastError();
}

cudaError_t enqueue_sort_from_keys(const StepArgs &a, cudaStream_t st) {
  if (a.n) k_hist_keys<<<grid_for(a.n, 256), 256, 0, st>>>(a);
  const uint32_t nblk = a.nh_pad / kScanTile;
  k_scan_reduce<<<nblk, kScanThreads, 0, st>>>(a);
  k_scan_top<<<1, 1024, 0, st>>>(a, nblk);
  k_scan_down<<<nblk, kScanThreads, 0, st>>>(a);
  if (a.n) {
    k_scatter<<<grid_for(a.n, 256), 256, 0, st>>>(a);
    k_reorder<<<grid_for(a.n, 256), 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

int fused_pja_blocks_per_sm(int block) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pja_fused, block, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per;
}

int detect_sweeps_blocks_per_sm(bool lists, uint32_t K) {
  int per = 0;
  const size_t smem = (size_t)K * kDetectSweepBlock * sizeof(uint32_t);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lists ? k_detect_sweeps<true> : k_detect_sweeps<false>,
                                                    kDetectSweepBlock, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per;
}

cudaError_t enqueue_prep_bodies(const StepArgs &a, cudaStream_t st) {
  const uint32_t nbt = a.n_envs * a.maxb;
  if (nbt) k_prep_bodies<<<grid_for(nbt, 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t enqueue_export_contacts(const StepArgs &a, uint32_t *rows, float *geom, float *lam, float *bgeom,
                                    float *blam, cudaStream_t st) {
  if (a.n) k_export_contacts<<<grid_for(a.n, 256), 256, 0, st>>>(a, rows, geom, lam, bgeom, blam);
  return cudaGetLastError();
}

// Particle state to and from a caller's pinned host buffers, read or written by the
// kernel itself over the host link (no staging copy): pos float[n][4], vel float[n][3]
// (either may be null).  A block moves kIoParticles particles.  The velocities go
// through shared memory, so that the host side is accessed word by word in order (each
// warp instruction covers whole 128-byte lines) instead of at a stride of three words;
// positions are float4 per particle, in order already.
constexpr int kIoThreads = 256;
constexpr uint32_t kIoParticles = 1024;

__global__ void __launch_bounds__(kIoThreads) k_state_out(const float4 *__restrict__ pos_id,
                                                          const float4 *__restrict__ vel_id, float4 *__restrict__ pos,
                                                          float *__restrict__ vel, uint32_t n, const DevCtrl *ctrl,
                                                          DevCtrl *ctrl_out) {
  __shared__ float sv[3 * kIoParticles];
  const uint32_t base = blockIdx.x * kIoParticles;
  if (ctrl_out && blockIdx.x == 0 && threadIdx.x == 0) *ctrl_out = *ctrl;  // the status word rides along
  const uint32_t m = min(kIoParticles, n - base);
#pragma unroll 4
  for (uint32_t k = threadIdx.x; k < m; k += kIoThreads) {
    if (pos) pos[base + k] = pos_id[base + k];
    if (vel) {
      const float4 v = vel_id[base + k];
      sv[3 * k] = v.x;
      sv[3 * k + 1] = v.y;
      sv[3 * k + 2] = v.z;
    }
  }
  if (!vel) return;  // uniform over the block
  __syncthreads();
  float *dst = vel + 3 * (size_t)base;
#pragma unroll 4
  for (uint32_t w = threadIdx.x; w < 3 * m; w += kIoThreads) dst[w] = sv[w];
}

__global__ void __launch_bounds__(kIoThreads) k_state_in(float4 *__restrict__ pos_id, float4 *__restrict__ vel_id,
                                                         const float4 *__restrict__ pos, const float *__restrict__ vel,
                                                         uint32_t n) {
  __shared__ float sv[3 * kIoParticles];
  const uint32_t base = blockIdx.x * kIoParticles;
  const uint32_t m = min(kIoParticles, n - base);
  if (vel) {
    const float *src = vel + 3 * (size_t)base;
#pragma unroll 4
    for (uint32_t w = threadIdx.x; w < 3 * m; w += kIoThreads) sv[w] = src[w];
  }
  if (pos) {
#pragma unroll 4
    for (uint32_t k = threadIdx.x; k < m; k += kIoThreads) pos_id[base + k] = pos[base + k];
  }
  if (!vel) return;  // uniform over the block
  __syncthreads();
#pragma unroll 4
  for (uint32_t k = threadIdx.x; k < m; k += kIoThreads) {
    const uint32_t i = base + k;
    vel_id[i] = make_float4(sv[3 * k], sv[3 * k + 1], sv[3 * k + 2], vel_id[i].w);
  }
}

cudaError_t enqueue_state_out(const float4 *pos_id, const float4 *vel_id, float *pos, float *vel, uint32_t n,
                              const DevCtrl *ctrl, DevCtrl *ctrl_out, cudaStream_t st) {
  if (n || ctrl_out)
    k_state_out<<<grid_for(n, kIoParticles), kIoThreads, 0, st>>>(pos_id, vel_id, reinterpret_cast<float4 *>(pos), vel,
                                                                  n, ctrl, ctrl_out);
  return cudaGetLastError();
}

cudaError_t enqueue_state_in(float4 *pos_id, float4 *vel_id, const float *pos, const float *vel, uint32_t n,
                             cudaStream_t st) {
  if (n)
    k_state_in<<<grid_for(n, kIoParticles), kIoThreads, 0, st>>>(pos_id, vel_id, reinterpret_cast<const float4 *>(pos),
                                                                 vel, n);
  return cudaGetLastError();
}

cudaError_t enqueue_vel3_to_vel4(float4 *vel_id, const float *vel3, uint32_t n, cudaStream_t st) {
  if (n) k_vel3_to_vel4<<<grid_for(n, 256), 256, 0, st>>>(vel_id, vel3, n);
  return cudaGetLastError();
}

cudaError_t enqueue_pack3(float4 *dst, const float *src3, uint32_t n, cudaStream_t st) {
  if (n) k_pack3<<<grid_for(n, 256), 256, 0, st>>>(dst, src3, n);
  return cudaGetLastError();
}

cudaError_t enqueue_vel4_to_vel3(const float4 *vel_id, float *vel3, uint32_t n, cudaStream_t st) {
  if (n) k_vel4_to_vel3<<<grid_for(n, 256), 256, 0, st>>>(vel_id, vel3, n);
  return cudaGetLastError();
}

cudaError_t enqueue_body_state(const DevBody *bodies, uint32_t nbt, float *out, cudaStream_t st) {
  if (nbt) k_body_state<<<grid_for(nbt, 128), 128, 0, st>>>(bodies, nbt, out);
  return cudaGetLastError();
}

}  // namespace gg
