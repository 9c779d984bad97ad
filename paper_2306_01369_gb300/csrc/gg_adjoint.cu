// gg_adjoint.cu -- reverse-mode adjoint of one time step (beyond the paper: its
// Sec. V lists differentiability as future work).
//
// The step is a piecewise-smooth map; its adjoint keeps the contact set and the
// branch of every projection (separating / sticking / sliding) as the forward
// took them.  Per step, after a taped forward of binning, contacts and the I
// sweeps (every iterate U^s, lambda^s kept):
//   k_adj_twins     position of each directed pair contact's twin (j -> i)
//   k_adj_begin     U-bar^I = v-bar + dt x-bar (integrator), clear accumulators
//   k_adj_iter  s   completes U-bar^{s+1} with the twin contacts' u-bar of sweep s+1
//                   (U-bar_i = sum over own contacts of u-bar_c - u-bar_twin(c)), then per
//                   contact: z-bar = J_proj^T (lambda-bar), u-bar = -w z-bar, psi-bar,
//                   n-bar, mu-bar; tool twist partials
//   k_adj_geom      completes U-bar^0; positions through psi, normals, SDF branches;
//                   tool pose partials
//   k_adj_tool      fixed-order sums, tool pose chain (p, R) -> twist gradient
// No floating-point atomics: every sum is per particle in contact order, per block
// in a fixed tree, then over blocks in index order.
#include <algorithm>

#include "gg_device.cuh"
#include "gg_internal.h"

namespace gg {

namespace {

constexpr int kAdjThreads = 256;
constexpr int kPart = 10;  // per-block partials: V(3), W(3), p(3), mu | geometry: p(3), r(3)

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float3 ld3(const float *p, size_t o, size_t plane) {
  return make_float3(p[o], p[o + plane], p[o + 2 * plane]);
}
__device__ __forceinline__ void st3(float *p, size_t o, size_t plane, float3 v) {
  p[o] = v.x;
  p[o + plane] = v.y;
  p[o + 2 * plane] = v.z;
}
__device__ __forceinline__ void acc3(float *p, size_t o, size_t plane, float3 v) {
  p[o] += v.x;
  p[o + plane] += v.y;
  p[o + 2 * plane] += v.z;
}

// Adjoint of the cone projection lambda = P(z; n, mu) of pja_cone, with the branch the
// forward took (recomputed from the same z).  Given abar = dL/dlambda returns
// zbar = (dP/dz)^T abar, adds (dP/dn)^T abar to *nbar and (dP/dmu) . abar to *mubar.
__device__ __forceinline__ float3 cone_adjoint(float3 z, float3 n, float mu, float3 abar, float3 *nbar,
                                               float *mubar) {
  const float ln = z.x * n.x + z.y * n.y + z.z * n.z;
  const float lnp = fmaxf(ln, 0.0f);
  const float3 t = make_float3(z.x - ln * n.x, z.y - ln * n.y, z.z - ln * n.z);
  const float t2 = t.x * t.x + t.y * t.y + t.z * t.z;
  const float lim = mu * lnp;
  if (!(ln > 0.0f)) return make_float3(0.f, 0.f, 0.f);  // separated: P = 0
  if (!(t2 > lim * lim)) return abar;                     // sticking: P = z (no n, mu dependence)
  // sliding: P = ln n + mu ln t^
  const float tn = sqrtf(t2), it = 1.0f / tn;
  const float3 th = mul(it, t);
  const float an = dot(abar, n), at = dot(abar, th);
  const float k = mu * ln * it;
  // zbar = n (an + mu at) + (mu ln / |t|) (abar - t^ at - n an)
  const float3 zb = add(mul(an + mu * at, n), mul(k, sub(sub(abar, mul(at, th)), mul(an, n))));
  // nbar += z (an + mu at - mu ln an / |t|) + ln abar - (mu ln^2 / |t|) (abar - t^ at)
  const float3 nb = add(add(mul(an + mu * at - k * an, z), mul(ln, abar)), mul(-k * ln, sub(abar, mul(at, th))));
  *nbar = add(*nbar, nb);
  *mubar += ln * at;
  return zb;
}

// Jacobian^T of the unit SDF gradient (body frame) for the branch taken, applied to gb.
// Flat-face branches have a constant gradient (zero Jacobian).
__device__ __forceinline__ float3 box_grad_adj(float3 y, const float *h, int branch, float3 gb) {
  if (branch != 3) return make_float3(0.f, 0.f, 0.f);
  const float a0 = fabsf(y.x) > h[0] ? 1.f : 0.f, a1 = fabsf(y.y) > h[1] ? 1.f : 0.f, a2 = fabsf(y.z) > h[2] ? 1.f : 0.f;
  const float m0 = a0 * copysignf(fabsf(y.x) - h[0], y.x), m1 = a1 * copysignf(fabsf(y.y) - h[1], y.y),
              m2 = a2 * copysignf(fabsf(y.z) - h[2], y.z);
  const float mn = sqrtf(m0 * m0 + m1 * m1 + m2 * m2);
  const float3 g = make_float3(m0 / mn, m1 / mn, m2 / mn);
  const float gg = dot(g, gb);
  // (I - g g^T) gb / |m|, then the active-axis mask
  return make_float3(a0 * (gb.x - g.x * gg) / mn, a1 * (gb.y - g.y * gg) / mn, a2 * (gb.z - g.z * gg) / mn);
}

// Gridded SDF: the unit gradient n = g / |g| of the trilinear interpolant has
// dn/dy = (I - n n^T) H / |g|, H the interpolant's Hessian in y (only its mixed terms
// are non-zero); H is symmetric, so (dn/dy)^T gb = H (I - n n^T) gb / |g|.
__device__ __forceinline__ float3 grid_grad_adj(const DevBody &b, float3 y, int branch, float3 gb) {
  float3 hm;
  const float ih = b.shape[4];
  const float3 g = mul(ih, grid_dt(b, y, branch, &hm));
  const float gl = sqrtf(dot(g, g));
  if (!(gl > 0.f)) return make_float3(0.f, 0.f, 0.f);
  const float3 n = mul(1.0f / gl, g);
  const float3 p = sub(gb, mul(dot(n, gb), n));
  const float s = ih * ih / gl;
  return make_float3(s * (hm.x * p.y + hm.y * p.z), s * (hm.x * p.x + hm.z * p.z), s * (hm.y * p.x + hm.z * p.y));
}

// d f / d y (body frame): the unit normal of a true SDF; for samples on a grid, the
// interpolant's own gradient (not unit length in general).
__device__ __forceinline__ float3 body_fgrad(const DevBody &b, float3 y, int branch) {
  if (b.kind == 4) return mul(b.shape[4], grid_dt(b, y, branch, nullptr));
  return body_grad(b, y, branch);
}

__device__ __forceinline__ float3 body_grad_adj(const DevBody &b, float3 y, int branch, float3 gb) {
  if (b.kind == 4) return grid_grad_adj(b, y, branch, gb);
  if (b.kind == 5) {  // tube: n = -(y_x, y_y, 0) / rho, dn/dy = -(I_2 - n n^T) / rho on the xy block
    const float rho = sqrtf(y.x * y.x + y.y * y.y);
    if (!(rho > 0.f)) return make_float3(0.f, 0.f, 0.f);
    const float nx = -y.x / rho, ny = -y.y / rho, d = nx * gb.x + ny * gb.y;
    return make_float3(-(gb.x - nx * d) / rho, -(gb.y - ny * d) / rho, 0.f);
  }
  if (b.kind == 1) return box_grad_adj(y, b.shape, branch, gb);
  if (b.kind == 2) {
    if (branch < 4) return box_grad_adj(y, b.shape, branch, gb);
    const float3 z = make_float3(y.x - b.shape[6], y.y - b.shape[7], y.z - b.shape[8]);
    return box_grad_adj(z, b.shape + 3, branch - 4, mul(-1.f, gb));
  }
  return make_float3(0.f, 0.f, 0.f);
}

__device__ __forceinline__ float3 rotT(const float *R, float3 v) {
  return make_float3(R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
                     R[2] * v.x + R[5] * v.y + R[8] * v.z);
}

// fixed-order block sum of kPart floats into part[blk][*]
__device__ __forceinline__ void block_partials(float v[kPart], float *dst) {
  __shared__ float sm[kAdjThreads / 32][kPart];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kPart; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kPart; ++k) sm[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x < kPart) {
    float s = sm[0][threadIdx.x];
    for (int w = 1; w < kAdjThreads / 32; ++w) s += sm[w][threadIdx.x];
    dst[threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_twins(StepArgs a, AdjArgs d) {
  pdl_enter();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const size_t n = a.n;
  const uint32_t npp = a.ccount[i] & 0xffu;
  for (uint32_t c = 0; c < npp; ++c) {
    const uint32_t j = a.cj[(size_t)c * n + i];
    const uint32_t nj = a.ccount[j] & 0xffu;
    uint32_t t = 0xffffffffu;
    for (uint32_t q = 0; q < nj; ++q)
      if (a.cj[(size_t)q * n + j] == i) t = q;
    if (t == 0xffffffffu) {  // only after a capacity overflow truncated one side
      atomicOr(&a.ctrl->status, kFlagPPOverflow);
      t = c;
    }
    d.twin[(size_t)c * n + i] = t;
  }
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_begin(StepArgs a, AdjArgs d) {
  pdl_enter();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const size_t n = a.n, KN = (size_t)a.K * n, KbN = (size_t)a.Kb * n;
  const uint32_t id = s;
  const float4 xb = d.xbar[id], vb = d.vbar[id];
  d.xbar_s[s] = xb;
  const float4 ub = make_float4(vb.x + a.dt * xb.x, vb.y + a.dt * xb.y, vb.z + a.dt * xb.z, 0.f);
  d.Ubar[0][s] = ub;
  d.basebar[s] = ub;
  const uint32_t cc = a.ccount[s];
  const uint32_t npp = cc & 0xffu, nbc = (cc >> 8) & 0xffu;
  const float3 zero = make_float3(0.f, 0.f, 0.f);
  for (uint32_t c = 0; c < npp; ++c) {
    const size_t o = (size_t)c * n + s;
    st3(d.Lbar, o, KN, zero);
    st3(d.nbar, o, KN, zero);
    d.psibar[o] = 0.f;
  }
  for (uint32_t c = 0; c < nbc; ++c) {
    const size_t o = (size_t)c * n + s;
    st3(d.bLbar, o, KbN, zero);
    st3(d.bnbar, o, KbN, zero);
    st3(d.bxcbar, o, KbN, zero);
    d.bpsibar[o] = 0.f;
  }
}

// Subtracts the twin contacts' u-bar (of the sweep whose u-bar is in `ub`) from U, the
// own-contact part of a U-bar, and adds the completed U-bar to the base velocity's.
__device__ __forceinline__ float4 complete_ubar(const StepArgs &a, const AdjArgs &d, uint32_t i, float4 U,
                                                const float *ub) {
  const size_t n = a.n, KN = (size_t)a.K * n;
  const uint32_t npp = a.ccount[i] & 0xffu;
#pragma unroll 4
  for (uint32_t c = 0; c < npp; ++c) {  // loads only: four contacts' gathers in flight
    const size_t o = (size_t)c * n + i;
    const uint32_t tw = d.twin[o], jt = a.cj[o];
    if (!GG_GUARD(a.ctrl, tw < a.K && jt < a.n)) continue;
    const size_t ot = (size_t)tw * n + jt;
    U.x -= ub[ot];
    U.y -= ub[ot + KN];
    U.z -= ub[ot + 2 * KN];
  }
  const float4 b = d.basebar[i];
  d.basebar[i] = make_float4(b.x + U.x, b.y + U.y, b.z + U.z, 0.f);
  return U;
}

// Reverse of sweep s (U^s, lambda^s -> lambda^{s+1}, U^{s+1}).  Ubar[cur] holds the
// own-contact part of the adjoint of U^{s+1} (complete for s + 1 = I); the own-contact
// part of the adjoint of U^s goes to Ubar[cur ^ 1], this sweep's u-bar to ubar[s & 1].
__global__ void __launch_bounds__(kAdjThreads) k_adj_iter(StepArgs a, AdjArgs d, uint32_t s, int cur) {
  pdl_enter();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  float part[kPart] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (i < a.n) {
    const size_t n = a.n, KN = (size_t)a.K * n, KbN = (size_t)a.Kb * n;
    float4 Un = d.Ubar[cur][i];
    if (s + 1 < d.I) Un = complete_ubar(a, d, i, Un, d.ubar[(s + 1) & 1u]);
    float *ubar = d.ubar[s & 1u];
    const float invm = a.vel_id[i].w;
    const float4 Ui = d.tp.Uh[(size_t)s * n + i];
    const float *lh = d.tp.lamh + (size_t)s * 3 * KN;
    const float *blh = d.tp.blamh + (size_t)s * 3 * KbN;
    const uint32_t cc = a.ccount[i];
    const uint32_t npp = cc & 0xffu, nbc = (cc >> 8) & 0xffu;
    float3 S = make_float3(0.f, 0.f, 0.f);
    float mub = 0.f;
    // Reverse of one contact update, from its loaded inputs; stores its adjoints.
    const float4 *Uh = d.tp.Uh + (size_t)s * n;
    auto contact = [&](size_t o, float4 nn, float3 lam, float3 Lb, float psb, float3 nbo, float4 Uj) {
      const float3 nv = f3(nn);
      const float w = 1.0f / (Ui.w + Uj.w);
      const float bias = a.ab * nn.w;
      const float3 z = pja_pre(lam, make_float3(Ui.x - Uj.x, Ui.y - Uj.y, Ui.z - Uj.z), nv, bias, w);
      const float3 abar = add(mul(invm, f3(Un)), Lb);
      float3 nb = make_float3(0.f, 0.f, 0.f);
      const float3 zb = cone_adjoint(z, nv, a.mu, abar, &nb, &mub);
      st3(d.Lbar, o, KN, zb);
      const float3 ub = mul(-w, zb);
      st3(ubar, o, KN, ub);
      S = add(S, ub);
      d.psibar[o] = psb + w * a.ab * dot(nv, zb);
      st3(d.nbar, o, KN, add(nbo, add(mul(w * bias, zb), nb)));
    };
    // two contacts per round: both contacts' loads are issued before either's stores
    uint32_t c = 0;
    for (; c + 1 < npp; c += 2) {
      const size_t o0 = (size_t)c * n + i, o1 = o0 + n;
      uint32_t j0 = a.cj[o0], j1 = a.cj[o1];
      if (!GG_GUARD(a.ctrl, j0 < a.n && j1 < a.n)) j0 = j1 = i;
      const float4 nn0 = a.cn[o0], nn1 = a.cn[o1];
      const float3 lm0 = ld3(lh, o0, KN), lm1 = ld3(lh, o1, KN);
      const float3 Lb0 = ld3(d.Lbar, o0, KN), Lb1 = ld3(d.Lbar, o1, KN);
      const float ps0 = d.psibar[o0], ps1 = d.psibar[o1];
      const float3 nb0 = ld3(d.nbar, o0, KN), nb1 = ld3(d.nbar, o1, KN);
      const float4 Uj0 = Uh[j0], Uj1 = Uh[j1];
      contact(o0, nn0, lm0, Lb0, ps0, nb0, Uj0);
      contact(o1, nn1, lm1, Lb1, ps1, nb1, Uj1);
    }
    if (c < npp) {
      const size_t o = (size_t)c * n + i;
      uint32_t j = a.cj[o];
      if (!GG_GUARD(a.ctrl, j < a.n)) j = i;
      contact(o, a.cn[o], ld3(lh, o, KN), ld3(d.Lbar, o, KN), d.psibar[o], ld3(d.nbar, o, KN), Uh[j]);
    }
    for (uint32_t c = 0; c < nbc; ++c) {
      const size_t o = (size_t)c * n + i;
      const uint32_t gb = a.bj[o];
      const DevBody &B = a.bodies[gb];
      const float4 nn = a.bn[o];
      const float3 nv = f3(nn);
      const float3 xc = f3(a.bxc[o]);
      const float3 r = make_float3(xc.x - B.p[0], xc.y - B.p[1], xc.z - B.p[2]);
      const float3 W = make_float3(B.w[0], B.w[1], B.w[2]);
      const float3 ubody = add(make_float3(B.v[0], B.v[1], B.v[2]), cross(W, r));
      const float w = 1.0f / Ui.w;
      const float bias = a.ab * nn.w;
      const float3 z = pja_pre(ld3(blh, o, KbN), sub(f3(Ui), ubody), nv, bias, w);
      const float3 abar = add(mul(invm, f3(Un)), ld3(d.bLbar, o, KbN));
      float3 nb = make_float3(0.f, 0.f, 0.f);
      const float3 zb = cone_adjoint(z, nv, a.mu, abar, &nb, &mub);
      st3(d.bLbar, o, KbN, zb);
      const float3 uu = mul(-w, zb);  // adjoint of u = U_i - u_body
      S = add(S, uu);
      d.bpsibar[o] += w * a.ab * dot(nv, zb);
      acc3(d.bnbar, o, KbN, add(mul(w * bias, zb), nb));
      const float3 ubb = mul(-1.f, uu);  // adjoint of the body point velocity
      acc3(d.bxcbar, o, KbN, mul(-1.f, cross(W, ubb)));  // u_body = V + W x (x_c - p)
      if (gb == d.tool) {
        const float3 wr = cross(r, ubb), pw = cross(W, ubb);
        part[0] += ubb.x;
        part[1] += ubb.y;
        part[2] += ubb.z;
        part[3] += wr.x;
        part[4] += wr.y;
        part[5] += wr.z;
        part[6] += pw.x;
        part[7] += pw.y;
        part[8] += pw.z;
      }
    }
    part[9] = mub;
    d.Ubar[cur ^ 1][i] = make_float4(S.x, S.y, S.z, 0.f);
  }
  block_partials(part, d.part + ((size_t)s * d.nblk + blockIdx.x) * kPart);
}

// gradient of a pair contact's psi and normal w.r.t. the particle's own position
__device__ __forceinline__ float3 pair_geom_grad(const AdjArgs &d, const StepArgs &a, size_t o, size_t KN, float dist) {
  const float4 nn = a.cn[o];
  const float3 nv = f3(nn);
  const float3 nb = ld3(d.nbar, o, KN);
  const float nbn = dot(nb, nv);
  const float id = dist > 0.f ? 1.0f / dist : 0.f;
  return add(mul(-d.psibar[o], nv), mul(id, sub(nb, mul(nbn, nv))));
}

// Ubar[cur] holds the own-contact part of the adjoint of U^0 (completed here with
// sweep 0's twin u-bar); then the adjoint of the step's input positions and velocities.
__global__ void __launch_bounds__(kAdjThreads) k_adj_geom(StepArgs a, AdjArgs d, int cur) {
  pdl_enter();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  float part[kPart] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (i < a.n) {
    (void)complete_ubar(a, d, i, d.Ubar[cur][i], d.ubar[0]);
    const size_t n = a.n, KN = (size_t)a.K * n, KbN = (size_t)a.Kb * n;
    const float4 pi = a.pos_id[i];
    float3 X = f3(d.xbar_s[i]);
    const uint32_t cc = a.ccount[i];
    const uint32_t npp = cc & 0xffu, nbc = (cc >> 8) & 0xffu;
    for (uint32_t c = 0; c < npp; ++c) {
      const size_t o = (size_t)c * n + i;
      const uint32_t j = a.cj[o];
      const float dist = pi.w + a.pos_id[j].w - a.cn[o].w;
      const size_t ot = (size_t)d.twin[o] * n + j;
      X = add(X, sub(pair_geom_grad(d, a, o, KN, dist), pair_geom_grad(d, a, ot, KN, dist)));
    }
    const float3 xi = f3(pi);
    for (uint32_t c = 0; c < nbc; ++c) {
      const size_t o = (size_t)c * n + i;
      const uint32_t gb = a.bj[o];
      const DevBody &B = a.bodies[gb];
      const float4 nn = a.bn[o];
      const float3 nv = f3(nn);
      const float f = pi.w - nn.w;
      const float3 xcb = ld3(d.bxcbar, o, KbN);
      // x_c = x - f n;  psi = r - f;  n = R g(y);  y = R^T (x - p)
      X = add(X, xcb);
      const float fb = -dot(xcb, nv) - d.bpsibar[o];
      const float3 nb = sub(ld3(d.bnbar, o, KbN), mul(f, xcb));
      const float3 dvec = make_float3(xi.x - B.p[0], xi.y - B.p[1], xi.z - B.p[2]);
      const float3 y = world_to_body(B, xi);
      int br;
      (void)body_sdf(B, y, &br);
      const float3 yb = body_grad_adj(B, y, br, rotT(B.R, nb));
      const float3 Ryb = rot_apply(B.R, yb);
      const float3 gw = rot_apply(B.R, body_fgrad(B, y, br));  // d f / d x
      X = add(X, add(mul(fb, gw), Ryb));
      if (gb == d.tool) {
        const float3 pb = mul(-1.f, add(mul(fb, gw), Ryb));
        const float3 rb = add(add(mul(fb, cross(gw, dvec)), cross(nv, nb)), cross(Ryb, dvec));
        part[0] += pb.x;
        part[1] += pb.y;
        part[2] += pb.z;
        part[3] += rb.x;
        part[4] += rb.y;
        part[5] += rb.z;
      }
    }
    const uint32_t id = i;
    d.xbar[id] = make_float4(X.x, X.y, X.z, 0.f);
    const float4 b = d.basebar[i];
    d.vbar[id] = make_float4(b.x, b.y, b.z, 0.f);
  }
  block_partials(part, d.part + ((size_t)d.I * d.nblk + blockIdx.x) * kPart);
}

__device__ void rodrigues(float3 phi, float R[9]) {
  const float th = sqrtf(dot(phi, phi));
  float A, Bc;
  if (th < 1e-4f) {
    A = 1.f - th * th / 6.f;
    Bc = 0.5f - th * th / 24.f;
  } else {
    A = sinf(th) / th;
    Bc = (1.f - cosf(th)) / (th * th);
  }
  const float K[9] = {0.f, -phi.z, phi.y, phi.z, 0.f, -phi.x, -phi.y, phi.x, 0.f};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      float kk = 0.f;
      for (int m = 0; m < 3; ++m) kk += K[3 * r + m] * K[3 * m + c];
      R[3 * r + c] = (r == c ? 1.f : 0.f) + A * K[3 * r + c] + Bc * kk;
    }
}

// left Jacobian of SO(3): Exp(phi + d) ~ Exp(J_l(phi) d) Exp(phi)
__device__ void left_jacobian(float3 phi, float J[9]) {
  const float th = sqrtf(dot(phi, phi));
  float A, Bc;
  if (th < 1e-3f) {
    A = 0.5f - th * th / 24.f;
    Bc = 1.f / 6.f - th * th / 120.f;
  } else {
    A = (1.f - cosf(th)) / (th * th);
    Bc = (th - sinf(th)) / (th * th * th);
  }
  const float K[9] = {0.f, -phi.z, phi.y, phi.z, 0.f, -phi.x, -phi.y, phi.x, 0.f};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      float kk = 0.f;
      for (int m = 0; m < 3; ++m) kk += K[3 * r + m] * K[3 * m + c];
      J[3 * r + c] = (r == c ? 1.f : 0.f) + A * K[3 * r + c] + Bc * kk;
    }
}

// Sums the partials in a fixed order (thread-strided over the (sweep, block) vectors in
// float, a fixed butterfly in each warp, then the warps in index order in double), and
// thread 0 runs the tool pose chain of step k.  k is the step counter less the one saved
// with the taped run's first checkpoint (`ctrl0`), so one captured graph serves every
// step.  (Double accumulation per thread cost 29 us per step on GB300's FP64 rate.)
constexpr int kToolThreads = 512;
__global__ void __launch_bounds__(kToolThreads) k_adj_tool(StepArgs a, AdjArgs d, const DevCtrl *ctrl0,
                                                          uint32_t n_taped) {
  pdl_enter();
  const uint32_t k_local = a.ctrl->step - ctrl0->step;
  float f[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) f[q] = 0.f;
  const uint32_t I = d.I, nb = d.nblk;
#pragma unroll 2
  for (uint32_t t = threadIdx.x; t < I * nb; t += kToolThreads) {  // t = s * nblk + b
    const float *p = d.part + (size_t)t * kPart;
#pragma unroll
    for (int q = 0; q < kPart; ++q) f[q] += p[q];
  }
  for (uint32_t b = threadIdx.x; b < nb; b += kToolThreads) {
    const float *g = d.part + ((size_t)I * nb + b) * kPart;
#pragma unroll
    for (int q = 0; q < 6; ++q) f[10 + q] += g[q];
  }
#pragma unroll
  for (int q = 0; q < 16; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f[q] += __shfl_xor_sync(0xffffffffu, f[q], o);
  __shared__ float sm[kToolThreads / 32][16];
  __shared__ double tot[16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 16; ++q) sm[wid][q] = f[q];
  __syncthreads();
  if (threadIdx.x < 16) {  // one component per thread, warps in index order
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kToolThreads / 32; ++w) t += (double)sm[w][threadIdx.x];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = tot[q];
  d.mubar[0] += v[9];
  if (d.tool == 0xffffffffu || k_local >= n_taped) return;
  const DevBody &B = a.bodies[d.tool];
  const float3 W = make_float3(B.w[0], B.w[1], B.w[2]);
  const float3 pb1 = make_float3(d.pose_bar[0], d.pose_bar[1], d.pose_bar[2]);
  const float3 rb1 = make_float3(d.pose_bar[3], d.pose_bar[4], d.pose_bar[5]);
  const float3 phi = mul(a.dt, W);
  float J[9], E[9];
  left_jacobian(phi, J);
  rodrigues(phi, E);
  const float3 Jt = rotT(J, rb1);
  const float3 Et = rotT(E, rb1);
  float *tw = d.dtwist + (size_t)k_local * 6;
  tw[0] = (float)v[0] + a.dt * pb1.x;
  tw[1] = (float)v[1] + a.dt * pb1.y;
  tw[2] = (float)v[2] + a.dt * pb1.z;
  tw[3] = (float)v[3] + a.dt * Jt.x;
  tw[4] = (float)v[4] + a.dt * Jt.y;
  tw[5] = (float)v[5] + a.dt * Jt.z;
  d.pose_bar[0] = pb1.x + (float)(v[6] + v[10]);
  d.pose_bar[1] = pb1.y + (float)(v[7] + v[11]);
  d.pose_bar[2] = pb1.z + (float)(v[8] + v[12]);
  d.pose_bar[3] = Et.x + (float)v[13];
  d.pose_bar[4] = Et.y + (float)v[14];
  d.pose_bar[5] = Et.z + (float)v[15];
}

inline unsigned blocks(uint32_t n) { return n ? (n + kAdjThreads - 1) / kAdjThreads : 1; }

// Up to four word regions copied in one launch (grid-stride over their concatenation).
__global__ void k_copy_regions(CopyRegions c) {
  size_t total = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) total += c.words[r];
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    size_t w = t;
    int r = 0;
    while (r < 3 && w >= c.words[r]) w -= c.words[r++];
    c.dst[r][w] = c.src[r][w];
  }
}

}  // namespace

cudaError_t enqueue_copy_regions(const CopyRegions &c, cudaStream_t st) {
  size_t total = 0;
  for (int r = 0; r < 4; ++r) total += c.words[r];
  if (total) k_copy_regions<<<(unsigned)std::min<size_t>((total + 255) / 256, 1024), 256, 0, st>>>(c);
  return cudaGetLastError();
}

uint32_t adjoint_blocks(uint32_t n) { return blocks(n); }

// The step's adjoint kernels, chained with programmatic dependent launch (every one
// begins with pdl_enter); the first follows the body-frame kernel of the step.
cudaError_t enqueue_adjoint_step(const StepArgs &a, const AdjArgs &d, const DevCtrl *ctrl0, uint32_t n_taped,
                                 cudaStream_t st) {
  const dim3 g(blocks(a.n));
  cudaError_t e;
  if (a.n) {
    if ((e = launch(true, k_adj_twins, g, kAdjThreads, 0, st, a, d)) != cudaSuccess) return e;
    if ((e = launch(true, k_adj_begin, g, kAdjThreads, 0, st, a, d)) != cudaSuccess) return e;
  }
  int cur = 0;
  for (int s = (int)d.I - 1; s >= 0; --s) {
    if ((e = launch(true, k_adj_iter, g, kAdjThreads, 0, st, a, d, (uint32_t)s, cur)) != cudaSuccess) return e;
    cur ^= 1;
  }
  if ((e = launch(true, k_adj_geom, g, kAdjThreads, 0, st, a, d, cur)) != cudaSuccess) return e;
  return launch(true, k_adj_tool, dim3(1), kToolThreads, 0, st, a, d, ctrl0, n_taped);
}

}  // namespace gg
