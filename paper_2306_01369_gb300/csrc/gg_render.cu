// gg_render.cu -- depth observations computed on the device (the paper's Sec. III-A
// "sky" and "ego" cameras): an orthographic height map of the particle surface and a
// perspective depth image of particles and rigid bodies.
//
// Particles are splatted: one thread per sphere visits the pixels its conservative
// footprint covers, tests each pixel exactly (FP32, fixed order) and folds its value
// into the pixel with an integer atomic max / min on the float's ordered bits, so the
// image does not depend on the order of the spheres.  Bodies are sphere traced per
// pixel (FP32, fixed order) and merged.  The decisions (coverage, ray-sphere hit,
// every tracing step) use the same operations in the same order as the oracle.
#include <cuda_runtime.h>

#include "gg_device.cuh"
#include "gg_internal.h"

namespace gg {

namespace {

// Order-preserving map of a float onto uint32 (for atomicMax over signed values);
// 0 is below every image of a float.
__device__ __forceinline__ uint32_t ordered(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_fill(uint32_t *img, uint32_t count, uint32_t v) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) img[p] = v;
}

__device__ __forceinline__ float pixel_centre(float base, uint32_t u, float step) {
  return __fadd_rn(base, __fmul_rn(__fadd_rn((float)u, 0.5f), step));
}

__global__ void k_splat_height(StepArgs a, uint32_t off, uint32_t n, RenderArgs c, uint32_t *img) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = a.pos_id[off + i];
  // conservative pixel range: |x - px| <= r with px = bx + (u + 1/2) sx
  const int u0 = max(0, (int)floorf((p.x - p.w - c.bx) / c.sx - 0.5f) - 1);
  const int u1 = min((int)c.W - 1, (int)ceilf((p.x + p.w - c.bx) / c.sx - 0.5f) + 1);
  const int v0 = max(0, (int)floorf((p.y - p.w - c.by) / c.sy - 0.5f) - 1);
  const int v1 = min((int)c.H - 1, (int)ceilf((p.y + p.w - c.by) / c.sy - 0.5f) + 1);
  const float r2 = __fmul_rn(p.w, p.w);
  for (int v = v0; v <= v1; ++v) {
    const float py = pixel_centre(c.by, (uint32_t)v, c.sy);
    const float dy = __fsub_rn(p.y, py);
    for (int u = u0; u <= u1; ++u) {
      const float px = pixel_centre(c.bx, (uint32_t)u, c.sx);
      const float dx = __fsub_rn(p.x, px);
      const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
      if (!(d2 <= r2)) continue;
      const float h = __fadd_rn(p.z, __fsqrt_rn(__fsub_rn(r2, d2)));
      atomicMax(&img[(size_t)v * c.W + u], ordered(h));
    }
  }
}

__global__ void k_finish_height(const uint32_t *img, uint32_t count, float empty, float *out) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) out[p] = img[p] ? from_ordered(img[p]) : empty;
}

// Unit ray of pixel (u, v) in the world frame, FP32 in the oracle's order.
__device__ __forceinline__ float3 pixel_ray(const RenderArgs &c, uint32_t u, uint32_t v) {
  const float ax = __fsub_rn(__fadd_rn((float)u, 0.5f), __fmul_rn(0.5f, (float)c.W));
  const float ay = __fsub_rn(__fadd_rn((float)v, 0.5f), __fmul_rn(0.5f, (float)c.H));
  const float dxc = __fdiv_rn(ax, c.f), dyc = __fdiv_rn(ay, c.f);
  const float s = __fadd_rn(__fadd_rn(__fmul_rn(dxc, dxc), __fmul_rn(dyc, dyc)), 1.0f);
  const float nr = __fsqrt_rn(s);
  const float dc[3] = {__fdiv_rn(dxc, nr), __fdiv_rn(dyc, nr), __fdiv_rn(1.0f, nr)};
  float d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    d[k] = __fadd_rn(__fadd_rn(__fmul_rn(c.R[3 * k], dc[0]), __fmul_rn(c.R[3 * k + 1], dc[1])),
                     __fmul_rn(c.R[3 * k + 2], dc[2]));
  return make_float3(d[0], d[1], d[2]);
}

// The ray of every pixel, once per image (the splat tests many spheres against each).
__global__ void k_make_rays(RenderArgs c) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.W * c.H) return;
  const float3 d = pixel_ray(c, p % c.W, p / c.W);
  c.rays[p] = make_float4(d.x, d.y, d.z, 0.f);
}

__global__ void k_splat_depth(StepArgs a, uint32_t off, uint32_t n, RenderArgs c, uint32_t *img) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = a.pos_id[off + i];
  const float oc0 = __fsub_rn(p.x, c.o[0]), oc1 = __fsub_rn(p.y, c.o[1]), oc2 = __fsub_rn(p.z, c.o[2]);
  const float rr = __fmul_rn(p.w, p.w);
  // conservative footprint from the centre in the camera frame (any rounding here
  // only widens or narrows the box by far less than the one-pixel margin)
  const float cx = c.R[0] * oc0 + c.R[3] * oc1 + c.R[6] * oc2;
  const float cy = c.R[1] * oc0 + c.R[4] * oc1 + c.R[7] * oc2;
  const float cz = c.R[2] * oc0 + c.R[5] * oc1 + c.R[8] * oc2;
  int u0 = 0, u1 = (int)c.W - 1, v0 = 0, v1 = (int)c.H - 1;
  if (cz - p.w > 0.5f * c.near) {
    const float zl = cz - p.w, zh = cz + p.w;
    const float xlo = fminf((cx - p.w) / zl, (cx - p.w) / zh), xhi = fmaxf((cx + p.w) / zl, (cx + p.w) / zh);
    const float ylo = fminf((cy - p.w) / zl, (cy - p.w) / zh), yhi = fmaxf((cy + p.w) / zl, (cy + p.w) / zh);
    u0 = max(u0, (int)floorf(c.f * xlo + 0.5f * c.W - 0.5f) - 1);
    u1 = min(u1, (int)ceilf(c.f * xhi + 0.5f * c.W - 0.5f) + 1);
    v0 = max(v0, (int)floorf(c.f * ylo + 0.5f * c.H - 0.5f) - 1);
    v1 = min(v1, (int)ceilf(c.f * yhi + 0.5f * c.H - 0.5f) + 1);
  } else if (cz + p.w <= 0.f) {
    return;  // entirely behind the camera
  }
  const float cc = __fsub_rn(__fadd_rn(__fadd_rn(__fmul_rn(oc0, oc0), __fmul_rn(oc1, oc1)), __fmul_rn(oc2, oc2)), rr);
  for (int v = v0; v <= v1; ++v)
    for (int u = u0; u <= u1; ++u) {
      const float4 d = c.rays[(size_t)v * c.W + u];
      const float b = __fadd_rn(__fadd_rn(__fmul_rn(d.x, oc0), __fmul_rn(d.y, oc1)), __fmul_rn(d.z, oc2));
      const float disc = __fsub_rn(__fmul_rn(b, b), cc);
      if (!(disc >= 0.0f)) continue;
      const float t0 = __fsub_rn(b, __fsqrt_rn(disc));
      if (!(t0 >= c.near && t0 <= c.far)) continue;
      atomicMin(&img[(size_t)v * c.W + u], __float_as_uint(t0));  // t0 > 0: bits order as floats
    }
}

// Distance used to step the tracing: the body's SDF; outside a GRID body's sampled box
// the distance to that box, at least eps.
__device__ __forceinline__ float march_sdf(const DevBody &b, float3 y, float eps) {
  int br;
  const float f = body_sdf(b, y, &br);
  if (b.kind != 4 || br >= 0) return f;
  const float yy[3] = {y.x, y.y, y.z};
  float q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float lo = b.shape[k];
    const float hi = __fadd_rn(b.shape[k], __fmul_rn(b.shape[3], (float)(b.gn[k] - 1u)));
    q[k] = fmaxf(fmaxf(__fsub_rn(lo, yy[k]), __fsub_rn(yy[k], hi)), 0.0f);
  }
  const float s = __fadd_rn(__fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1])), __fmul_rn(q[2], q[2]));
  return fmaxf(__fsqrt_rn(s), eps);
}

__global__ void k_trace_depth(StepArgs a, uint32_t gb0, uint32_t nb, RenderArgs c, const uint32_t *img, float *out) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.W * c.H) return;
  float best = __uint_as_float(img[p]);
  if (nb && c.mask) {
    const float4 d = c.rays[p];
    float t = c.near;
    for (uint32_t k = 0; k < c.steps; ++k) {
      const float3 x = make_float3(__fadd_rn(c.o[0], __fmul_rn(t, d.x)), __fadd_rn(c.o[1], __fmul_rn(t, d.y)),
                                   __fadd_rn(c.o[2], __fmul_rn(t, d.z)));
      float fmin = __int_as_float(0x7f800000);
      for (uint32_t b = 0; b < nb && b < 32u; ++b) {
        if (!((c.mask >> b) & 1u)) continue;
        const DevBody &B = a.bodies[gb0 + b];
        fmin = fminf(fmin, march_sdf(B, world_to_body(B, x), c.eps));
      }
      if (fmin < c.eps) {
        best = fminf(best, t);
        break;
      }
      t = __fadd_rn(t, fmin);
      if (!(t <= c.far)) break;
    }
  }
  out[p] = best <= c.far ? best : c.far;
}

inline unsigned cdiv(uint32_t a, unsigned b) { return a ? (a + b - 1) / b : 1; }

}  // namespace

cudaError_t enqueue_render(const StepArgs &a, uint32_t env_off, uint32_t env_n, uint32_t gb0, uint32_t nb,
                           const RenderArgs &c, uint32_t *img, float *out, cudaStream_t st) {
  const uint32_t np = c.W * c.H;
  if (c.kind == 0) {
    k_fill<<<cdiv(np, 256), 256, 0, st>>>(img, np, 0u);
    if (env_n) k_splat_height<<<cdiv(env_n, 128), 128, 0, st>>>(a, env_off, env_n, c, img);
    k_finish_height<<<cdiv(np, 256), 256, 0, st>>>(img, np, c.empty, out);
  } else {
    k_fill<<<cdiv(np, 256), 256, 0, st>>>(img, np, 0x7f800000u);
    k_make_rays<<<cdiv(np, 128), 128, 0, st>>>(c);
    if (env_n) k_splat_depth<<<cdiv(env_n, 128), 128, 0, st>>>(a, env_off, env_n, c, img);
    k_trace_depth<<<cdiv(np, 128), 128, 0, st>>>(a, gb0, nb, c, img, out);
  }
  return cudaGetLastError();
}

}  // namespace gg
