/*
 * gg_oracle.c -- plain, slow FP64 CPU oracle of the granular contact step.
 *
 * TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's
 * cpu_baseline leg).  Written from the paper's text, one stage per function, in
 * the paper's order: spatial hash (Eq. 6), bucket walk over the 27 neighbour
 * cells (Sec. II-B), sphere and SDF narrowphase (Sec. II-C, Eq. 7), projected
 * Jacobi (Alg. 1 with Eq. 1-3 and Baumgarte), symplectic Euler (Eq. 4-5).
 *
 * Readings of the paper where it is silent or garbled (each is repeated at the
 * code it governs):
 *  - Eq. 4-5: v+ = v + dt g + dv, x+ = x + dt v+ (dv is already a velocity change).
 *  - Alg. 1 relative velocity: both sides' current velocity estimates, gamma = 1.
 *  - Alg. 1 has no effective mass: mass splitting, w = 1 / (n_i/m_i + n_j/m_j),
 *    n_i = number of contacts of particle i (Tonge, Benevolenski & Voroshilov,
 *    ACM TOG 2012).  Its fixed point is the NCP of Eq. 1-3.
 *  - The clamp of Alg. 1 is applied to the accumulated impulse of each contact,
 *    so that it can decrease again; from zero the first iteration is Alg. 1's.
 *  - psi is the penetration depth (>= 0 in contact); Eq. 7's sign is flipped.
 *  - Buckets reached twice from one particle (two neighbour cells with the same
 *    hash) are walked once.
 *  - Coincident centres: normal = +z if id_i > id_j else -z.
 *  - Free rigid bodies (beyond the paper, whose bodies are kinematic): 6-DoF,
 *    gyroscopic term neglected, mass-split effective mass; box corners of a free
 *    body are tested as points against the non-free bodies.
 */
#include "gg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define HASH_P1 73856093u /* Eq. 6 constants */
#define HASH_P2 19349663u
#define HASH_P3 83492791u
#define HASH_Q 100u

/* ------------------------------------------------------------------------- */
/* FP32 decisions (no FMA: compile with -ffp-contract=off)                    */
/* ------------------------------------------------------------------------- */

float orc_inv_cell(float cell_size) { return (float)(1.0 / (double)cell_size); }

int32_t orc_cell_index(float x, float inv_cell) {
  float t = x * inv_cell;
  t = t + 0.5f;
  return (int32_t)floorf(t);
}

uint32_t orc_hash(int32_t k0, int32_t k1, int32_t k2, uint32_t n_h) {
  uint32_t a = ((uint32_t)k0 - HASH_Q) * HASH_P1;
  uint32_t b = ((uint32_t)k1 - HASH_Q) * HASH_P2;
  uint32_t c = ((uint32_t)k2 - HASH_Q) * HASH_P3;
  return (a ^ b ^ c) % n_h;
}

/* Sphere test ||x_i - x_j||^2 <= (r_i + r_j)^2 (Sec. II-C) in FP32, fixed order. */
static int pp_hit_f32(const float *xi, float ri, const float *xj, float rj) {
  float dx = xi[0] - xj[0];
  float dy = xi[1] - xj[1];
  float dz = xi[2] - xj[2];
  float d2 = dx * dx;
  float t = dy * dy;
  d2 = d2 + t;
  t = dz * dz;
  d2 = d2 + t;
  float rs = ri + rj;
  float rs2 = rs * rs;
  return d2 <= rs2;
}

typedef struct {
  int32_t kind;
  float s[12];
  float p[3];
  float R[9]; /* row-major, body -> world */
  const float *grid;
  uint32_t gn[3];
} bodyf;

static void rot_f32(const float *q, float *R) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
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

static void body_to_f32(const orc_body *b, bodyf *o) {
  float q[4];
  o->kind = b->kind;
  for (int k = 0; k < 12; ++k) o->s[k] = (float)b->shape[k];
  for (int k = 0; k < 3; ++k) o->p[k] = (float)b->pos[k];
  for (int k = 0; k < 4; ++k) q[k] = (float)b->quat[k];
  rot_f32(q, o->R);
  o->grid = b->grid;
  for (int k = 0; k < 3; ++k) o->gn[k] = b->grid_dims[k];
}

/* y = R^T (x - p), each row summed left to right. */
static void to_body_f32(const bodyf *b, const float *x, float *y) {
  float d0 = x[0] - b->p[0], d1 = x[1] - b->p[1], d2 = x[2] - b->p[2];
  for (int k = 0; k < 3; ++k) {
    float a = b->R[0 + k] * d0;
    float c = b->R[3 + k] * d1;
    a = a + c;
    c = b->R[6 + k] * d2;
    y[k] = a + c;
  }
}

/* Box SDF in FP32; branch 0..2 = inside, nearest face on that axis; 3 = outside. */
static float box_f32(const float *y, const float *h, int *branch) {
  float q0 = fabsf(y[0]) - h[0];
  float q1 = fabsf(y[1]) - h[1];
  float q2 = fabsf(y[2]) - h[2];
  float m0 = fmaxf(q0, 0.0f), m1 = fmaxf(q1, 0.0f), m2 = fmaxf(q2, 0.0f);
  float s = m0 * m0;
  float t = m1 * m1;
  s = s + t;
  t = m2 * m2;
  s = s + t;
  float o = sqrtf(s);
  float mx = fmaxf(fmaxf(q0, q1), q2);
  float f = o + fminf(mx, 0.0f);
  if (mx > 0.0f)
    *branch = 3;
  else if (q0 >= q1 && q0 >= q2)
    *branch = 0;
  else if (q1 >= q2)
    *branch = 1;
  else
    *branch = 2;
  return f;
}

/* Gridded SDF (Sec. II-C): trilinear interpolation of the samples around y.
 * FP32, in this order: u_k = (y_k - o_k) * float(1/h); cell i_k = floor(u_k), at most
 * n_k - 2; t_k = u_k - i_k; lerp(a, b, t) = a + t (b - a) along x (4 edges), then y,
 * then z.  Outside the sampled box [0, n_k - 1] (or NaN): no contact (+inf), branch -1;
 * inside, the branch is the cell's linear index. */
static float lerp_f32(float a, float b, float t) {
  float d = b - a;
  float m = t * d;
  return a + m;
}

static float grid_f32(const bodyf *b, const float *y, int *branch) {
  const float ih = (float)(1.0 / (double)b->s[3]);
  int32_t i[3];
  float t[3];
  for (int k = 0; k < 3; ++k) {
    float d = y[k] - b->s[k];
    float u = d * ih;
    float top = (float)(b->gn[k] - 1);
    if (!(u >= 0.0f && u <= top)) {
      *branch = -1;
      return INFINITY;
    }
    int32_t c = (int32_t)floorf(u);
    if (c > (int32_t)b->gn[k] - 2) c = (int32_t)b->gn[k] - 2;
    i[k] = c;
    t[k] = u - (float)c;
  }
  const size_t nx = b->gn[0], nxy = (size_t)b->gn[0] * b->gn[1];
  const float *v = b->grid + (size_t)i[2] * nxy + (size_t)i[1] * nx + (size_t)i[0];
  float c00 = lerp_f32(v[0], v[1], t[0]);
  float c10 = lerp_f32(v[nx], v[nx + 1], t[0]);
  float c01 = lerp_f32(v[nxy], v[nxy + 1], t[0]);
  float c11 = lerp_f32(v[nxy + nx], v[nxy + nx + 1], t[0]);
  float c0 = lerp_f32(c00, c10, t[1]);
  float c1 = lerp_f32(c01, c11, t[1]);
  *branch = (int)((size_t)i[2] * nxy + (size_t)i[1] * nx + (size_t)i[0]);
  return lerp_f32(c0, c1, t[2]);
}

/* SDF of body b at body-frame point y, FP32, with the active branch. */
static float sdf_f32(const bodyf *b, const float *y, int *branch) {
  switch (b->kind) {
  case ORC_PLANE:
    *branch = 0;
    return y[2];
  case ORC_BOX:
    return box_f32(y, b->s, branch);
  case ORC_BOX_MINUS_BOX: {
    int ba, bb;
    float fa = box_f32(y, b->s, &ba);
    float z[3] = {y[0] - b->s[6], y[1] - b->s[7], y[2] - b->s[8]};
    float fb = box_f32(z, b->s + 3, &bb);
    float nfb = -fb;
    if (fa >= nfb) {
      *branch = ba;
      return fa;
    }
    *branch = 4 + bb;
    return nfb;
  }
  case ORC_OPEN_BOX: {
    float w[5];
    w[0] = b->s[0] - y[0];
    w[1] = y[0] + b->s[0];
    w[2] = b->s[1] - y[1];
    w[3] = y[1] + b->s[1];
    w[4] = y[2] + b->s[2];
    float f = w[0];
    int br = 0;
    for (int k = 1; k < 5; ++k)
      if (w[k] < f) {
        f = w[k];
        br = k;
      }
    *branch = br;
    return f;
  }
  case ORC_GRID:
    return grid_f32(b, y, branch);
  case ORC_TUBE: { /* inside of a vertical cylinder of radius s[0]: f = R - |(y0, y1)| */
    float q = y[0] * y[0];
    float t = y[1] * y[1];
    q = q + t;
    *branch = 0;
    return b->s[0] - sqrtf(q);
  }
  default:
    *branch = -1;
    return INFINITY;
  }
}

/* ------------------------------------------------------------------------- */
/* FP64 geometry                                                              */
/* ------------------------------------------------------------------------- */

static void rot64(const double *qin, double *R) {
  double nq = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  double w = qin[0] / nq, x = qin[1] / nq, y = qin[2] / nq, z = qin[3] / nq;
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static double sgn1(double v) { return v < 0 ? -1.0 : 1.0; }

/* Box SDF value and unit gradient of the branch chosen in FP32. */
static double box64(const double *y, const double *h, int branch, double *g) {
  double q[3] = {fabs(y[0]) - h[0], fabs(y[1]) - h[1], fabs(y[2]) - h[2]};
  g[0] = g[1] = g[2] = 0;
  if (branch == 3) {
    double m[3] = {q[0] > 0 ? q[0] : 0, q[1] > 0 ? q[1] : 0, q[2] > 0 ? q[2] : 0};
    double o = sqrt(dot3(m, m));
    if (o > 0) {
      for (int k = 0; k < 3; ++k) g[k] = m[k] * sgn1(y[k]) / o;
      return o;
    }
    /* FP64 sees the point on the surface: use the face of the largest q */
    branch = (q[0] >= q[1] && q[0] >= q[2]) ? 0 : (q[1] >= q[2] ? 1 : 2);
  }
  g[branch] = sgn1(y[branch]);
  return q[branch];
}

/* Gridded SDF in FP64 on the cell chosen in FP32: the trilinear interpolant of that
 * cell's eight samples, sum over corners v_abc w_a(t_x) w_b(t_y) w_c(t_z) with
 * w_0(t) = 1 - t, w_1(t) = t, t_k = (y_k - o_k) / h - i_k, and its unit gradient
 * (d f / d y_k = (1/h) d f / d t_k); a zero gradient gives +z. */
static double grid64(const orc_body *b, const double *y, int cell, double *g) {
  const uint32_t nx = b->grid_dims[0], ny = b->grid_dims[1];
  const size_t nxy = (size_t)nx * ny;
  const int32_t i[3] = {(int32_t)((size_t)cell % nx), (int32_t)(((size_t)cell / nx) % ny), (int32_t)((size_t)cell / nxy)};
  const double h = (double)(float)b->shape[3];
  double t[3], w[3][2], dw[2] = {-1.0, 1.0};
  for (int k = 0; k < 3; ++k) {
    t[k] = (y[k] - (double)(float)b->shape[k]) / h - (double)i[k];
    w[k][0] = 1.0 - t[k];
    w[k][1] = t[k];
  }
  const float *v = b->grid + (size_t)cell;
  double f = 0.0, df[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < 2; ++c)
    for (int bb = 0; bb < 2; ++bb)
      for (int a = 0; a < 2; ++a) {
        const double s = (double)v[(size_t)c * nxy + (size_t)bb * nx + (size_t)a];
        f += s * w[0][a] * w[1][bb] * w[2][c];
        df[0] += s * dw[a] * w[1][bb] * w[2][c];
        df[1] += s * w[0][a] * dw[bb] * w[2][c];
        df[2] += s * w[0][a] * w[1][bb] * dw[c];
      }
  const double gn = sqrt(dot3(df, df));
  if (gn > 0.0) {
    for (int k = 0; k < 3; ++k) g[k] = df[k] / gn;
  } else {
    g[0] = 0.0;
    g[1] = 0.0;
    g[2] = 1.0;
  }
  return f;
}

static double sdf64_branch(const orc_body *b, const double *y, int branch, double *g) {
  switch (b->kind) {
  case ORC_PLANE:
    g[0] = 0;
    g[1] = 0;
    g[2] = 1;
    return y[2];
  case ORC_BOX:
    return box64(y, b->shape, branch, g);
  case ORC_BOX_MINUS_BOX:
    if (branch < 4) return box64(y, b->shape, branch, g);
    {
      double z[3] = {y[0] - b->shape[6], y[1] - b->shape[7], y[2] - b->shape[8]};
      double f = box64(z, b->shape + 3, branch - 4, g);
      g[0] = -g[0];
      g[1] = -g[1];
      g[2] = -g[2];
      return -f;
    }
  case ORC_OPEN_BOX: {
    static const double gn[5][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, 1}};
    double w[5] = {b->shape[0] - y[0], y[0] + b->shape[0], b->shape[1] - y[1], y[1] + b->shape[1],
                   y[2] + b->shape[2]};
    for (int k = 0; k < 3; ++k) g[k] = gn[branch][k];
    return w[branch];
  }
  case ORC_GRID:
    if (branch >= 0) return grid64(b, y, branch, g);
    break;
  case ORC_TUBE: {
    const double rho = sqrt(y[0] * y[0] + y[1] * y[1]);
    if (rho > 0) {
      g[0] = -y[0] / rho;
      g[1] = -y[1] / rho;
    } else {
      g[0] = -1.0;
      g[1] = 0.0;
    }
    g[2] = 0.0;
    return b->shape[0] - rho;
  }
  }
  g[0] = g[1] = g[2] = 0;
  return INFINITY;
}

/* FP64 branch choice, for orc_sdf (no FP32 decision involved). */
static int branch64(const orc_body *b, const double *y) {
  float yf[3] = {(float)y[0], (float)y[1], (float)y[2]};
  bodyf bf;
  int br;
  body_to_f32(b, &bf);
  (void)sdf_f32(&bf, yf, &br);
  return br;
}

static void world_to_body64(const orc_body *b, const double *R, const double *x, double *y) {
  double d[3] = {x[0] - b->pos[0], x[1] - b->pos[1], x[2] - b->pos[2]};
  for (int k = 0; k < 3; ++k) y[k] = R[0 + k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];
}

static void body_to_world_vec64(const double *R, const double *g, double *n) {
  for (int a = 0; a < 3; ++a) n[a] = R[3 * a + 0] * g[0] + R[3 * a + 1] * g[1] + R[3 * a + 2] * g[2];
}

double orc_sdf(const orc_body *b, const double *xw, double *normal_world) {
  double R[9], y[3], g[3];
  rot64(b->quat, R);
  world_to_body64(b, R, xw, y);
  int br = branch64(b, y);
  double f = sdf64_branch(b, y, br, g);
  if (normal_world) body_to_world_vec64(R, g, normal_world);
  return f;
}

/* ------------------------------------------------------------------------- */
/* Binning (Eq. 6) and the sorted bucket table                                */
/* ------------------------------------------------------------------------- */

void orc_cell_keys(uint32_t n, const double *x, float inv_cell, uint32_t n_h, uint32_t *keys) {
  for (uint32_t i = 0; i < n; ++i) {
    int32_t k0 = orc_cell_index((float)x[3 * i + 0], inv_cell);
    int32_t k1 = orc_cell_index((float)x[3 * i + 1], inv_cell);
    int32_t k2 = orc_cell_index((float)x[3 * i + 2], inv_cell);
    keys[i] = orc_hash(k0, k1, k2, n_h);
  }
}

typedef struct {
  uint32_t key, id;
} keyid;

static int cmp_keyid(const void *a, const void *b) {
  const keyid *x = (const keyid *)a, *y = (const keyid *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}

void orc_sort_perm(uint32_t n, const uint32_t *keys, uint32_t *perm) {
  keyid *a = (keyid *)malloc(sizeof(keyid) * (n ? n : 1));
  for (uint32_t i = 0; i < n; ++i) {
    a[i].key = keys[i];
    a[i].id = i;
  }
  qsort(a, n, sizeof(keyid), cmp_keyid);
  for (uint32_t i = 0; i < n; ++i) perm[i] = a[i].id;
  free(a);
}

/* ------------------------------------------------------------------------- */
/* Contacts                                                                   */
/* ------------------------------------------------------------------------- */

#define MAX_FOUND 256

typedef struct {
  uint32_t n, nb;
  uint32_t *pp_off, *pp_j;
  double *pp_n, *pp_psi;
  uint32_t *bc_off, *bc_b;
  double *bc_n, *bc_psi, *bc_xc;
  /* free-box corners against non-free bodies */
  uint32_t n_cc;
  uint32_t *cc_b, *cc_o;
  double *cc_n, *cc_psi, *cc_xc;
} contacts;

static void contacts_free(contacts *C) {
  free(C->pp_off);
  free(C->pp_j);
  free(C->pp_n);
  free(C->pp_psi);
  free(C->bc_off);
  free(C->bc_b);
  free(C->bc_n);
  free(C->bc_psi);
  free(C->bc_xc);
  free(C->cc_b);
  free(C->cc_o);
  free(C->cc_n);
  free(C->cc_psi);
  free(C->cc_xc);
  memset(C, 0, sizeof(*C));
}

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

typedef struct {
  const orc_params *p;
  uint32_t n;
  const float *xf, *rf;
  float inv_cell;
  uint32_t n_h;
  const uint32_t *perm, *start;
  int brute;
} search_ctx;

/* Partners of particle i, ascending by id.  Returns the count (or -1 on overflow). */
static int find_partners(const search_ctx *s, uint32_t i, uint32_t *found) {
  int cnt = 0;
  const float *xi = s->xf + 3 * i;
  float ri = s->rf[i];
  if (s->brute) {
    for (uint32_t j = 0; j < s->n; ++j) {
      if (j == i) continue;
      if (pp_hit_f32(xi, ri, s->xf + 3 * j, s->rf[j])) {
        if (cnt == MAX_FOUND) return -1;
        found[cnt++] = j;
      }
    }
    return cnt;
  }
  int32_t k0 = orc_cell_index(xi[0], s->inv_cell);
  int32_t k1 = orc_cell_index(xi[1], s->inv_cell);
  int32_t k2 = orc_cell_index(xi[2], s->inv_cell);
  uint32_t seen[27];
  int n_seen = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        uint32_t h = orc_hash(k0 + dx, k1 + dy, k2 + dz, s->n_h);
        int dup = 0;
        for (int q = 0; q < n_seen; ++q)
          if (seen[q] == h) dup = 1;
        if (dup) continue; /* reading: a bucket reached twice is walked once */
        seen[n_seen++] = h;
        for (uint32_t t = s->start[h]; t < s->start[h + 1]; ++t) {
          uint32_t j = s->perm[t];
          if (j == i) continue;
          if (pp_hit_f32(xi, ri, s->xf + 3 * j, s->rf[j])) {
            if (cnt == MAX_FOUND) return -1;
            found[cnt++] = j;
          }
        }
      }
  qsort(found, cnt, sizeof(uint32_t), cmp_u32);
  return cnt;
}

/* Particle-body test in FP32 (Eq. 7: contact iff f(y) <= r), FP64 geometry. */
static int body_hit(const orc_body *B, const bodyf *bf, const double *R, const double *x, double r,
                    const float *xf, float rf, double *nrm, double *psi, double *xc) {
  float yf[3];
  int br;
  to_body_f32(bf, xf, yf);
  float f32 = sdf_f32(bf, yf, &br);
  if (!(f32 <= rf)) return 0;
  double y[3], g[3];
  world_to_body64(B, R, x, y);
  double f = sdf64_branch(B, y, br, g);
  body_to_world_vec64(R, g, nrm);
  *psi = r - f; /* reading: psi = penetration depth, positive in contact */
  for (int k = 0; k < 3; ++k) xc[k] = x[k] - f * nrm[k];
  return 1;
}

static int build_contacts(const orc_params *p, uint32_t n, const double *x, const double *r,
                          uint32_t nb, const orc_body *bodies, int brute, contacts *C) {
  memset(C, 0, sizeof(*C));
  C->n = n;
  C->nb = nb;
  float *xf = (float *)malloc(sizeof(float) * 3 * (n ? n : 1));
  float *rf = (float *)malloc(sizeof(float) * (n ? n : 1));
  for (uint32_t i = 0; i < 3 * n; ++i) xf[i] = (float)x[i];
  for (uint32_t i = 0; i < n; ++i) rf[i] = (float)r[i];
  search_ctx s;
  s.p = p;
  s.n = n;
  s.xf = xf;
  s.rf = rf;
  s.inv_cell = orc_inv_cell(p->cell_size);
  s.n_h = p->hash_size;
  s.brute = brute;
  uint32_t *keys = NULL, *perm = NULL, *start = NULL;
  if (!brute) {
    keys = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    perm = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    start = (uint32_t *)calloc((size_t)p->hash_size + 1, sizeof(uint32_t));
    orc_cell_keys(n, x, s.inv_cell, p->hash_size, keys);
    orc_sort_perm(n, keys, perm);
    for (uint32_t i = 0; i < n; ++i) start[keys[i] + 1]++;
    for (uint32_t h = 0; h < p->hash_size; ++h) start[h + 1] += start[h];
  }
  s.perm = perm;
  s.start = start;

  bodyf *bf = (bodyf *)malloc(sizeof(bodyf) * (nb ? nb : 1));
  double *Rb = (double *)malloc(sizeof(double) * 9 * (nb ? nb : 1));
  for (uint32_t b = 0; b < nb; ++b) {
    body_to_f32(&bodies[b], &bf[b]);
    rot64(bodies[b].quat, Rb + 9 * b);
  }

  int err = 0;
  C->pp_off = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
  C->bc_off = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
  /* pass 1: counts */
#pragma omp parallel for num_threads(p->n_threads > 0 ? p->n_threads : 1) schedule(dynamic, 256)
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t found[MAX_FOUND];
    int c = find_partners(&s, i, found);
    if (c < 0) {
#pragma omp atomic write
      err = 1;
      c = 0;
    }
    C->pp_off[i + 1] = (uint32_t)c;
    uint32_t nbc = 0;
    for (uint32_t b = 0; b < nb; ++b) {
      double nrm[3], psi, xc[3];
      if (body_hit(&bodies[b], &bf[b], Rb + 9 * b, x + 3 * i, r[i], xf + 3 * i, rf[i], nrm, &psi, xc)) ++nbc;
    }
    C->bc_off[i + 1] = nbc;
  }
  for (uint32_t i = 0; i < n; ++i) {
    C->pp_off[i + 1] += C->pp_off[i];
    C->bc_off[i + 1] += C->bc_off[i];
  }
  size_t npp = C->pp_off[n], nbc = C->bc_off[n];
  C->pp_j = (uint32_t *)malloc(sizeof(uint32_t) * (npp ? npp : 1));
  C->pp_n = (double *)malloc(sizeof(double) * 3 * (npp ? npp : 1));
  C->pp_psi = (double *)malloc(sizeof(double) * (npp ? npp : 1));
  C->bc_b = (uint32_t *)malloc(sizeof(uint32_t) * (nbc ? nbc : 1));
  C->bc_n = (double *)malloc(sizeof(double) * 3 * (nbc ? nbc : 1));
  C->bc_psi = (double *)malloc(sizeof(double) * (nbc ? nbc : 1));
  C->bc_xc = (double *)malloc(sizeof(double) * 3 * (nbc ? nbc : 1));
  /* pass 2: fill */
#pragma omp parallel for num_threads(p->n_threads > 0 ? p->n_threads : 1) schedule(dynamic, 256)
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t found[MAX_FOUND];
    int c = find_partners(&s, i, found);
    if (c < 0) c = 0;
    uint32_t o = C->pp_off[i];
    for (int q = 0; q < c; ++q) {
      uint32_t j = found[q];
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      double dist = sqrt(dot3(d, d));
      double *nn = C->pp_n + 3 * (o + q);
      if (dist > 0) {
        for (int k = 0; k < 3; ++k) nn[k] = d[k] / dist;
      } else { /* reading: coincident centres get an antisymmetric vertical normal */
        nn[0] = 0;
        nn[1] = 0;
        nn[2] = (i > j) ? 1.0 : -1.0;
      }
      C->pp_j[o + q] = j;
      C->pp_psi[o + q] = r[i] + r[j] - dist;
    }
    uint32_t ob = C->bc_off[i];
    for (uint32_t b = 0; b < nb; ++b) {
      double nrm[3], psi, xc[3];
      if (body_hit(&bodies[b], &bf[b], Rb + 9 * b, x + 3 * i, r[i], xf + 3 * i, rf[i], nrm, &psi, xc)) {
        C->bc_b[ob] = b;
        for (int k = 0; k < 3; ++k) {
          C->bc_n[3 * ob + k] = nrm[k];
          C->bc_xc[3 * ob + k] = xc[k];
        }
        C->bc_psi[ob] = psi;
        ++ob;
      }
    }
  }
  /* corners of free boxes against every non-free body (reading for free bodies) */
  {
    uint32_t cap = 0;
    for (uint32_t b = 0; b < nb; ++b)
      if (bodies[b].is_free && bodies[b].kind == ORC_BOX) cap += 8 * nb;
    C->cc_b = (uint32_t *)malloc(sizeof(uint32_t) * (cap ? cap : 1));
    C->cc_o = (uint32_t *)malloc(sizeof(uint32_t) * (cap ? cap : 1));
    C->cc_n = (double *)malloc(sizeof(double) * 3 * (cap ? cap : 1));
    C->cc_psi = (double *)malloc(sizeof(double) * (cap ? cap : 1));
    C->cc_xc = (double *)malloc(sizeof(double) * 3 * (cap ? cap : 1));
    uint32_t m = 0;
    for (uint32_t b = 0; b < nb; ++b) {
      if (!(bodies[b].is_free && bodies[b].kind == ORC_BOX)) continue;
      for (int k = 0; k < 8; ++k) {
        float cf[3], wf[3];
        double c[3], w[3];
        for (int a = 0; a < 3; ++a) {
          double sg = ((k >> a) & 1) ? 1.0 : -1.0;
          c[a] = sg * bodies[b].shape[a];
          cf[a] = (float)sg * bf[b].s[a];
        }
        for (int a = 0; a < 3; ++a) { /* corner in world: p + R c, FP32 fixed order */
          float t = bf[b].R[3 * a + 0] * cf[0];
          float u = bf[b].R[3 * a + 1] * cf[1];
          t = t + u;
          u = bf[b].R[3 * a + 2] * cf[2];
          t = t + u;
          wf[a] = bf[b].p[a] + t;
        }
        body_to_world_vec64(Rb + 9 * b, c, w);
        for (int a = 0; a < 3; ++a) w[a] += bodies[b].pos[a];
        for (uint32_t o = 0; o < nb; ++o) {
          if (o == b || bodies[o].is_free) continue;
          double nrm[3], psi, xc[3];
          if (body_hit(&bodies[o], &bf[o], Rb + 9 * o, w, 0.0, wf, 0.0f, nrm, &psi, xc)) {
            C->cc_b[m] = b;
            C->cc_o[m] = o;
            for (int a = 0; a < 3; ++a) {
              C->cc_n[3 * m + a] = nrm[a];
              C->cc_xc[3 * m + a] = xc[a];
            }
            C->cc_psi[m] = psi;
            ++m;
          }
        }
      }
    }
    C->n_cc = m;
  }
  free(xf);
  free(rf);
  free(keys);
  free(perm);
  free(start);
  free(bf);
  free(Rb);
  return err ? -1 : 0;
}

static void fill_stats(const contacts *C, orc_stats *st) {
  if (!st) return;
  st->n_pp = C->pp_off[C->n];
  st->n_body = C->bc_off[C->n];
  st->n_corner = C->n_cc;
  st->max_pp = 0;
  st->max_body = 0;
  st->max_psi = 0;
  for (uint32_t i = 0; i < C->n; ++i) {
    int a = (int)(C->pp_off[i + 1] - C->pp_off[i]);
    int b = (int)(C->bc_off[i + 1] - C->bc_off[i]);
    if (a > st->max_pp) st->max_pp = a;
    if (b > st->max_body) st->max_body = b;
  }
  for (uint32_t c = 0; c < C->pp_off[C->n]; ++c)
    if (C->pp_psi[c] > st->max_psi) st->max_psi = C->pp_psi[c];
  for (uint32_t c = 0; c < C->bc_off[C->n]; ++c)
    if (C->bc_psi[c] > st->max_psi) st->max_psi = C->bc_psi[c];
}

int orc_contacts(const orc_params *p, uint32_t n, const double *x, const double *r, uint32_t n_bodies,
                 const orc_body *bodies, int brute, uint32_t *pp_off, uint32_t *pp_j, double *pp_geom,
                 uint32_t *bc_off, uint32_t *bc_b, double *bc_geom, orc_stats *st) {
  contacts C;
  int rc = build_contacts(p, n, x, r, n_bodies, bodies, brute, &C);
  if (rc == 0) {
    uint32_t npp = C.pp_off[n], nbc = C.bc_off[n];
    if (pp_off) memcpy(pp_off, C.pp_off, sizeof(uint32_t) * (n + 1));
    if (pp_j) memcpy(pp_j, C.pp_j, sizeof(uint32_t) * npp);
    if (pp_geom)
      for (uint32_t c = 0; c < npp; ++c) {
        for (int k = 0; k < 3; ++k) pp_geom[4 * c + k] = C.pp_n[3 * c + k];
        pp_geom[4 * c + 3] = C.pp_psi[c];
      }
    if (bc_off) memcpy(bc_off, C.bc_off, sizeof(uint32_t) * (n + 1));
    if (bc_b) memcpy(bc_b, C.bc_b, sizeof(uint32_t) * nbc);
    if (bc_geom)
      for (uint32_t c = 0; c < nbc; ++c) {
        for (int k = 0; k < 3; ++k) bc_geom[7 * c + k] = C.bc_n[3 * c + k];
        bc_geom[7 * c + 3] = C.bc_psi[c];
        for (int k = 0; k < 3; ++k) bc_geom[7 * c + 4 + k] = C.bc_xc[3 * c + k];
      }
    fill_stats(&C, st);
  }
  contacts_free(&C);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Projected Jacobi (Alg. 1) and symplectic Euler (Eq. 4-5)                   */
/* ------------------------------------------------------------------------- */

/*
 * One contact update.  lam is the accumulated impulse on the first side, u the
 * relative velocity of the first side w.r.t. the second, nrm the unit normal
 * from the second side into the first, bias = alpha psi / dt (Baumgarte), w the
 * mass-split effective mass.  Target relative velocity: bias along nrm, zero
 * tangentially; then the normal part is kept non-negative (Eq. 2) and the
 * tangential part is scaled onto the cone of Eq. 3 (Alg. 1's projection).
 */
static void pja_update(double *lam, const double *u, const double *nrm, double bias, double w, double mu) {
  double s[3];
  for (int k = 0; k < 3; ++k) s[k] = lam[k] - w * (u[k] - bias * nrm[k]);
  double ln = dot3(s, nrm);
  double lnp = ln > 0 ? ln : 0;
  double t[3];
  for (int k = 0; k < 3; ++k) t[k] = s[k] - ln * nrm[k];
  double tn = sqrt(dot3(t, t));
  if (tn > mu * lnp) {
    double sc = mu * lnp / tn;
    for (int k = 0; k < 3; ++k) t[k] *= sc;
  }
  for (int k = 0; k < 3; ++k) lam[k] = lnp * nrm[k] + t[k];
}

/* I_w^{-1} a with I_w = R diag(I) R^T */
static void inv_inertia_world(const double *R, const double *I, const double *a, double *out) {
  double b[3];
  for (int k = 0; k < 3; ++k) b[k] = (R[0 + k] * a[0] + R[3 + k] * a[1] + R[6 + k] * a[2]) / I[k];
  body_to_world_vec64(R, b, out);
}

/* 1/M + (a x n) . I_w^{-1} (a x n): inverse effective mass of a free body along n at arm a */
static double free_inv_mass(const orc_body *B, const double *R, const double *a, const double *nrm) {
  double an[3], t[3];
  cross3(a, nrm, an);
  inv_inertia_world(R, B->inertia, an, t);
  return 1.0 / B->mass + dot3(an, t);
}

static void point_vel(const double *V, const double *W, const double *p, const double *xc, double *u) {
  double a[3] = {xc[0] - p[0], xc[1] - p[1], xc[2] - p[2]}, c[3];
  cross3(W, a, c);
  for (int k = 0; k < 3; ++k) u[k] = V[k] + c[k];
}

/*
 * Residual of one contact at a fixed point of the iteration, in velocity units:
 * complementarity of Eq. 2 with the Baumgarte target (|min(lambda_n/m, u_n - bias)|),
 * the cone of Eq. 3 (excess of |lambda_t| over mu lambda_n), and for a pressed
 * contact either no slip (inside the cone) or slip opposite to the friction
 * impulse (on the cone).
 */
static double contact_residual(const double *lam, const double *u, const double *nrm, double bias, double mi,
                               double mu) {
  double ln = dot3(lam, nrm), un = dot3(u, nrm);
  double lt[3], ut[3];
  for (int k = 0; k < 3; ++k) {
    lt[k] = (lam[k] - ln * nrm[k]) / mi;
    ut[k] = u[k] - un * nrm[k];
  }
  double lnv = ln / mi, unb = un - bias;
  double r1 = fabs(lnv < unb ? lnv : unb);
  double ltn = sqrt(dot3(lt, lt));
  double r2 = ltn - mu * lnv;
  if (r2 < 0) r2 = 0;
  double r3;
  if (lnv <= 0) {
    r3 = 0; /* separated contact: tangential velocity is free (r2 bounds the friction impulse) */
  } else if (ltn < mu * lnv * (1 - 1e-9)) {
    r3 = sqrt(dot3(ut, ut));
  } else {
    double utn = sqrt(dot3(ut, ut)), e[3];
    for (int k = 0; k < 3; ++k) e[k] = ut[k] + (ltn > 0 ? utn * lt[k] / ltn : 0);
    r3 = sqrt(dot3(e, e));
  }
  double rr = r1 > r2 ? r1 : r2;
  return r3 > rr ? r3 : rr;
}

static void quat_integrate(double *q, const double *w, double dt) {
  double th[3] = {w[0] * dt, w[1] * dt, w[2] * dt};
  double ang = sqrt(dot3(th, th));
  if (ang == 0) return;
  double s = sin(0.5 * ang) / ang, c = cos(0.5 * ang);
  double d[4] = {c, th[0] * s, th[1] * s, th[2] * s};
  double r[4];
  r[0] = d[0] * q[0] - d[1] * q[1] - d[2] * q[2] - d[3] * q[3];
  r[1] = d[0] * q[1] + d[1] * q[0] + d[2] * q[3] - d[3] * q[2];
  r[2] = d[0] * q[2] - d[1] * q[3] + d[2] * q[0] + d[3] * q[1];
  r[3] = d[0] * q[3] + d[1] * q[2] - d[2] * q[1] + d[3] * q[0];
  double nq = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
  for (int k = 0; k < 4; ++k) q[k] = r[k] / nq;
}

int orc_step(const orc_params *p, uint32_t n, double *x, double *v, const double *r, const double *m,
             uint32_t nb, orc_body *bodies, const double *twist, double *wrench, double *pp_lam,
             double *bc_lam, orc_stats *st) {
  if (p->pja_weight)
    for (uint32_t b = 0; b < nb; ++b)
      if (bodies[b].is_free) return -2;
  contacts C;
  if (build_contacts(p, n, x, r, nb, bodies, 0, &C) != 0) {
    contacts_free(&C);
    return -1;
  }
  const double dt = p->dt, mu = p->mu, ab = p->alpha / p->dt;
  const double *g = p->gravity;
  uint32_t npp = C.pp_off[n], nbc = C.bc_off[n], ncc = C.n_cc;
  int nthr = p->n_threads > 0 ? p->n_threads : 1;

  double *Rb = (double *)malloc(sizeof(double) * 9 * (nb ? nb : 1));
  double *Vb = (double *)malloc(sizeof(double) * 6 * (nb ? nb : 1)); /* current body twists (V, W) */
  double *Vn = (double *)malloc(sizeof(double) * 6 * (nb ? nb : 1));
  double *base_b = (double *)malloc(sizeof(double) * 6 * (nb ? nb : 1));
  uint32_t *ncb = (uint32_t *)calloc(nb ? nb : 1, sizeof(uint32_t));
  for (uint32_t b = 0; b < nb; ++b) {
    rot64(bodies[b].quat, Rb + 9 * b);
    const double *tv = bodies[b].lin_vel, *tw = bodies[b].ang_vel;
    if (!bodies[b].is_free && twist) {
      tv = twist + 6 * b;
      tw = twist + 6 * b + 3;
    }
    for (int k = 0; k < 3; ++k) {
      base_b[6 * b + k] = tv[k] + (bodies[b].is_free ? dt * g[k] : 0.0);
      base_b[6 * b + 3 + k] = tw[k];
    }
    memcpy(Vb + 6 * b, base_b + 6 * b, sizeof(double) * 6);
  }
  for (uint32_t c = 0; c < nbc; ++c) ncb[C.bc_b[c]]++;
  for (uint32_t c = 0; c < ncc; ++c) ncb[C.cc_b[c]]++;

  double *base = (double *)malloc(sizeof(double) * 3 * (n ? n : 1)); /* v + dt g */
  double *U = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
  double *Un = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
  double *lp = (double *)calloc(3 * (size_t)(npp ? npp : 1), sizeof(double));
  double *lb = (double *)calloc(3 * (size_t)(nbc ? nbc : 1), sizeof(double));
  double *lc = (double *)calloc(3 * (size_t)(ncc ? ncc : 1), sizeof(double));
  double *nci = (double *)malloc(sizeof(double) * (n ? n : 1)); /* n_i / m_i */
  for (uint32_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) base[3 * i + k] = v[3 * i + k] + dt * g[k];
    memcpy(U + 3 * i, base + 3 * i, sizeof(double) * 3);
    uint32_t cnt = (C.pp_off[i + 1] - C.pp_off[i]) + (C.bc_off[i + 1] - C.bc_off[i]);
    nci[i] = (double)cnt / m[i];
  }

  for (int it = 0; it < p->pja_iters; ++it) {
#pragma omp parallel for num_threads(nthr) schedule(static)
    for (uint32_t i = 0; i < n; ++i) {
      double S[3] = {0, 0, 0};
      for (uint32_t c = C.pp_off[i]; c < C.pp_off[i + 1]; ++c) {
        uint32_t j = C.pp_j[c];
        double u[3];
        for (int k = 0; k < 3; ++k) u[k] = U[3 * i + k] - U[3 * j + k];
        /* mass splitting; or Alg. 1 as printed, where i takes the whole correction */
        double w = p->pja_weight ? m[i] : 1.0 / (nci[i] + nci[j]);
        pja_update(lp + 3 * c, u, C.pp_n + 3 * c, ab * C.pp_psi[c], w, mu);
        for (int k = 0; k < 3; ++k) S[k] += lp[3 * c + k];
      }
      for (uint32_t c = C.bc_off[i]; c < C.bc_off[i + 1]; ++c) {
        uint32_t b = C.bc_b[c];
        double ub[3], u[3];
        point_vel(Vb + 6 * b, Vb + 6 * b + 3, bodies[b].pos, C.bc_xc + 3 * c, ub);
        for (int k = 0; k < 3; ++k) u[k] = U[3 * i + k] - ub[k];
        double inv = p->pja_weight ? 1.0 / m[i] : nci[i];
        if (bodies[b].is_free) {
          double a[3] = {C.bc_xc[3 * c] - bodies[b].pos[0], C.bc_xc[3 * c + 1] - bodies[b].pos[1],
                         C.bc_xc[3 * c + 2] - bodies[b].pos[2]};
          inv += (double)ncb[b] * free_inv_mass(&bodies[b], Rb + 9 * b, a, C.bc_n + 3 * c);
        }
        pja_update(lb + 3 * c, u, C.bc_n + 3 * c, ab * C.bc_psi[c], 1.0 / inv, mu);
        for (int k = 0; k < 3; ++k) S[k] += lb[3 * c + k];
      }
      for (int k = 0; k < 3; ++k) Un[3 * i + k] = base[3 * i + k] + S[k] / m[i];
    }
    /* free-box corners against non-free bodies */
    for (uint32_t c = 0; c < ncc; ++c) {
      uint32_t b = C.cc_b[c], o = C.cc_o[c];
      double ub[3], uo[3], u[3];
      point_vel(Vb + 6 * b, Vb + 6 * b + 3, bodies[b].pos, C.cc_xc + 3 * c, ub);
      point_vel(Vb + 6 * o, Vb + 6 * o + 3, bodies[o].pos, C.cc_xc + 3 * c, uo);
      for (int k = 0; k < 3; ++k) u[k] = ub[k] - uo[k];
      double a[3] = {C.cc_xc[3 * c] - bodies[b].pos[0], C.cc_xc[3 * c + 1] - bodies[b].pos[1],
                     C.cc_xc[3 * c + 2] - bodies[b].pos[2]};
      double inv = (double)ncb[b] * free_inv_mass(&bodies[b], Rb + 9 * b, a, C.cc_n + 3 * c);
      pja_update(lc + 3 * c, u, C.cc_n + 3 * c, ab * C.cc_psi[c], 1.0 / inv, mu);
    }
    /* free bodies: new twist from the impulses of this iteration */
    for (uint32_t b = 0; b < nb; ++b) {
      memcpy(Vn + 6 * b, Vb + 6 * b, sizeof(double) * 6);
      if (!bodies[b].is_free) continue;
      double P[3] = {0, 0, 0}, L[3] = {0, 0, 0};
      for (uint32_t i = 0; i < n; ++i)
        for (uint32_t c = C.bc_off[i]; c < C.bc_off[i + 1]; ++c) {
          if (C.bc_b[c] != b) continue;
          double a[3] = {C.bc_xc[3 * c] - bodies[b].pos[0], C.bc_xc[3 * c + 1] - bodies[b].pos[1],
                         C.bc_xc[3 * c + 2] - bodies[b].pos[2]};
          double f[3] = {-lb[3 * c], -lb[3 * c + 1], -lb[3 * c + 2]}, t[3];
          cross3(a, f, t);
          for (int k = 0; k < 3; ++k) {
            P[k] += f[k];
            L[k] += t[k];
          }
        }
      for (uint32_t c = 0; c < ncc; ++c) {
        if (C.cc_b[c] != b) continue;
        double a[3] = {C.cc_xc[3 * c] - bodies[b].pos[0], C.cc_xc[3 * c + 1] - bodies[b].pos[1],
                       C.cc_xc[3 * c + 2] - bodies[b].pos[2]};
        double t[3];
        cross3(a, lc + 3 * c, t);
        for (int k = 0; k < 3; ++k) {
          P[k] += lc[3 * c + k];
          L[k] += t[k];
        }
      }
      double dw[3];
      inv_inertia_world(Rb + 9 * b, bodies[b].inertia, L, dw);
      for (int k = 0; k < 3; ++k) {
        Vn[6 * b + k] = base_b[6 * b + k] + P[k] / bodies[b].mass;
        Vn[6 * b + 3 + k] = base_b[6 * b + 3 + k] + dw[k];
      }
    }
    double *t = U;
    U = Un;
    Un = t;
    t = Vb;
    Vb = Vn;
    Vn = t;
  }

  /* fixed-point residual of the last iterate (complementarity, cone, sliding direction) */
  if (st) {
    double res = 0, vs = sqrt(dot3(g, g)) * dt;
    for (uint32_t i = 0; i < n; ++i) {
      double vi = sqrt(dot3(U + 3 * i, U + 3 * i));
      if (vi > vs) vs = vi;
    }
    if (vs == 0) vs = 1;
    for (uint32_t i = 0; i < n; ++i) {
      for (uint32_t c = C.pp_off[i]; c < C.pp_off[i + 1]; ++c) {
        uint32_t j = C.pp_j[c];
        double u[3];
        for (int k = 0; k < 3; ++k) u[k] = U[3 * i + k] - U[3 * j + k];
        double rr = contact_residual(lp + 3 * c, u, C.pp_n + 3 * c, ab * C.pp_psi[c], m[i], mu);
        if (rr > res) res = rr;
      }
      for (uint32_t c = C.bc_off[i]; c < C.bc_off[i + 1]; ++c) {
        uint32_t b = C.bc_b[c];
        double ub[3], u[3];
        point_vel(Vb + 6 * b, Vb + 6 * b + 3, bodies[b].pos, C.bc_xc + 3 * c, ub);
        for (int k = 0; k < 3; ++k) u[k] = U[3 * i + k] - ub[k];
        double rr = contact_residual(lb + 3 * c, u, C.bc_n + 3 * c, ab * C.bc_psi[c], m[i], mu);
        if (rr > res) res = rr;
      }
    }
    st->ncp_residual = res / vs;
  }

  /* symplectic Euler (reading of Eq. 4-5): velocity first, then position; then the
     cyclic vertical boundary of the gear tower (the paper's Sec. III: particles leaving
     through the bottom re-enter at the top with the same velocity) */
  const int cyclic = p->cyclic_z[1] > p->cyclic_z[0];
  for (uint32_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) {
      v[3 * i + k] = U[3 * i + k];
      x[3 * i + k] += dt * v[3 * i + k];
    }
    if (cyclic && x[3 * i + 2] < p->cyclic_z[0]) x[3 * i + 2] += p->cyclic_z[1] - p->cyclic_z[0];
  }

  /* wrench on each body = -(impulses it gives) / dt */
  if (wrench) {
    memset(wrench, 0, sizeof(double) * 6 * nb);
    for (uint32_t i = 0; i < n; ++i)
      for (uint32_t c = C.bc_off[i]; c < C.bc_off[i + 1]; ++c) {
        uint32_t b = C.bc_b[c];
        double a[3] = {C.bc_xc[3 * c] - bodies[b].pos[0], C.bc_xc[3 * c + 1] - bodies[b].pos[1],
                       C.bc_xc[3 * c + 2] - bodies[b].pos[2]};
        double f[3] = {-lb[3 * c] / dt, -lb[3 * c + 1] / dt, -lb[3 * c + 2] / dt}, t[3];
        cross3(a, f, t);
        for (int k = 0; k < 3; ++k) {
          wrench[6 * b + k] += f[k];
          wrench[6 * b + 3 + k] += t[k];
        }
      }
    for (uint32_t c = 0; c < ncc; ++c) {
      uint32_t b = C.cc_b[c], o = C.cc_o[c];
      for (int side = 0; side < 2; ++side) {
        uint32_t bb = side ? o : b;
        double sg = side ? -1.0 : 1.0;
        double a[3] = {C.cc_xc[3 * c] - bodies[bb].pos[0], C.cc_xc[3 * c + 1] - bodies[bb].pos[1],
                       C.cc_xc[3 * c + 2] - bodies[bb].pos[2]};
        double f[3] = {sg * lc[3 * c] / dt, sg * lc[3 * c + 1] / dt, sg * lc[3 * c + 2] / dt}, t[3];
        cross3(a, f, t);
        for (int k = 0; k < 3; ++k) {
          wrench[6 * bb + k] += f[k];
          wrench[6 * bb + 3 + k] += t[k];
        }
      }
    }
  }

  /* bodies: kinematic ones follow their twist, free ones the solved twist */
  for (uint32_t b = 0; b < nb; ++b) {
    double V[3], W[3];
    for (int k = 0; k < 3; ++k) {
      V[k] = Vb[6 * b + k];
      W[k] = Vb[6 * b + 3 + k];
    }
    if (bodies[b].is_free)
      for (int k = 0; k < 3; ++k) {
        bodies[b].lin_vel[k] = V[k];
        bodies[b].ang_vel[k] = W[k];
      }
    for (int k = 0; k < 3; ++k) bodies[b].pos[k] += dt * V[k];
    quat_integrate(bodies[b].quat, W, dt);
  }

  if (pp_lam) memcpy(pp_lam, lp, sizeof(double) * 3 * npp);
  if (bc_lam) memcpy(bc_lam, lb, sizeof(double) * 3 * nbc);
  if (st) {
    double res = st->ncp_residual;
    fill_stats(&C, st);
    st->ncp_residual = res;
  }
  free(Rb);
  free(Vb);
  free(Vn);
  free(base_b);
  free(ncb);
  free(base);
  free(U);
  free(Un);
  free(lp);
  free(lb);
  free(lc);
  free(nci);
  contacts_free(&C);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Loss for the differentiable workload (smooth mass inside the scoop cavity) */
/* ------------------------------------------------------------------------- */

double orc_scoop_loss(uint32_t n, const double *x, const double *m, const orc_body *scoop, double eps) {
  double R[9];
  rot64(scoop->quat, R);
  double L = 0;
  for (uint32_t i = 0; i < n; ++i) {
    double y[3], z[3];
    world_to_body64(scoop, R, x + 3 * i, y);
    for (int k = 0; k < 3; ++k) z[k] = y[k] - scoop->shape[6 + k];
    double q[3] = {fabs(z[0]) - scoop->shape[3], fabs(z[1]) - scoop->shape[4], fabs(z[2]) - scoop->shape[5]};
    double mq[3] = {q[0] > 0 ? q[0] : 0, q[1] > 0 ? q[1] : 0, q[2] > 0 ? q[2] : 0};
    double mx = q[0] > q[1] ? q[0] : q[1];
    if (q[2] > mx) mx = q[2];
    double f = sqrt(dot3(mq, mq)) + (mx < 0 ? mx : 0);
    L += m[i] / (1.0 + exp(f / eps));
  }
  return L;
}

/* ------------------------------------------------------------------------- */
/* Depth observations (Sec. III-A)                                            */
/* ------------------------------------------------------------------------- */

/* SDF used to step the sphere tracing: the body's FP32 SDF; outside a GRID body's
 * sampled box (where the SDF is not defined) the distance to that box, at least eps. */
static float march_f32(const bodyf *b, const float *y, float eps) {
  int br;
  float f = sdf_f32(b, y, &br);
  if (b->kind != ORC_GRID || br >= 0) return f;
  float q[3];
  for (int k = 0; k < 3; ++k) {
    float lo = b->s[k];
    float hi = b->s[k] + b->s[3] * (float)(b->gn[k] - 1);
    float a = lo - y[k];
    float c = y[k] - hi;
    q[k] = fmaxf(fmaxf(a, c), 0.0f);
  }
  float s2 = q[0] * q[0];
  float t = q[1] * q[1];
  s2 = s2 + t;
  t = q[2] * q[2];
  s2 = s2 + t;
  return fmaxf(sqrtf(s2), eps);
}

void orc_render(const orc_camera *cam, uint32_t n, const double *x, const double *r, uint32_t nb,
                const orc_body *bodies, double *out) {
  const int W = cam->width, H = cam->height;
  if (cam->kind == 0) {
    const float cx = (float)cam->pos[0], cy = (float)cam->pos[1];
    const float ex = (float)cam->extent[0], ey = (float)cam->extent[1];
    const float sx = ex / (float)W, sy = ey / (float)H;
    const float bx = cx - 0.5f * ex, by = cy - 0.5f * ey;
    for (int v = 0; v < H; ++v)
      for (int u = 0; u < W; ++u) {
        const float px = bx + ((float)u + 0.5f) * sx;
        const float py = by + ((float)v + 0.5f) * sy;
        double best = -INFINITY;
        int hit = 0;
        for (uint32_t i = 0; i < n; ++i) {
          const float dx = (float)x[3 * i] - px, dy = (float)x[3 * i + 1] - py, rf = (float)r[i];
          float d2 = dx * dx;
          float t = dy * dy;
          d2 = d2 + t;
          if (!(d2 <= rf * rf)) continue;
          const double ddx = x[3 * i] - (double)px, ddy = x[3 * i + 1] - (double)py;
          const double h2 = r[i] * r[i] - (ddx * ddx + ddy * ddy);
          const double h = x[3 * i + 2] + sqrt(h2 > 0 ? h2 : 0.0);
          if (!hit || h > best) best = h;
          hit = 1;
        }
        out[(size_t)v * W + u] = hit ? best : cam->empty;
      }
    return;
  }
  /* perspective depth */
  const float f = (float)(0.5 * (double)H / tan(0.5 * (double)(float)cam->fov_y));
  float q[4], R[9], o[3];
  for (int k = 0; k < 4; ++k) q[k] = (float)cam->quat[k];
  rot_f32(q, R);
  for (int k = 0; k < 3; ++k) o[k] = (float)cam->pos[k];
  const float nearc = (float)cam->near_clip, farc = (float)cam->far_clip, eps = (float)cam->march_eps;
  const uint32_t steps = cam->march_steps;
  bodyf *bf = (bodyf *)malloc(sizeof(bodyf) * (nb ? nb : 1));
  for (uint32_t b = 0; b < nb; ++b) body_to_f32(&bodies[b], &bf[b]);
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      const float ax = ((float)u + 0.5f) - 0.5f * (float)W;
      const float ay = ((float)v + 0.5f) - 0.5f * (float)H;
      const float dxc = ax / f, dyc = ay / f;
      float s2 = dxc * dxc;
      float t2 = dyc * dyc;
      s2 = s2 + t2;
      s2 = s2 + 1.0f;
      const float nr = sqrtf(s2);
      const float dc[3] = {dxc / nr, dyc / nr, 1.0f / nr};
      float d[3];
      for (int k = 0; k < 3; ++k) {
        float a = R[3 * k] * dc[0];
        float c = R[3 * k + 1] * dc[1];
        a = a + c;
        c = R[3 * k + 2] * dc[2];
        d[k] = a + c;
      }
      double best = INFINITY;
      /* spheres: FP32 hit decision, FP64 distance */
      for (uint32_t i = 0; i < n; ++i) {
        const float oc0 = (float)x[3 * i] - o[0], oc1 = (float)x[3 * i + 1] - o[1], oc2 = (float)x[3 * i + 2] - o[2];
        const float rf = (float)r[i];
        float b = d[0] * oc0;
        float tt = d[1] * oc1;
        b = b + tt;
        tt = d[2] * oc2;
        b = b + tt;
        float c = oc0 * oc0;
        tt = oc1 * oc1;
        c = c + tt;
        tt = oc2 * oc2;
        c = c + tt;
        c = c - rf * rf;
        const float disc = b * b - c;
        if (!(disc >= 0.0f)) continue;
        const float t0 = b - sqrtf(disc);
        if (!(t0 >= nearc && t0 <= farc)) continue;
        const double e0 = x[3 * i] - (double)o[0], e1 = x[3 * i + 1] - (double)o[1], e2 = x[3 * i + 2] - (double)o[2];
        const double bb = (double)d[0] * e0 + (double)d[1] * e1 + (double)d[2] * e2;
        const double cc = e0 * e0 + e1 * e1 + e2 * e2 - r[i] * r[i];
        const double dd = bb * bb - cc;
        const double td = bb - sqrt(dd > 0 ? dd : 0.0);
        if (td < best) best = td;
      }
      /* bodies: FP32 sphere tracing */
      if (nb && cam->body_mask) {
        float t = nearc;
        for (uint32_t k = 0; k < steps; ++k) {
          float p[3];
          for (int a = 0; a < 3; ++a) {
            float m = t * d[a];
            p[a] = o[a] + m;
          }
          float fmin = INFINITY;
          for (uint32_t b = 0; b < nb && b < 32; ++b) {
            if (!((cam->body_mask >> b) & 1u)) continue;
            float y[3];
            to_body_f32(&bf[b], p, y);
            const float fb = march_f32(&bf[b], y, eps);
            fmin = fminf(fmin, fb);
          }
          if (fmin < eps) {
            if ((double)t < best) best = (double)t;
            break;
          }
          t = t + fmin;
          if (!(t <= farc)) break;
        }
      }
      out[(size_t)v * W + u] = best <= (double)farc ? best : (double)farc;
    }
  free(bf);
}
