"""Planted-mistake check of the oracle's pins (run by hand: python tests/oracle_mutations.py).

Each entry below is a plausible slip in oracle/gg_oracle.c: a reversed sign, lever arm or
cross product, a dropped term, count or weight, a transposed rotation, a wrong tie order,
summation order or pixel axis.  For each one the script compiles a copy of the oracle with
that single change into a temporary directory (the oracle's own source is never touched),
points the oracle's loader at it (GG_ORACLE_LIB) and runs tests/test_oracle_pins.py.  A
slip that no pin fails is reported; the script exits non-zero if any such slip is not
marked as the same arithmetic written another way.

Not collected by pytest (the file name does not start with test_): one run compiles and
tests about ninety copies, a few minutes of CPU.  An argument restricts the run to the
mistakes whose name contains it.
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

SRC = os.path.join(ROOT, "oracle", "gg_oracle.c")

# (name, text in the oracle, replacement, same arithmetic as the original)
MUTATIONS = [
    # projected-Jacobi sweep (Alg. 1, mass splitting, Baumgarte)
    ("pair relative velocity reversed",
     "u[k] = U[3 * i + k] - U[3 * j + k];\n        /* mass splitting",
     "u[k] = U[3 * j + k] - U[3 * i + k];\n        /* mass splitting", False),
    ("partner's count dropped from w", "1.0 / (nci[i] + nci[j]);", "1.0 / (nci[i] + nci[i]);", False),
    ("gravity dropped from the base velocity", "base[3 * i + k] = v[3 * i + k] + dt * g[k];",
     "base[3 * i + k] = v[3 * i + k];", False),
    ("pair Baumgarte bias dropped", "ab * C.pp_psi[c], w, mu);", "0.0 * C.pp_psi[c], w, mu);", False),
    ("body Baumgarte bias dropped", "ab * C.bc_psi[c], 1.0 / inv, mu);", "0.0 * C.bc_psi[c], 1.0 / inv, mu);", False),
    ("body contact weight without the count", "double inv = p->pja_weight ? 1.0 / m[i] : nci[i];",
     "double inv = 1.0 / m[i];", False),
    ("n_i counts pair contacts only",
     "uint32_t cnt = (C.pp_off[i + 1] - C.pp_off[i]) + (C.bc_off[i + 1] - C.bc_off[i]);",
     "uint32_t cnt = (C.pp_off[i + 1] - C.pp_off[i]);", False),
    ("body relative velocity reversed", "u[k] = U[3 * i + k] - ub[k];\n        double inv",
     "u[k] = ub[k] - U[3 * i + k];\n        double inv", False),
    ("impulse sum halved", "Un[3 * i + k] = base[3 * i + k] + S[k] / m[i];",
     "Un[3 * i + k] = base[3 * i + k] + S[k] / m[i] / 2;", False),
    ("bias sign", "s[k] = lam[k] - w * (u[k] - bias * nrm[k]);", "s[k] = lam[k] - w * (u[k] + bias * nrm[k]);", False),
    ("cone: tangential clamp off", "  if (tn > mu * lnp) {", "  if (0 && tn > mu * lnp) {", False),
    ("cone: normal impulse unclamped", "  double lnp = ln > 0 ? ln : 0;", "  double lnp = ln;", False),
    ("cone: scale from the unclamped normal", "    double sc = mu * lnp / tn;", "    double sc = mu * ln / tn;", False),
    ("Alg. 1 weight from the partner's mass", "double w = p->pja_weight ? m[i] :", "double w = p->pja_weight ? m[j] :",
     False),
    ("Alg. 1 body weight halved", "double inv = p->pja_weight ? 1.0 / m[i] : nci[i];",
     "double inv = p->pja_weight ? 2.0 / m[i] : nci[i];", False),
    ("Alg. 1 body weight mass-split", "double inv = p->pja_weight ? 1.0 / m[i] : nci[i];", "double inv = nci[i];",
     False),
    # integration, bodies
    ("position from the old velocity", "      v[3 * i + k] = U[3 * i + k];\n      x[3 * i + k] += dt * v[3 * i + k];",
     "      x[3 * i + k] += dt * v[3 * i + k];\n      v[3 * i + k] = U[3 * i + k];", False),
    ("cyclic wrap the wrong way", "x[3 * i + 2] += p->cyclic_z[1] - p->cyclic_z[0];",
     "x[3 * i + 2] -= p->cyclic_z[1] - p->cyclic_z[0];", False),
    ("quaternion update with the full angle", "  double s = sin(0.5 * ang) / ang, c = cos(0.5 * ang);",
     "  double s = sin(ang) / ang, c = cos(ang);", False),
    ("body-frame quaternion update", "  r[1] = d[0] * q[1] + d[1] * q[0] + d[2] * q[3] - d[3] * q[2];",
     "  r[1] = d[0] * q[1] + d[1] * q[0] - d[2] * q[3] + d[3] * q[2];", False),
    ("driven body ignores its table", "    if (!bodies[b].is_free && twist) {", "    if (0 && !bodies[b].is_free && twist) {",
     False),
    ("surface velocity lever arm reversed", "  cross3(W, a, c);", "  cross3(a, W, c);", False),
    ("wrench torque reversed", "        cross3(a, f, t);\n        for (int k = 0; k < 3; ++k) {\n          wrench[6 * b + k]",
     "        cross3(f, a, t);\n        for (int k = 0; k < 3; ++k) {\n          wrench[6 * b + k]", False),
    ("free body without gravity", "base_b[6 * b + k] = tv[k] + (bodies[b].is_free ? dt * g[k] : 0.0);",
     "base_b[6 * b + k] = tv[k];", False),
    ("free body impulse sign", "Vn[6 * b + k] = base_b[6 * b + k] + P[k] / bodies[b].mass;",
     "Vn[6 * b + k] = base_b[6 * b + k] - P[k] / bodies[b].mass;", False),
    ("free body angular impulse sign", "Vn[6 * b + 3 + k] = base_b[6 * b + 3 + k] + dw[k];",
     "Vn[6 * b + 3 + k] = base_b[6 * b + 3 + k] - dw[k];", False),
    ("free body contact count dropped", "inv += (double)ncb[b] * free_inv_mass(", "inv += free_inv_mass(", False),
    ("free body torque reversed",
     "          double f[3] = {-lb[3 * c], -lb[3 * c + 1], -lb[3 * c + 2]}, t[3];\n          cross3(a, f, t);",
     "          double f[3] = {-lb[3 * c], -lb[3 * c + 1], -lb[3 * c + 2]}, t[3];\n          cross3(f, a, t);", False),
    ("world inertia not rotated",
     "  for (int k = 0; k < 3; ++k) b[k] = (R[0 + k] * a[0] + R[3 + k] * a[1] + R[6 + k] * a[2]) / I[k];",
     "  for (int k = 0; k < 3; ++k) b[k] = a[k] / I[k];", False),
    ("world inertia with R for R^T",
     "  for (int k = 0; k < 3; ++k) b[k] = (R[0 + k] * a[0] + R[3 + k] * a[1] + R[6 + k] * a[2]) / I[k];",
     "  for (int k = 0; k < 3; ++k) b[k] = (R[3 * k] * a[0] + R[3 * k + 1] * a[1] + R[3 * k + 2] * a[2]) / I[k];",
     False),
    ("effective-mass cross product reversed", "  cross3(a, nrm, an);", "  cross3(nrm, a, an);", True),
    ("free twist not kept", "        bodies[b].lin_vel[k] = V[k];\n        bodies[b].ang_vel[k] = W[k];",
     "        (void)V[k];\n        (void)W[k];", False),
    ("corner impulse sign on the box", "          P[k] += lc[3 * c + k];", "          P[k] -= lc[3 * c + k];", False),
    ("corner relative velocity reversed", "u[k] = ub[k] - uo[k];", "u[k] = uo[k] - ub[k];", False),
    ("corner FP32 position with R^T",
     "          float t = bf[b].R[3 * a + 0] * cf[0];\n          float u = bf[b].R[3 * a + 1] * cf[1];\n"
     "          t = t + u;\n          u = bf[b].R[3 * a + 2] * cf[2];",
     "          float t = bf[b].R[a] * cf[0];\n          float u = bf[b].R[3 + a] * cf[1];\n"
     "          t = t + u;\n          u = bf[b].R[6 + a] * cf[2];", False),
    ("corner without the box position", "        for (int a = 0; a < 3; ++a) w[a] += bodies[b].pos[a];",
     "        for (int a = 0; a < 3; ++a) w[a] += 0.0 * bodies[b].pos[a];", False),
    ("corners against free bodies too", "          if (o == b || bodies[o].is_free) continue;",
     "          if (o == b) continue;", False),
    # contact geometry (Sec. II-C, Eq. 7)
    ("contact point outside the surface", "xc[k] = x[k] - f * nrm[k];", "xc[k] = x[k] + f * nrm[k];", False),
    ("body normal left in the body frame", "  body_to_world_vec64(R, g, nrm);\n  *psi = r - f;",
     "  for (int k = 0; k < 3; ++k) nrm[k] = g[k];\n  *psi = r - f;", False),
    ("world to body with R for R^T",
     "  for (int k = 0; k < 3; ++k) y[k] = R[0 + k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];",
     "  for (int k = 0; k < 3; ++k) y[k] = R[3 * k] * d[0] + R[3 * k + 1] * d[1] + R[3 * k + 2] * d[2];", False),
    ("pair psi without r_j", "C->pp_psi[o + q] = r[i] + r[j] - dist;", "C->pp_psi[o + q] = r[i] + r[i] - dist;",
     False),
    ("pair normal reversed", "nn[k] = d[k] / dist;", "nn[k] = -d[k] / dist;", False),
    ("coincident normal reversed", "nn[2] = (i > j) ? 1.0 : -1.0;", "nn[2] = (i < j) ? 1.0 : -1.0;", False),
    ("cavity normal x not negated", "      g[0] = -g[0];\n      g[1] = -g[1];", "      g[0] = g[0];\n      g[1] = -g[1];",
     False),
    ("cavity normal z not negated", "      g[1] = -g[1];\n      g[2] = -g[2];", "      g[1] = -g[1];\n      g[2] = g[2];",
     False),
    ("tube normal outward", "      g[0] = -y[0] / rho;\n      g[1] = -y[1] / rho;",
     "      g[0] = y[0] / rho;\n      g[1] = y[1] / rho;", False),
    ("tube distance sign", "    return b->shape[0] - rho;", "    return rho - b->shape[0];", False),
    ("grid x derivative", "        df[0] += s * dw[a] * w[1][bb] * w[2][c];",
     "        df[0] += s * w[0][a] * w[1][bb] * w[2][c];", False),
    ("grid local coordinate shifted", "    t[k] = (y[k] - (double)(float)b->shape[k]) / h - (double)i[k];",
     "    t[k] = (y[k] - (double)(float)b->shape[k]) / h - (double)i[k] - 0.5;", False),
    ("open box floor normal down", "{0, 1, 0}, {0, 0, 1}};", "{0, 1, 0}, {0, 0, -1}};", False),
    ("open box floor above the origin (FP64)", "                   y[2] + b->shape[2]};",
     "                   y[2] - b->shape[2]};", False),
    ("box edge gradient without signs", "      for (int k = 0; k < 3; ++k) g[k] = m[k] * sgn1(y[k]) / o;",
     "      for (int k = 0; k < 3; ++k) g[k] = m[k] / o;", False),
    # FP32 decisions (readings g9, g12, g14)
    ("FP32 body frame with R for R^T",
     "    float a = b->R[0 + k] * d0;\n    float c = b->R[3 + k] * d1;\n    a = a + c;\n    c = b->R[6 + k] * d2;",
     "    float a = b->R[3 * k] * d0;\n    float c = b->R[3 * k + 1] * d1;\n    a = a + c;\n    c = b->R[3 * k + 2] * d2;",
     False),
    ("FP32 box without the inside term", "  float f = o + fminf(mx, 0.0f);", "  float f = o;", False),
    ("FP32 box x-y tie to y", "  else if (q0 >= q1 && q0 >= q2)", "  else if (q0 > q1 && q0 > q2)", False),
    ("FP32 box y-z tie to z", "  else if (q1 >= q2)", "  else if (q1 > q2)", False),
    ("FP32 scoop takes the minimum", "    if (fa >= nfb) {", "    if (fa <= nfb) {", False),
    ("FP32 open box floor above the origin", "    w[4] = y[2] + b->s[2];", "    w[4] = y[2] - b->s[2];", False),
    ("FP32 grid last-cell clamp off", "    if (c > (int32_t)b->gn[k] - 2) c = (int32_t)b->gn[k] - 2;",
     "    if (0) c = (int32_t)b->gn[k] - 2;", False),
    ("FP32 grid y and z edges swapped",
     "  float c10 = lerp_f32(v[nx], v[nx + 1], t[0]);\n  float c01 = lerp_f32(v[nxy], v[nxy + 1], t[0]);",
     "  float c01 = lerp_f32(v[nx], v[nx + 1], t[0]);\n  float c10 = lerp_f32(v[nxy], v[nxy + 1], t[0]);", False),
    ("FP32 grid accepts points below its samples", "    if (!(u >= 0.0f && u <= top)) {",
     "    if (!(u >= -1.0f && u <= top)) {", False),
    ("FP32 tube distance sign", "    return b->s[0] - sqrtf(q);", "    return sqrtf(q) - b->s[0];", False),
    ("FP64 rotation transposed", "  R[1] = 2 * (x * y - w * z);", "  R[1] = 2 * (x * y + w * z);", False),
    ("FP32 rotation transposed", "  R[1] = 2.0f * (xy - wz);", "  R[1] = 2.0f * (xy + wz);", False),
    # binning and the sphere test (Eq. 6, Sec. II-B)
    ("sphere test summed in another order",
     "  float d2 = dx * dx;\n  float t = dy * dy;\n  d2 = d2 + t;\n  t = dz * dz;\n  d2 = d2 + t;",
     "  float d2 = dy * dy;\n  float t = dz * dz;\n  d2 = d2 + t;\n  t = dx * dx;\n  d2 = t + d2;", False),
    ("touching spheres not in contact", "  return d2 <= rs2;", "  return d2 < rs2;", False),
    ("cell index truncated", "  return (int32_t)floorf(t);", "  return (int32_t)t;", False),
    ("cell index with a fused multiply-add", "  float t = x * inv_cell;\n  t = t + 0.5f;",
     "  float t = fmaf(x, inv_cell, 0.5f);", False),
    ("hash offset added", "  uint32_t a = ((uint32_t)k0 - HASH_Q) * HASH_P1;", "  uint32_t a = ((uint32_t)k0 + HASH_Q) * HASH_P1;",
     False),
    ("equal keys by descending id", "  if (x->id != y->id) return x->id < y->id ? -1 : 1;",
     "  if (x->id != y->id) return x->id > y->id ? -1 : 1;", False),
    ("bucket reached twice walked twice", "        if (dup) continue; /* reading: a bucket reached twice is walked once */",
     "        (void)dup;", False),
    ("one plane of neighbour cells", "  for (int dz = -1; dz <= 1; ++dz)", "  for (int dz = 0; dz <= 0; ++dz)", False),
    # depth observations (Sec. III-A)
    ("sky pixel corner instead of centre", "        const float px = bx + ((float)u + 0.5f) * sx;",
     "        const float px = bx + ((float)u) * sx;", False),
    ("sky rows with the column pitch", "        const float py = by + ((float)v + 0.5f) * sy;",
     "        const float py = by + ((float)v + 0.5f) * sx;", False),
    ("sky keeps the lowest surface", "          if (!hit || h > best) best = h;", "          if (!hit || h < best) best = h;",
     False),
    ("sky cap height r", "          const double h = x[3 * i + 2] + sqrt(h2 > 0 ? h2 : 0.0);",
     "          const double h = x[3 * i + 2] + r[i];", False),
    ("ego focal length", "  const float f = (float)(0.5 * (double)H / tan(0.5 * (double)(float)cam->fov_y));",
     "  const float f = (float)(0.5 * (double)W / tan((double)(float)cam->fov_y));", False),
    ("ego y up", "      const float ay = ((float)v + 0.5f) - 0.5f * (float)H;",
     "      const float ay = 0.5f * (float)H - ((float)v + 0.5f);", False),
    ("ego x left", "      const float ax = ((float)u + 0.5f) - 0.5f * (float)W;",
     "      const float ax = 0.5f * (float)W - ((float)u + 0.5f);", False),
    ("ego camera rotation transposed",
     "        float a = R[3 * k] * dc[0];\n        float c = R[3 * k + 1] * dc[1];\n        a = a + c;\n"
     "        c = R[3 * k + 2] * dc[2];",
     "        float a = R[k] * dc[0];\n        float c = R[3 + k] * dc[1];\n        a = a + c;\n        c = R[6 + k] * dc[2];",
     False),
    ("ego far intersection", "        const double td = bb - sqrt(dd > 0 ? dd : 0.0);",
     "        const double td = bb + sqrt(dd > 0 ? dd : 0.0);", False),
    ("ego near clip ignored", "        if (!(t0 >= nearc && t0 <= farc)) continue;", "        if (!(t0 <= farc)) continue;",
     False),
    ("ego march never stops", "          if (fmin < eps) {", "          if (fmin < 0.0f) {", False),
    ("ego grid box distance from the wrong side", "    float a = lo - y[k];", "    float a = y[k] - lo;", False),
    # loss of the differentiable workload
    ("scoop loss counts the outside", "    L += m[i] / (1.0 + exp(f / eps));", "    L += m[i] / (1.0 + exp(-f / eps));",
     False),
    ("scoop loss cavity offset sign", "z[k] = y[k] - scoop->shape[6 + k];", "z[k] = y[k] + scoop->shape[6 + k];", False),
]


def run(only: str = "") -> int:
    """Check every planted mistake (or those whose name contains `only`)."""
    src = open(SRC).read()
    survivors, rows = [], []
    chosen = [m for m in MUTATIONS if only in m[0]]
    with tempfile.TemporaryDirectory() as tmp:
        for name, old, new, same in chosen:
            if src.count(old) != 1:
                rows.append((name, f"text found {src.count(old)} times"))
                survivors.append(name)
                continue
            path = os.path.join(tmp, "gg_oracle.c")
            with open(path, "w") as f:
                f.write(src.replace(old, new))
            so = os.path.join(tmp, f"libgg_oracle_{len(rows)}.so")
            hdr = os.path.join(ROOT, "oracle")
            subprocess.check_call(["gcc", *oracle.CFLAGS, "-I", hdr, "-o", so, path, "-lm"])
            env = dict(os.environ, GG_ORACLE_LIB=so)
            r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                                "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True)
            failed = [line for line in r.stdout.splitlines() if line.startswith("FAILED")]
            if failed:
                rows.append((name, "caught by " + failed[0].split("::", 1)[1].split(" ")[0]))
            else:
                rows.append((name, "same arithmetic, passes" if same else "NOT CAUGHT"))
                if not same:
                    survivors.append(name)
            print(f"{rows[-1][0]:48s} {rows[-1][1]}", flush=True)
    print(f"{len(chosen)} planted mistakes, {len(survivors)} not caught")
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(run(sys.argv[1] if len(sys.argv) > 1 else ""))
