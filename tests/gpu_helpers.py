"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest

F32 = np.float32


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_01369_gb300 import _build
    _build.build()
    return torch


def csr_lists(res, key_off, key_val):
    off, val = res[key_off], res[key_val]
    return [list(val[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def assert_contacts_equal(got, want):
    """Bit-exact contact sets and canonical order (partners by id, bodies by index)."""
    for k in ("pp_off", "bc_off"):
        if not np.array_equal(got[k], want[k]):
            d = np.nonzero(np.diff(got[k].astype(np.int64)) != np.diff(want[k].astype(np.int64)))[0]
            raise AssertionError(f"{k} differs for {len(d)} particles, first {d[:5]}")
    assert np.array_equal(got["pp_j"], want["pp_j"]), "partner ids differ"
    assert np.array_equal(got["bc_b"], want["bc_b"]), "body indices differ"


def oracle_advanced(scene, k, n_threads=8):
    """The FP64 oracle run k steps from the scene's initial state."""
    import oracle
    o = oracle.Sim(scene.pos_r, scene.vel, scene.mass, scene.bodies, scene.params, twist=scene.twist,
                   n_threads=n_threads)
    if k:
        o.step(k)
    return o


def fp32_scene(scene, o):
    """The oracle's state after o.step_index steps, rounded to float32, as a new scene
    (bodies at the oracle's pose, tool twists from that step on).  Both the GPU and
    a fresh oracle start from it: lockstep inputs that never come from the GPU."""
    from paper_2306_01369_gb300 import scenes as S
    k = o.step_index
    pos_r = np.empty((scene.n, 4), F32)
    pos_r[:, :3] = o.x
    pos_r[:, 3] = scene.pos_r[:, 3]
    bodies = []
    for b, body in enumerate(scene.bodies):
        pose = o.body_pose(b)
        tw = o.body_twist(b)
        bodies.append(S.Body(kind=body.kind, shape=body.shape, pos=tuple(float(F32(v)) for v in pose[:3]),
                             quat=tuple(float(F32(v)) for v in pose[3:]),
                             lin_vel=tuple(float(v) for v in tw[:3]), ang_vel=tuple(float(v) for v in tw[3:]),
                             is_free=body.is_free, mass=body.mass, inertia=body.inertia,
                             grid=getattr(body, "grid", None)))
    twist = {b: t[k:] for b, t in scene.twist.items() if t.shape[0] > k}
    return S.Scene(f"{scene.name}@{k}", pos_r, o.v.astype(F32), scene.mass, bodies, scene.params,
                   max(0, scene.n_steps - k), twist=twist, env_offsets=scene.env_offsets,
                   body_offsets=scene.body_offsets, info=dict(scene.info))


def lockstep_pair(gg, scene, k, n_threads=8, **sim_kw):
    """(GPU sim, oracle sim, scene) both starting from the oracle's FP32 state after k steps."""
    import oracle
    s32 = fp32_scene(scene, oracle_advanced(scene, k, n_threads)) if k else scene
    sim = gg.Sim.from_scene(s32, **sim_kw)
    o = oracle.Sim(s32.pos_r, s32.vel, s32.mass, s32.bodies, s32.params, twist=s32.twist, n_threads=n_threads)
    return sim, o, s32


EPS32 = 2.0 ** -24


def vel_tol(scene, v_orc, length=None):
    """Tolerance of one-step velocities, GPU (FP32) vs oracle (FP64), from the same
    FP32 state: 1e-5 of the scene's velocity scale max(max_i |v_i|, g dt), plus the
    FP32 floor of the Baumgarte bias.  psi = (r_i + r_j) - |x_i - x_j| evaluated in
    FP32 carries up to ~8 eps32 * L of rounding (L = 2 r_max for particle pairs, the
    body-frame coordinate scale for SDF contacts), which the bias alpha psi / dt turns
    into (alpha / dt) 8 eps32 L of velocity."""
    p = scene.params
    vscale = max(float(np.abs(v_orc).max()), 9.81 * p.dt)
    L = 2.0 * float(scene.pos_r[:, 3].max()) if length is None else length
    return 1e-5 * vscale + (p.alpha / p.dt) * 8.0 * EPS32 * L


def vel_err(v_gpu, v_orc, scene, length=None):
    """Largest one-step velocity difference as a fraction of vel_tol (pass: < 1)."""
    return float(np.abs(v_gpu.astype(np.float64) - v_orc).max()) / vel_tol(scene, v_orc, length)

