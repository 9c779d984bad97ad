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


def body_scale(body, x):
    """Body-frame coordinate scale of a particle at x in contact with `body`: the size
    of the FP32 numbers the SDF query rounds (|x - p|, plus a grid's sampled extent,
    whose cell coordinates are measured from its origin)."""
    L = float(np.linalg.norm(np.asarray(x, np.float64) - np.asarray(body.pos, np.float64)))
    g = getattr(body, "grid", None)
    if g is not None:
        ext = float(np.linalg.norm(g.origin)) + float(g.spacing) * float(max(g.values.shape))
        L += ext
    return L


def vel_tol(scene, v_orc, contacts, x=None, per_contact=False):
    """Per-particle tolerance of one-step velocities, GPU (FP32) vs oracle (FP64), from
    the same FP32 state: 1e-5 of the particle's own speed (at least g dt), plus the FP32
    floor of the Baumgarte bias of the contacts it has.  psi evaluated in FP32 carries up
    to ~8 eps32 L of rounding, L = the size of the coordinates it is computed from:
    2 r_max for a particle pair (|x_i - x_j| <= r_i + r_j), the body-frame coordinate
    scale for an SDF contact (particles with a body contact, and their direct partners;
    further away, scaled by the mass-splitting share of every contact on the way); the
    bias alpha psi / dt turns that into (alpha / dt) 8 eps32 L of velocity.
    `contacts`: the oracle's contact lists of the step's start state; x: its positions.
    per_contact: the floor once per contact of the particle (weightings that hand a
    particle each contact's whole correction, Alg. 1 as printed)."""
    p = scene.params
    v_orc = np.asarray(v_orc, np.float64)
    n = v_orc.shape[0]
    x = scene.pos_r[:, :3] if x is None else x
    scale = np.maximum(np.linalg.norm(v_orc, axis=1), 9.81 * p.dt)
    Lb = np.full(n, 2.0 * float(scene.pos_r[:, 3].max()))
    off, bb = contacts["bc_off"], contacts["bc_b"]
    for i in np.nonzero(np.diff(off.astype(np.int64)))[0]:
        for b in bb[off[i]:off[i + 1]]:
            Lb[i] = max(Lb[i], body_scale(scene.bodies[int(b)], x[i]))
    # a Jacobi sweep hands a particle part of each partner's estimate, so a partner's
    # body-contact rounding reaches it too (attenuated by the mass-splitting weight, about
    # 1 / (n_i + n_j) per hop): the floor of a particle is the largest of its own and its
    # partners' scales (one hop)
    L = Lb.copy()
    po, pj = contacts["pp_off"].astype(np.int64), contacts["pp_j"].astype(np.int64)
    has = np.diff(po) > 0
    if has.any():
        owner = np.repeat(np.arange(n), np.diff(po))
        np.maximum.at(L, owner, Lb[pj])
        # beyond the first hop the hand-off is the mass-splitting share of the contact,
        # w_ij / m_i = 1 / (n_i + n_j m_i / m_j): a scale reaches a particle h hops away
        # multiplied by the shares along the way (at most pja_iters hops, one per sweep)
        cnt = np.diff(po) + np.diff(off.astype(np.int64))
        m = np.asarray(scene.mass, np.float64)
        share = 1.0 / (cnt[owner] + cnt[pj] * m[owner] / m[pj])
        for _ in range(p.pja_iters - 1):
            reach = np.zeros(n)
            np.maximum.at(reach, owner, share * L[pj])
            grown = np.maximum(L, reach)
            if np.array_equal(grown, L):
                break
            L = grown
    floor = (p.alpha / p.dt) * 8.0 * EPS32 * L
    if per_contact:
        cnt = np.diff(contacts["pp_off"].astype(np.int64)) + np.diff(off.astype(np.int64))
        floor = floor * np.maximum(cnt, 1)
    return 1e-5 * scale + floor


def vel_err(v_gpu, v_orc, scene, contacts, x=None):
    """Largest per-particle one-step velocity difference as a fraction of that particle's
    vel_tol (pass: < 1); the worst particle is named in the message of check_vel."""
    d = np.abs(np.asarray(v_gpu, np.float64) - np.asarray(v_orc, np.float64)).max(axis=1)
    return float((d / vel_tol(scene, v_orc, contacts, x)).max())


def check_vel(v_gpu, v_orc, scene, contacts, x=None, per_contact=False):
    """Assert vel_err < 1 with a message that says which particle failed and why."""
    tol = vel_tol(scene, v_orc, contacts, x, per_contact)
    d = np.abs(np.asarray(v_gpu, np.float64) - np.asarray(v_orc, np.float64)).max(axis=1)
    r = d / tol
    i = int(np.argmax(r))
    off, boff = contacts["pp_off"], contacts["bc_off"]
    assert r[i] < 1, (f"particle {i}: |dv| {d[i]:.3e} > tol {tol[i]:.3e} (ratio {r[i]:.2f}); speed "
                      f"{np.linalg.norm(v_orc[i]):.3e}, {int(off[i + 1] - off[i])} pair and "
                      f"{int(boff[i + 1] - boff[i])} body contacts; "
                      f"{int((r > 1).sum())} particles fail, median ratio {float(np.median(r)):.3f}")
    return float(r[i])


def pos_err(x_gpu, x_orc, L_scene):
    """Per-particle one-step position difference over 1e-5 max(|x_i|, L_scene)."""
    x_orc = np.asarray(x_orc, np.float64)
    d = np.abs(np.asarray(x_gpu, np.float64) - x_orc).max(axis=1)
    return float((d / (1e-5 * np.maximum(np.linalg.norm(x_orc, axis=1), L_scene))).max())
