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


def bodies_from_gpu(scene_bodies, bstate):
    """Scene bodies with the GPU's FP32 pose (lockstep input for the oracle)."""
    from paper_2306_01369_gb300 import scenes as S
    out = []
    for b, body in enumerate(scene_bodies):
        row = bstate[b]
        out.append(S.Body(kind=body.kind, shape=body.shape, pos=tuple(float(v) for v in row[0:3]),
                          quat=tuple(float(v) for v in row[3:7]), lin_vel=body.lin_vel, ang_vel=body.ang_vel,
                          is_free=body.is_free, mass=body.mass, inertia=body.inertia))
    return out


def oracle_from_gpu(sim, scene, step_index, n_threads=4):
    """An oracle Sim started from the GPU's current FP32 state (lockstep)."""
    import oracle
    pos = sim.pos()
    vel = sim.vel()
    bodies = bodies_from_gpu(scene.bodies, sim.body_state()) if scene.bodies else []
    o = oracle.Sim(pos, vel, scene.mass, bodies, scene.params, twist=scene.twist, n_threads=n_threads)
    o.step_index = step_index
    return o


def vel_err(v_gpu, v_orc, dt, g=9.81):
    """Largest velocity difference relative to the scene's velocity scale
    max(max_i |v_i|, g dt)."""
    vref = max(float(np.abs(v_orc).max()), g * dt)
    return float(np.abs(v_gpu.astype(np.float64) - v_orc).max()) / vref
