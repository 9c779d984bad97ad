"""Batched environments (many independent scenes stepped by the same launches).

Each environment of a batched run must equal its own single-environment run
bit for bit (same kernels, same canonical orders, its own hash range), and an
environment's contact lists must match the oracle's in lockstep.
"""
import numpy as np
import pytest

from gpu_helpers import assert_contacts_equal, check_vel, need_gpu
from paper_2306_01369_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    need_gpu()
    from paper_2306_01369_gb300 import gg
    return gg


def small_batch(n_envs=6, n_steps=30):
    return S.batched_beds(n_envs=n_envs, seed=1003, n_steps=n_steps, n_min=600, n_max=5000)


def env_scene(sc, e):
    o0, o1 = int(sc.env_offsets[e]), int(sc.env_offsets[e + 1])
    b0, b1 = int(sc.body_offsets[e]), int(sc.body_offsets[e + 1])
    tw = {gb - b0: t for gb, t in sc.twist.items() if b0 <= gb < b1}
    return S.Scene(f"env{e}", sc.pos_r[o0:o1].copy(), sc.vel[o0:o1].copy(), sc.mass[o0:o1].copy(),
                   sc.bodies[b0:b1], sc.params, sc.n_steps, twist=tw), o0, o1


def test_batched_equals_single_env_runs_bitwise(gg):
    sc = small_batch()
    bat = gg.Sim.from_scene(sc, wrench_history=4)
    bat.step(25)
    pos, vel = bat.pos(), bat.vel()
    bst = bat.body_state()
    wr = bat.wrench()
    st = bat.stats()
    assert st["n_pp"] > 0 and st["n_body"] > 0
    for e in range(len(sc.env_offsets) - 1):
        es, o0, o1 = env_scene(sc, e)
        one = gg.Sim.from_scene(es, wrench_history=4)
        one.step(25)
        assert np.array_equal(one.pos(), pos[o0:o1]), e
        assert np.array_equal(one.vel(), vel[o0:o1]), e
        nb = len(es.bodies)
        assert np.array_equal(one.body_state()[:nb], bst[e * 8:e * 8 + nb]), e
        assert np.array_equal(one.wrench()[:, :nb], wr[:, e * 8:e * 8 + nb]), e
        one.close()


@pytest.mark.parametrize("k", [0, 40])
def test_batched_env_contacts_match_oracle_lockstep(gg, k):
    """Every environment of a batched step matches its own oracle: contact lists
    bit for bit and velocities within tolerance, from the oracle's FP32 state
    after k steps of each environment."""
    from gpu_helpers import fp32_scene, oracle_advanced
    import oracle
    sc = small_batch(n_envs=4, n_steps=80)
    envs = [env_scene(sc, e)[0] for e in range(4)]
    if k:
        envs = [fp32_scene(es, oracle_advanced(es, k, 4)) for es in envs]
    pos = np.concatenate([es.pos_r for es in envs])
    vel = np.concatenate([es.vel for es in envs])
    mass = np.concatenate([es.mass for es in envs])
    bat = gg.Sim(pos, vel, mass, sc.params, env_offsets=sc.env_offsets)
    for e, es in enumerate(envs):
        bat.set_bodies(es.bodies, e)
        for b, tw in es.twist.items():
            bat.set_trajectory(b, tw, e)
    bat.step(1)
    got = bat.contacts()
    v = bat.vel()
    n_pp = 0
    for e, es in enumerate(envs):
        o0, o1 = int(sc.env_offsets[e]), int(sc.env_offsets[e + 1])
        o = oracle.Sim(es.pos_r, es.vel, es.mass, es.bodies, es.params, twist=es.twist, n_threads=4)
        want = o.contacts()
        n_pp += want["stats"]["n_pp"]
        sub = {"pp_off": got["pp_off"][o0:o1 + 1] - got["pp_off"][o0],
               "pp_j": got["pp_j"][got["pp_off"][o0]:got["pp_off"][o1]] - o0,
               "bc_off": got["bc_off"][o0:o1 + 1] - got["bc_off"][o0],
               "bc_b": got["bc_b"][got["bc_off"][o0]:got["bc_off"][o1]]}
        assert_contacts_equal(sub, want)
        o.step(1)
        check_vel(v[o0:o1], o.v, es, want)
    if k:
        assert n_pp > 1000


def test_batched_full_recipe_sixteen_envs_lockstep(gg):
    """Sixteen environments at the batched workload's own sizes (8k-64k spheres each,
    525,557 in all) under the launch shapes and table size its benchmark runs (set 22,
    n_h = 8n): from each environment's oracle state after 40 steps, every environment's
    contact lists bit for bit and its one-step velocities per particle."""
    from gpu_helpers import fp32_scene, oracle_advanced
    import oracle
    sc = S.batched_beds(n_envs=16, seed=1003, n_steps=80)
    envs = [fp32_scene(es, oracle_advanced(es, 40, 16)) for es in (env_scene(sc, e)[0] for e in range(16))]
    pos = np.concatenate([es.pos_r for es in envs])
    vel = np.concatenate([es.vel for es in envs])
    mass = np.concatenate([es.mass for es in envs])
    bat = gg.Sim(pos, vel, mass, sc.params, env_offsets=sc.env_offsets, tuning=22, hash_factor=8)
    for e, es in enumerate(envs):
        bat.set_bodies(es.bodies, e)
        for b, tw in es.twist.items():
            bat.set_trajectory(b, tw, e)
    bat.step(1)
    got = bat.contacts()
    v = bat.vel()
    bat.close()
    n_pp = 0
    for e, es in enumerate(envs):
        o0, o1 = int(sc.env_offsets[e]), int(sc.env_offsets[e + 1])
        o = oracle.Sim(es.pos_r, es.vel, es.mass, es.bodies, es.params, twist=es.twist, n_threads=16)
        want = o.contacts()
        n_pp += want["stats"]["n_pp"]
        sub = {"pp_off": got["pp_off"][o0:o1 + 1] - got["pp_off"][o0],
               "pp_j": got["pp_j"][got["pp_off"][o0]:got["pp_off"][o1]] - o0,
               "bc_off": got["bc_off"][o0:o1 + 1] - got["bc_off"][o0],
               "bc_b": got["bc_b"][got["bc_off"][o0]:got["bc_off"][o1]]}
        assert_contacts_equal(sub, want)
        o.step(1)
        check_vel(v[o0:o1], o.v, es, want)
    assert sc.n > 500000 and n_pp > 200000
