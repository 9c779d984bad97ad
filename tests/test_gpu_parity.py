"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer work -- bucket keys, sort permutation, bucket table, contact sets and
their order -- must match bit for bit, in lockstep: the GPU's FP32 state after k
steps is handed to the oracle's binning and contact stages.  Dynamics are
compared with tolerances: after one step every velocity within 1e-5 of the
scene's velocity scale, and after ten steps every position within 1e-3 r_i.
"""
import math

import numpy as np
import pytest

from gpu_helpers import F32, assert_contacts_equal, check_vel, lockstep_pair, need_gpu, pos_err
from paper_2306_01369_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def gg(torch):
    from paper_2306_01369_gb300 import gg
    return gg


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def squeezed_box(n=4096, factor=0.92, seed=1000, vel_scale=0.05):
    """The 0.2 m box scene with its lattice squeezed (pitch x factor) and lowered
    1 mm: many particle-particle contacts and floor contacts from the first step."""
    sc = S.settle_box(n=n, seed=seed)
    sc.pos_r[:, :2] = (sc.pos_r[:, :2] - np.float32(0.1)) * np.float32(factor) + np.float32(0.1)
    sc.pos_r[:, 2] = sc.pos_r[:, 2] * np.float32(factor) - np.float32(0.001)
    rng = np.random.default_rng(seed)
    sc.vel = (vel_scale * rng.uniform(-1, 1, (n, 3))).astype(F32)
    return sc


# --------------------------------------------------------------------------- #
# bit-exact integer stages
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("n,hash_size", [(4096, 0), (3001, 0), (2000, 97)])
def test_binning_sort_table_bit_exact(gg, orc, n, hash_size):
    sc = squeezed_box(n)
    sc.params.hash_size = hash_size
    sim = gg.Sim.from_scene(sc)
    sim.step(1)
    sim.sync()
    nh = hash_size or 2 * n
    cs = orc.default_cell_size(float(sc.pos_r[:, 3].max()))
    keys = orc.cell_keys(sc.pos_r[:, :3].astype(np.float64), cs, nh)
    assert np.array_equal(sim.cell_keys(), keys)
    perm = orc.sort_perm(keys)
    assert np.array_equal(sim.sort_perm(), perm)
    start = np.zeros(nh + 1, np.uint32)
    np.add.at(start, keys.astype(np.int64) + 1, 1)
    start = np.cumsum(start).astype(np.uint32)
    assert np.array_equal(sim.cell_start(), start)


LOCKSTEP_CASES = [("squeezed", 0), ("squeezed", 3), ("settle", 400), ("settle", 1200)]


def lockstep_scene(kind):
    return squeezed_box(4096) if kind == "squeezed" else S.settle_box(n=4096)


@pytest.mark.parametrize("kind,steps_before", LOCKSTEP_CASES)
def test_contacts_bit_exact_lockstep(gg, orc, kind, steps_before):
    """Contact sets from the same FP32 state (the oracle's after k steps)."""
    sim, o, _ = lockstep_pair(gg, lockstep_scene(kind), steps_before)
    want = o.contacts()
    sim.step(1)
    sim.sync()
    got = sim.contacts()
    assert want["stats"]["n_pp"] > 1500 and want["stats"]["n_body"] > 100
    assert_contacts_equal(got, want)
    # brute force agrees too (the bucket walk misses nothing)
    brute = o.contacts(brute=True)
    assert np.array_equal(brute["pp_j"], want["pp_j"])


def test_contacts_bit_exact_random_cloud_tiny_table(gg, orc):
    """Many hash collisions (n_h = 5) force duplicate buckets in the 27-cell walk."""
    pr, vel = S.random_cloud(1500, seed=21, box=0.07, overlap=1.0)
    p = S.Params(dt=1e-4, gravity=(0, 0, 0), mu=0.5, pja_iters=5, hash_size=5, max_contacts=32)
    sim = gg.Sim(pr, vel, S.sphere_mass(pr[:, 3]), p)
    sim.step(1)
    sim.sync()
    want = orc.contacts(pr[:, :3], pr[:, 3], [], p)
    assert want["stats"]["max_pp"] <= 32
    assert_contacts_equal(sim.contacts(), want)


def test_half_stencil_sets_on_a_dense_cloud(gg, orc):
    """The two-pass pair search on a cloud where many spheres have more than eight
    partners, so both halves of a sphere's scratch hold more entries than the first
    pass keeps in shared memory and the second pass loads in its first batch: every
    half-stencil launch shape, both table sizes, the oracle's lists."""
    pr, vel = S.random_cloud(1500, seed=22, box=0.035, overlap=1.0)
    p = S.Params(dt=1e-4, gravity=(0, 0, 0), mu=0.5, pja_iters=5, max_contacts=32)
    want = orc.contacts(pr[:, :3], pr[:, 3], [], p)
    deg = np.diff(want["pp_off"].astype(np.int64))
    assert 12 <= want["stats"]["max_pp"] <= 32 and (deg > 8).sum() > 100
    sets = [k for k in range(1, gg.load().gg_tuning_count() + 1) if "half" in gg.tuning_flags(k)]
    assert sets
    for tuning in sets:
        for hf in (2, 8):
            sim = gg.Sim(pr, vel, S.sphere_mass(pr[:, 3]), p, tuning=tuning, hash_factor=hf)
            sim.step(1)
            sim.sync()
            assert_contacts_equal(sim.contacts(), want)
            sim.close()


# --------------------------------------------------------------------------- #
# dynamics
# --------------------------------------------------------------------------- #

def test_one_step_dynamics(gg, orc):
    sc = squeezed_box(4096)
    sim = gg.Sim.from_scene(sc)
    o = orc.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params)
    want = o.contacts()
    sim.step(1)
    o.step(1)
    check_vel(sim.vel(), o.v, sc, want)
    assert pos_err(sim.pos()[:, :3], o.x, 0.2) < 1


@pytest.mark.parametrize("kind,steps_before", LOCKSTEP_CASES[1:])
def test_one_step_dynamics_lockstep(gg, orc, kind, steps_before):
    sim, o, sc = lockstep_pair(gg, lockstep_scene(kind), steps_before)
    want = o.contacts()
    sim.step(1)
    o.step(1)
    check_vel(sim.vel(), o.v, sc, want)
    assert pos_err(sim.pos()[:, :3], o.x, 0.2) < 1


def test_contact_geometry_and_impulses(gg, orc):
    sim, o, sc = lockstep_pair(gg, squeezed_box(2048), 4)
    want = o.contacts()
    npp, nbc = int(want["pp_off"][-1]), int(want["bc_off"][-1])
    lam = np.zeros((npp, 3))
    blam = np.zeros((nbc, 3))
    o.step(1, pp_lam=lam, bc_lam=blam)
    sim.step(1)
    got = sim.contacts()
    assert_contacts_equal(got, want)
    assert np.abs(got["pp_geom"][:, :3] - want["pp_geom"][:, :3]).max() < 1e-5
    assert np.abs(got["pp_geom"][:, 3] - want["pp_geom"][:, 3]).max() < 1e-7 * 1   # psi in metres
    assert nbc > 100
    assert np.abs(got["bc_geom"][:, :3] - want["bc_geom"][:, :3]).max() < 1e-5
    assert np.abs(got["bc_geom"][:, 3] - want["bc_geom"][:, 3]).max() < 1e-7
    scale = max(np.abs(lam).max(), np.abs(blam).max())
    assert np.abs(got["pp_lam"] - lam).max() < 1e-4 * scale
    assert np.abs(got["bc_lam"] - blam).max() < 1e-4 * scale


@pytest.mark.parametrize("steps_before", [0, 1200])
def test_ten_steps_within_radius_fraction(gg, orc, steps_before):
    """From the lattice at rest, and from the settled box (the oracle's state after
    1200 steps), ten steps stay within 1e-3 r_i of the oracle."""
    sim, o, sc = lockstep_pair(gg, S.settle_box(n=4096), steps_before)
    sim.step(10)
    o.step(10)
    d = np.linalg.norm(sim.pos()[:, :3].astype(np.float64) - o.x, axis=1)
    assert np.all(d <= 1e-3 * sc.pos_r[:, 3]), float((d / sc.pos_r[:, 3]).max())


def test_momentum_and_antisymmetric_impulses(gg, orc):
    pr, vel = S.random_cloud(3000, seed=9, box=0.08, overlap=1.0, vel_scale=0.3)
    m = S.sphere_mass(pr[:, 3])
    p = S.Params(dt=1e-4, gravity=(0, 0, 0), mu=0.4, pja_iters=20, max_contacts=32)
    sim = gg.Sim(pr, vel, m, p)
    sim.step(1)
    c = sim.contacts()
    off, jj, lam = c["pp_off"], c["pp_j"], c["pp_lam"]
    assert off[-1] > 1000
    # lambda_ji == -lambda_ij bit for bit
    pos = {}
    for i in range(len(off) - 1):
        for k in range(off[i], off[i + 1]):
            pos[(i, int(jj[k]))] = k
    for (i, j), k in pos.items():
        assert np.array_equal(lam[pos[(j, i)]], -lam[k])
    sim.step(4)
    v = sim.vel().astype(np.float64)
    P0 = (m[:, None].astype(np.float64) * vel).sum(0)
    P1 = (m[:, None].astype(np.float64) * v).sum(0)
    scale = (m[:, None] * np.abs(vel)).sum()
    assert np.abs(P1 - P0).max() < 2e-6 * scale


def test_resting_sphere_baumgarte_decay(gg):
    r = F32(0.005)
    psi0 = 1e-6
    pr = np.array([[0.0, 0.0, F32(float(r) - psi0), r]], F32)
    p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=20)
    sim = gg.Sim(pr, np.zeros((1, 3), F32), np.array([0.01], F32), p)
    sim.set_bodies([S.Body(kind=S.PLANE)])
    psi = float(r) - float(pr[0, 2])
    for k in range(1, 6):
        sim.step(1)
        got = float(r) - float(sim.pos()[0, 2])
        want = (1 - 0.2) ** k * psi
        assert abs(got - want) < 4 * 2 ** -24 * 0.005 * k, (k, got, want)


@pytest.mark.parametrize("dtheta_deg", [-2.0, 2.0])
def test_incline_threshold(gg, dtheta_deg):
    mu = 0.5
    theta = math.atan(mu) + math.radians(dtheta_deg)
    quat = (math.cos(theta / 2), math.sin(theta / 2), 0.0, 0.0)
    r = 0.005
    nrm = np.array([0.0, -math.sin(theta), math.cos(theta)])
    x0 = (r - 1e-8) * nrm
    pr = np.array([[x0[0], x0[1], x0[2], r]], F32)
    sim = gg.Sim(pr, np.zeros((1, 3), F32), np.array([0.02], F32), S.Params(dt=1e-4, mu=mu, alpha=0.0, pja_iters=20))
    sim.set_bodies([S.Body(kind=S.PLANE, quat=quat)])
    sim.step(1)
    v = sim.vel()[0].astype(np.float64)
    vt = v - np.dot(v, nrm) * nrm
    want = 1e-4 * 9.81 * max(0.0, math.sin(theta) - mu * math.cos(theta))
    assert abs(np.linalg.norm(vt) - want) < 1e-5 * 9.81e-4 + 1e-6 * want


def test_wrench_matches_oracle_with_kinematic_scoop(gg, orc):
    sim, o, sc = lockstep_pair(gg, S.scoop_bed(n=4096, n_steps=200, dims=(16, 16, 16)), 150,
                               wrench_history=8)
    want = o.contacts()
    sim.step(1)
    o.step(1)
    got = sim.contacts()
    assert_contacts_equal(got, want)
    w = sim.wrench()[-1, :len(sc.bodies)].astype(np.float64)   # newest step is the last row
    scale = np.abs(o.wrench[:len(sc.bodies)]).max()
    assert scale > 0
    assert np.abs(w - o.wrench[:len(sc.bodies)]).max() < 2e-4 * scale
    check_vel(sim.vel(), o.v, sc, want)
    # kinematic pose follows the prescribed twist
    bs = sim.body_state()[1]
    assert np.allclose(bs[0:3], o.body_pose(1)[0:3], atol=1e-6)
    assert np.allclose(np.abs(np.dot(bs[3:7], o.body_pose(1)[3:7])), 1.0, atol=1e-6)


def test_scoop_scene_ten_steps(gg, orc):
    sim, o, sc = lockstep_pair(gg, S.scoop_bed(n=4096, n_steps=200, dims=(16, 16, 16)), 150)
    sim.step(10)
    o.step(10)
    d = np.linalg.norm(sim.pos()[:, :3].astype(np.float64) - o.x, axis=1)
    assert np.all(d <= 1e-3 * sc.pos_r[:, 3])


# --------------------------------------------------------------------------- #
# invariance, determinism, checkpoints
# --------------------------------------------------------------------------- #

def test_results_invariant_to_launch_shape_and_table_size(gg):
    sc = squeezed_box(3000)
    ref = None
    for tuning in range(1, gg.load().gg_tuning_count() + 1):
        for hf in (0, 1, 4, 8):
            sim = gg.Sim.from_scene(sc, tuning=tuning, hash_factor=hf)
            sim.step(6)
            out = np.concatenate([sim.pos().ravel(), sim.vel().ravel()])
            if ref is None:
                ref = out
            assert np.array_equal(out, ref), (tuning, hf)
            sim.close()


def test_results_invariant_to_cell_size(gg):
    """The cell edge only decides which buckets are walked (every cell within reach is,
    and the pair test is exact): positions and velocities are bit-identical for edges
    of 2.002, 2.2 and 2.5 r_max, with both binnings."""
    import dataclasses
    sc = squeezed_box(3000)
    rmax = float(sc.pos_r[:, 3].max())
    ref = None
    for f in (2.002, 2.2, 2.5):
        for tuning in (1, 7, 11):
            s2 = dataclasses.replace(sc, params=dataclasses.replace(sc.params, cell_size=float(np.float32(f * rmax))))
            sim = gg.Sim.from_scene(s2, tuning=tuning)
            sim.step(6)
            out = np.concatenate([sim.pos().ravel(), sim.vel().ravel()])
            if ref is None:
                ref = out
            assert np.array_equal(out, ref), (f, tuning)
            sim.close()


def test_autotuner_picks_a_set_and_changes_nothing(gg):
    sc = squeezed_box(4096)
    ref = gg.Sim.from_scene(sc, tuning=1)
    ref.step(8)
    auto = gg.Sim.from_scene(sc, tuning=0)
    auto.step(5)
    auto.autotune()                 # re-timed mid-run: the state is restored bit-exactly
    auto.step(3)
    assert 1 <= auto.tuning_selected <= gg.load().gg_tuning_count()
    assert np.array_equal(auto.pos(), ref.pos()) and np.array_equal(auto.vel(), ref.vel())
    ref.autotune()                  # a fixed set: nothing to do
    assert ref.tuning_selected == 1


@pytest.mark.parametrize("binning", [1, 2])
def test_autotuned_table_size_changes_nothing_but_the_keys(gg, orc, binning):
    """hash_tune: the autotuner also picks n_h among 2n, 4n, 8n and the cell edge among
    2.002, 2.2, 2.5 r_max (twice here, once at the first step and once mid-run, so the
    tables change between steps).  The state matches a fixed 2n table bit-exactly; the
    keys and the bucket table are Eq. 6's under the n_h and cell edge in use."""
    sc = squeezed_box(4096)
    ref = gg.Sim.from_scene(sc, tuning=1)
    ref.step(9)
    auto = gg.Sim.from_scene(sc, hash_tune=1, binning=binning)
    auto.step(5)
    assert auto.hash_size() in (2 * sc.n, 4 * sc.n, 8 * sc.n)
    auto.autotune()
    auto.step(3)
    pos_before = auto.pos()
    auto.step(1)
    nh = auto.hash_size()
    assert nh in (2 * sc.n, 4 * sc.n, 8 * sc.n)
    assert np.array_equal(auto.pos(), ref.pos()) and np.array_equal(auto.vel(), ref.vel())
    cs = auto.cell_size()
    rmax = float(sc.pos_r[:, 3].max())
    assert cs in [float(np.float32(f * rmax)) for f in (2.002, 2.2, 2.5)], cs
    keys = orc.cell_keys(pos_before[:, :3].astype(np.float64), cs, nh)
    assert np.array_equal(auto.cell_keys(), keys)
    assert np.array_equal(auto.sort_perm(), orc.sort_perm(keys))
    start = np.zeros(nh + 1, np.uint32)
    np.add.at(start, keys.astype(np.int64) + 1, 1)
    assert np.array_equal(auto.cell_start(), np.cumsum(start).astype(np.uint32))
    auto.close()
    ref.close()


def test_grid_barrier_wait_runs_out_and_reports(gg):
    """The fused sweep's grid barrier waits are bounded: with a phantom participant
    (a flag that nothing sets) every wait runs out, the step reports
    GG_ERR_DEVICE_TIMEOUT, and the GPU context stays usable."""
    sc = squeezed_box(2048)
    n_sets = gg.load().gg_tuning_count()
    fused = [k for k in range(1, n_sets + 1) if "fused" in gg.tuning_flags(k)]
    detect = [k for k in range(1, n_sets + 1) if "detect" in gg.tuning_flags(k)]
    import time
    for k in (fused[0], detect[0]):          # sweeps fused; detection and sweeps fused
        for limit_us, slowest_s in ((0, 30.0), (20000, 5.0)):   # the default bound, and a 20 ms one
            sim = gg.Sim(sc.pos_r, sc.vel, sc.mass, sc.params, tuning=k, barrier_test_phantoms=1,
                         wait_limit_us=limit_us)
            sim.set_bodies(sc.bodies)
            t0 = time.perf_counter()
            sim.step(1)
            with pytest.raises(gg.GGError) as e:
                sim.sync()
            assert e.value.status == gg.ERR_DEVICE_TIMEOUT
            assert time.perf_counter() - t0 < slowest_s
            sim.close()
        ok = gg.Sim.from_scene(sc, tuning=k)
        ok.step(2)
        ok.sync()


def test_run_to_run_deterministic(gg):
    sc = squeezed_box(4096)
    outs = []
    for _ in range(3):
        sim = gg.Sim.from_scene(sc)
        sim.step(15)
        outs.append(sim.pos().copy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_checkpoint_resume_bit_exact(gg):
    sc = S.scoop_bed(n=4096, n_steps=40, dims=(16, 16, 16))
    a = gg.Sim.from_scene(sc)
    a.step(20)
    b = gg.Sim.from_scene(sc)
    b.step(10)
    blob = b.state()
    b.step(3)   # wander off, then come back
    b.set_state(blob)
    b.step(10)
    assert np.array_equal(a.pos(), b.pos()) and np.array_equal(a.vel(), b.vel())
    assert np.array_equal(a.body_state(), b.body_state())


def test_stage_timing_switch_changes_nothing(gg):
    """Switching between the plain and the instrumented step graph leaves results
    bit-identical; stage times are positive and cover the step."""
    sc = squeezed_box(4096)
    a = gg.Sim.from_scene(sc, tuning=1)
    b = gg.Sim.from_scene(sc, tuning=1)
    a.step(12)
    for k in range(12):
        b.enable_timing(k % 3 == 1)
        b.step(1)
        if k % 3 == 1:
            st = b.stage_ms()
            assert all(v > 0 for v in st.values()), st
    b.enable_timing(False)
    with pytest.raises(gg.GGError):
        b.stage_ms()
    assert np.array_equal(a.pos(), b.pos()) and np.array_equal(a.vel(), b.vel())


def test_host_buffer_round_trip(gg, torch):
    """POS_VEL equals POS then VEL, to host and device buffers; set_particles from the
    same pinned buffer restores the state the step reads (the end-to-end loop)."""
    sc = squeezed_box(3001)
    sim = gg.Sim.from_scene(sc)
    sim.step(7)
    pos, vel = sim.pos(), sim.vel()
    p2, v2 = sim.pos_vel()
    assert np.array_equal(p2, pos) and np.array_equal(v2, vel)
    pinned = torch.empty(7 * sc.n, dtype=torch.float32).pin_memory()
    sim.read("POS_VEL", out=pinned)
    assert np.array_equal(pinned.numpy()[:4 * sc.n].reshape(-1, 4), pos)
    d = torch.empty(7 * sc.n, dtype=torch.float32, device="cuda")
    sim.read("POS_VEL", out=d)
    assert np.array_equal(d.cpu().numpy(), pinned.numpy())
    other = gg.Sim.from_scene(sc)
    other.set_particles(pinned[:4 * sc.n].view(sc.n, 4), pinned[4 * sc.n:].view(sc.n, 3))
    ref = gg.Sim.from_scene(sc)
    ref.step(7)
    for s in (ref, other):
        s.step(3)
    assert np.array_equal(ref.pos(), other.pos()) and np.array_equal(ref.vel(), other.vel())


# --------------------------------------------------------------------------- #
# edge cases and errors
# --------------------------------------------------------------------------- #

def test_empty_and_single_particle(gg):
    p = S.Params(dt=1e-4)
    sim = gg.Sim(np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), p)
    sim.set_bodies([S.Body(kind=S.PLANE)])
    sim.step(3)
    sim.sync()
    assert sim.stats()["steps"] == 3
    one = gg.Sim(np.array([[0, 0, 1.0, 0.01]], F32), None, None, p)
    one.step(10)
    v = one.vel()
    assert abs(v[0, 2] + 10 * float(F32(1e-4)) * float(F32(9.81))) < 1e-6


def test_overflow_is_reported(gg):
    pr, vel = S.random_cloud(500, seed=3, box=0.02, overlap=0.5)
    p = S.Params(dt=1e-4, max_contacts=2)
    sim = gg.Sim(pr, vel, S.sphere_mass(pr[:, 3]), p)
    sim.step(1)
    with pytest.raises(gg.GGError) as e:
        sim.sync()
    assert e.value.status == gg.ERR_CONTACT_OVERFLOW


def test_invalid_arguments(gg):
    p = S.Params(dt=1e-4)
    with pytest.raises(gg.GGError) as e:
        gg.Sim(np.array([[0, 0, 0, -1.0]], F32), None, None, p)   # negative radius
    assert e.value.status == gg.ERR_INVALID_ARG
    bad = S.Params(dt=-1.0)
    with pytest.raises(gg.GGError):
        gg.Sim(np.array([[0, 0, 0, 1.0]], F32), None, None, bad)
    sim = gg.Sim(np.array([[0, 0, 0, 1.0]], F32), None, None, p)
    with pytest.raises(gg.GGError):
        sim.set_bodies([S.Body(kind=9)])
    with pytest.raises(gg.GGError):
        sim.set_trajectory(3, np.zeros((4, 6), F32))   # no such body


# --------------------------------------------------------------------------- #
# full size: the column-collapse workload of the benchmark
# --------------------------------------------------------------------------- #

TEN = 10


@pytest.fixture(scope="module")
def column_800(orc):
    """The 262,144-sphere column as the oracle has it after 800 steps (bottom layers
    landed), rounded to float32; the oracle's own trajectory from there for ten steps:
    positions and contact lists at the start of each step, and the velocities after
    the first."""
    from gpu_helpers import fp32_scene, oracle_advanced
    import oracle
    sc = fp32_scene(S.column_collapse(), oracle_advanced(S.column_collapse(), 800, 16))
    o = oracle.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params, twist=sc.twist, n_threads=16)
    xs, lists = [], []
    v1 = None
    for k in range(TEN):
        xs.append(o.x.copy())
        lists.append(o.contacts())
        o.step(1)
        if k == 0:
            v1 = o.v.copy()
    xs.append(o.x.copy())
    return sc, lists, xs, v1


def _pair_sets(c):
    off, jj = c["pp_off"].astype(np.int64), c["pp_j"].astype(np.int64)
    return off, jj


def _list_moments(off, jj):
    """Per particle: partner count and the sums of j, j^2, j^3 over its list (int64, exact)."""
    n = off.size - 1
    cnt = np.diff(off)
    out = [cnt]
    for p in (1, 2, 3):
        v = np.zeros(n, np.int64)
        np.add.at(v, np.repeat(np.arange(n), cnt), jj.astype(np.int64) ** p)
        out.append(v)
    return np.stack(out, 1)


def _lists_differ(og, jg, oo, jo):
    """Particles whose partner lists differ (moments first, then the lists themselves)."""
    cand = np.nonzero((_list_moments(og, jg) != _list_moments(oo, jo)).any(1))[0]
    return [int(i) for i in cand]


def _column_check(gg, orc, column_800, tuning, hash_factor):
    """One step: bit-exact keys, sort order and contacts, per-particle velocities and
    positions.  Ten steps (the bar: within 1e-3 r_i): the two runs then take their
    contact decisions from their own states, FP32 and FP64, which differ by ~1e-5 r
    after a few steps, so a pair whose gap is within that distance of zero can be in
    contact on one side only; such a pair's impulse sends both of its spheres (and
    their near neighbours) on slightly different paths.  Checked: every pair whose
    contact decision differs is within 4 times the two runs' position difference of
    touching (a rounding-level flip, not a missed contact), and every particle farther
    than three contacts from any such pair is within 1e-3 r_i after ten steps."""
    sc, lists, xs, v1 = column_800
    want = lists[0]
    n = sc.n
    sim = gg.Sim.from_scene(sc, tuning=tuning, hash_factor=hash_factor)
    nh = sim.hash_size()
    r = sc.pos_r[:, 3].astype(np.float64)
    flipped = np.zeros(n, bool)
    for k in range(TEN):
        xg0 = sim.pos()[:, :3].astype(np.float64)
        sim.step(1)
        got = sim.contacts()
        if k == 0:
            cs = orc.default_cell_size(float(sc.pos_r[:, 3].max()))
            keys = orc.cell_keys(sc.pos_r[:, :3].astype(np.float64), cs, nh)
            assert np.array_equal(sim.cell_keys(), keys)
            assert np.array_equal(sim.sort_perm(), orc.sort_perm(keys))
            assert want["stats"]["n_pp"] > 20000
            assert_contacts_equal(got, want)
            check_vel(sim.vel(), v1, sc, want)
            assert pos_err(sim.pos()[:, :3], xs[1], 0.2) < 1
            continue
        # pairs on one side only: both endpoints flagged, each explained by the state gap
        og, jg = _pair_sets(got)
        oo, jo = _pair_sets(lists[k])
        xo = xs[k]
        dx = np.linalg.norm(xg0 - xo, axis=1)
        for i in _lists_differ(og, jg, oo, jo):
            a = set(jg[og[i]:og[i + 1]].tolist())
            b = set(jo[oo[i]:oo[i + 1]].tolist())
            if a == b:
                continue
            flipped[i] = True
            for j in a ^ b:
                flipped[j] = True
                gap = abs(float(np.linalg.norm(xo[i] - xo[j])) - (r[i] + r[j]))
                assert gap <= 4.0 * (dx[i] + dx[j]) + 1e-12, (k, i, j, gap, dx[i], dx[j])
    assert flipped.sum() < 1e-3 * n, int(flipped.sum())
    near = flipped.copy()
    off, jj = _pair_sets(lists[-1])
    owner = np.repeat(np.arange(n), np.diff(off))
    for _ in range(3):
        nxt = near.copy()
        nxt[jj[near[owner]]] = True
        near = nxt
    d = np.linalg.norm(sim.pos()[:, :3].astype(np.float64) - xs[TEN], axis=1)
    far = ~near
    assert np.all(d[far] <= 1e-3 * r[far]), float((d[far] / r[far]).max())
    assert np.median(d / r) < 1e-4
    sim.close()


def test_column_collapse_full_size_parity(gg, orc, column_800):
    """262,144 spheres at the paper's n_h = 2n under the autotuner's launch shapes, from
    the oracle's state after 800 steps (see _column_check)."""
    _column_check(gg, orc, column_800, 0, 2)


@pytest.mark.parametrize("tuning", list(range(1, 23)))
def test_column_collapse_full_size_every_launch_shape_at_8n(gg, orc, column_800, tuning):
    """The same at n_h = 8n under every launch-shape set, the benchmark's configuration
    among them (the autotuner picks one of these sets and a table of 2n, 4n or 8n)."""
    if tuning > gg.load().gg_tuning_count():
        pytest.skip("no such set")
    _column_check(gg, orc, column_800, tuning, 8)


@pytest.fixture(scope="module")
def excavation_65k():
    """A 65,536-sphere excavation bed (container, scoop, two free 3 cm cubes) after 500
    steps of the oracle: settled under the cubes, the scoop moving."""
    from gpu_helpers import fp32_scene, oracle_advanced
    import oracle
    base = S.excavation(n=65536, n_steps=800)
    sc = fp32_scene(base, oracle_advanced(base, 500, 16))
    o = oracle.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params, twist=sc.twist, n_threads=16)
    want = o.contacts()
    o.step(1)
    return sc, want, o.v.copy(), [o.body_twist(b) for b in range(len(sc.bodies))], o.wrench.copy()


@pytest.mark.parametrize("flag", ["lean", "half", "plain"])
def test_excavation_65k_one_step_lockstep(gg, excavation_65k, flag):
    """The excavation workload on a 65,536-sphere bed, one step from the oracle's
    state: contact lists bit-exact, per-particle velocities, the free cubes' twists and
    the body wrenches, under launch-shape sets with the lean sweep, the half-stencil
    pair search, and neither."""
    sc, want, v1, tw1, wr1 = excavation_65k
    n_sets = gg.load().gg_tuning_count()
    sets = [k for k in range(1, n_sets + 1) if (flag in gg.tuning_flags(k)) or
            (flag == "plain" and not gg.tuning_flags(k) & {"lean", "half", "fused"})]
    assert sets
    for k in sets:
        sim = gg.Sim.from_scene(sc, tuning=k, wrench_history=2)
        sim.step(1)
        assert want["stats"]["n_pp"] > 50000 and want["stats"]["n_body"] > 1000
        assert all(int((want["bc_b"] == b).sum()) >= 5 for b in (2, 3))   # cubes resting on the bed
        assert_contacts_equal(sim.contacts(), want)
        check_vel(sim.vel(), v1, sc, want)
        bs = sim.body_state()
        for b in (2, 3):
            assert np.abs(bs[b, 7:10] - tw1[b][:3]).max() < 1e-4 * max(1.0, np.abs(tw1[b][:3]).max())
        w = sim.wrench()[-1, :4].astype(np.float64)
        assert np.abs(w - wr1[:4]).max() < 1e-3 * np.abs(wr1[:4]).max()
        sim.close()


def test_tilted_kinematic_body_pose_closed_form(gg):
    """Sec. II: the twist of a driven body is in the world frame.  A box tilted 90
    degrees about x spinning about world z at omega: after k steps its orientation is
    exp(k dt omega / 2) (x) q0 (one axis, so the increments commute); the body-frame
    product q0 (x) exp(...) would be a different rotation."""
    q0 = np.array([math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0])
    w = 30.0
    p = S.Params(dt=1e-4, gravity=(0, 0, 0))
    sim = gg.Sim(np.array([[5.0, 5.0, 5.0, 0.01]], F32), None, None, p)
    sim.set_bodies([S.Body(kind=S.BOX, shape=(0.01, 0.01, 0.01), pos=(0.0, 0.0, 1.0), quat=tuple(q0),
                           ang_vel=(0.0, 0.0, w))])
    k = 53
    sim.step(k)
    q = sim.body_state()[0, 3:7].astype(np.float64)
    ang = k * float(F32(1e-4)) * float(F32(w))
    e = np.array([math.cos(ang / 2), 0.0, 0.0, math.sin(ang / 2)])
    aw, ax, ay, az = e
    bw, bx, by, bz = q0
    want = np.array([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw])
    assert abs(abs(float(np.dot(q, want))) - 1.0) < 1e-6, (q, want)
    body = np.array([bw * aw - bx * ax - by * ay - bz * az, bw * ax + bx * aw + by * az - bz * ay,
                     bw * ay - bx * az + by * aw + bz * ax, bw * az + bx * ay - by * ax + bz * aw])
    assert abs(abs(float(np.dot(body, want))) - 1.0) > 1e-6


@pytest.mark.parametrize("iters", [1, 2, 3, 4])
def test_literal_alg1_weight_head_on_pair(gg, iters):
    """Alg. 1 as printed (pja_weight = 1, w = m_i) on the CUDA path: two touching
    spheres of unequal mass approaching head-on exchange their normal velocities after
    an odd number of iterations and keep them after an even number (the oracle pins the
    same closed form)."""
    pr = np.array([[0.0, 0.0, 0.0, 0.5], [1.0, 0.0, 0.0, 0.5]], F32)
    vel = np.array([[0.75, 0.1, 0.0], [-0.25, 0.0, 0.0]], F32)
    p = S.Params(dt=1e-4, gravity=(0, 0, 0), mu=0.0, pja_iters=iters, cell_size=1.2, pja_weight=1)
    sim = gg.Sim(pr, vel, np.array([1.0, 3.0], F32), p)
    sim.step(1)
    want = vel.astype(np.float64)
    if iters % 2:
        want[0, 0], want[1, 0] = want[1, 0], want[0, 0]
    assert np.abs(sim.vel() - want).max() < 1e-6, (iters, sim.vel())


@pytest.mark.parametrize("iters", [1, 3])
def test_literal_alg1_weight_lockstep(gg, orc, iters):
    """Alg. 1 as printed on the squeezed box, one step from the same FP32 state:
    contact lists bit-exact, velocities within the per-particle tolerance with the
    Baumgarte floor counted once per contact (each contact hands particle i its whole
    correction, so each contact's psi rounding reaches i in full)."""
    import dataclasses
    sc = squeezed_box(4096)
    sc.params = dataclasses.replace(sc.params, pja_weight=1, pja_iters=iters)
    sim = gg.Sim.from_scene(sc)
    o = orc.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params)
    want = o.contacts()
    sim.step(1)
    o.step(1)
    assert_contacts_equal(sim.contacts(), want)
    check_vel(sim.vel(), o.v, sc, want, per_contact=True)
    mix = gg.Sim.from_scene(dataclasses.replace(sc, params=dataclasses.replace(sc.params, pja_weight=0)))
    mix.step(1)
    assert not np.array_equal(mix.vel(), sim.vel())      # the weighting is in effect


def test_literal_alg1_weight_unsupported_combinations(gg):
    p = S.Params(dt=1e-4, pja_weight=1)
    pr = np.array([[0.0, 0.0, 0.0, 0.01]], F32)
    with pytest.raises(gg.GGError) as e:
        gg.Sim(pr, None, None, p, max_free_bodies=1)
    assert e.value.status == gg.ERR_UNSUPPORTED
    sim = gg.Sim(pr, None, None, p)
    sim.set_bodies([S.Body(kind=S.PLANE), S.Body(kind=S.BOX, shape=(0.01, 0.01, 0.01), pos=(0, 0, 1))])
    with pytest.raises(gg.GGError) as e:
        sim.tape_reserve(4, 2)
    assert e.value.status == gg.ERR_UNSUPPORTED


def test_nonfinite_state_is_reported(gg):
    """Velocities near FLT_MAX set through gg_set_particles: two touching spheres
    approach at +-3e38 m/s, their relative velocity overflows to inf in the contact
    update, the state becomes non-finite, and gg_sync reports GG_ERR_NONFINITE.  The
    context stays usable."""
    pr = np.array([[0.0, 0.0, 0.0, 0.01], [0.019, 0.0, 0.0, 0.01]], F32)
    p = S.Params(dt=1e-4, gravity=(0, 0, 0))
    sim = gg.Sim(pr, np.zeros((2, 3), F32), None, p)
    sim.step(1)
    sim.sync()
    sim.set_particles(pr, np.array([[3e38, 0, 0], [-3e38, 0, 0]], F32))
    sim.step(1)
    with pytest.raises(gg.GGError) as e:
        sim.sync()
    assert e.value.status == gg.ERR_NONFINITE
    sim.close()
    ok = gg.Sim(pr, None, None, p)
    ok.step(2)
    ok.sync()


def test_crowded_bucket_is_reported_quickly(gg):
    """A cell size far above 2 r_max puts 3,000 spheres in one cell: the in-bucket
    ordering and the bucket walks stop at their bound, the step finishes in well under
    a second of GPU time and reports GG_ERR_INVALID_ARG; the context stays usable."""
    import time
    pr, vel = S.random_cloud(3000, seed=12, box=0.05, overlap=0.3)
    for binning in (1, 2):
        p = S.Params(dt=1e-4, gravity=(0, 0, 0), cell_size=1.0, max_contacts=32)
        sim = gg.Sim(pr, vel, S.sphere_mass(pr[:, 3]), p, binning=binning, tuning=1 if binning == 1 else 7)
        t0 = time.perf_counter()
        sim.step(1)
        with pytest.raises(gg.GGError) as e:
            sim.sync()
        assert e.value.status == gg.ERR_INVALID_ARG
        assert time.perf_counter() - t0 < 5.0
        sim.close()
    pr2, vel2 = S.random_cloud(300, seed=13, box=0.05)
    ok = gg.Sim(pr2, vel2, S.sphere_mass(pr2[:, 3]), S.Params(dt=1e-4, max_contacts=32))
    ok.step(2)
    ok.sync()


@pytest.mark.parametrize("n", [1, 3, 4, 5, 4097])
def test_pinned_transfers_ragged_and_misaligned(gg, torch, n):
    """set_particles from pinned host buffers (velocities 16-byte aligned or not) and the
    POS_VEL readback into a pinned buffer move every value bit for bit, whatever n mod 4."""
    pr0, vel = S.random_cloud(n, seed=31 + n, box=0.5, vel_scale=0.2)
    pr = pr0.copy()
    pr[:, :3] += np.float32(0.01)
    p = S.Params(dt=1e-4, gravity=(0, 0, 0))
    for shift in (0, 1):   # velocity buffer at a 16-byte boundary, and 4 bytes past one
        sim = gg.Sim(pr0, np.zeros_like(vel), S.sphere_mass(pr0[:, 3]), p)
        pos_h = torch.from_numpy(pr.copy()).pin_memory()
        vbuf = torch.zeros(3 * n + 4, dtype=torch.float32).pin_memory()
        vbuf[shift:shift + 3 * n] = torch.from_numpy(vel.reshape(-1))
        sim.set_particles(pos_h, vbuf[shift:shift + 3 * n].view(n, 3))
        assert np.array_equal(sim.pos(), pr) and np.array_equal(sim.vel(), vel)
        out = torch.full((7 * n,), -1.0, dtype=torch.float32).pin_memory()
        sim.read("POS_VEL", out=out)
        o = out.numpy()
        assert np.array_equal(o[:4 * n].reshape(n, 4), pr) and np.array_equal(o[4 * n:].reshape(n, 3), vel)
        sim.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_step_io_equals_the_three_calls(gg, torch, pinned):
    """gg_step_io (one graph for pinned buffers, the three calls otherwise) moves the same
    state and steps to the same result, bit for bit, as set_particles + step + POS_VEL."""
    sc = squeezed_box(3001)
    a, b = gg.Sim.from_scene(sc, tuning=11), gg.Sim.from_scene(sc, tuning=11)
    a.step(3)
    b.step(3)
    p0, v0 = a.pos_vel()

    def buf(x):   # a copy (the loops below write into these buffers)
        t = torch.from_numpy(np.array(x, dtype=F32, copy=True))
        return t.pin_memory() if pinned else t

    pos_h, vel_h = buf(p0), buf(v0)
    out = buf(np.zeros(7 * sc.n, F32))
    for _ in range(4):                       # the same buffers: the graph is reused
        a.step_io(pos_h, vel_h, out)
        pos_h.copy_(out[:4 * sc.n].view(sc.n, 4))
        vel_h.copy_(out[4 * sc.n:].view(sc.n, 3))
    for _ in range(4):
        b.set_particles(p0, v0)
        b.step(1)
        p0, v0 = b.pos_vel()
    o = out.numpy()
    assert np.array_equal(o[:4 * sc.n].reshape(-1, 4), p0) and np.array_equal(o[4 * sc.n:].reshape(-1, 3), v0)
    assert a.stats()["steps"] == b.stats()["steps"]
    other = buf(np.zeros(7 * sc.n, F32))     # new output buffer: the graph is captured again
    a.step_io(pos_h, vel_h, other)
    b.step(1)
    assert np.array_equal(other.numpy()[:4 * sc.n].reshape(-1, 4), b.pos())
