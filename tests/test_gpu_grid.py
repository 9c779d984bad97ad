"""Bodies whose SDF is sampled on a regular grid (Sec. II-C: trilinear interpolation of
precomputed samples), on the CUDA path against the oracle.

Geometry: an involute helical gear (teeth 8, module 3 mm, 12 mm wide) baked on a
0.75 mm grid, spinning at 4 rad/s inside a bed of 4,096 spheres (r = 1.5 mm +-10 %);
and the excavation scoop baked on a grid, as the differentiated tool."""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import F32, assert_contacts_equal, check_vel, lockstep_pair, need_gpu, oracle_advanced
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
def gear_scene():
    return S.gear_bed(n=4096)


def test_gear_contacts_bit_exact_lockstep(gg, gear_scene):
    sim, o, _ = lockstep_pair(gg, gear_scene, 400)
    want = o.contacts()
    sim.step(1)
    sim.sync()
    got = sim.contacts()
    assert int((want["bc_b"] == 1).sum()) > 30 and want["stats"]["n_pp"] > 3000
    assert_contacts_equal(got, want)


def test_gear_one_step_and_ten_steps(gg, gear_scene):
    sim, o, sc = lockstep_pair(gg, gear_scene, 400)
    want = o.contacts()
    sim.step(1)
    o.step(1)
    check_vel(sim.vel(), o.v, sc, want)
    sim.step(9)
    o.step(9)
    dx = np.linalg.norm(sim.pos()[:, :3].astype(np.float64) - o.x, axis=1)
    assert dx.max() < 1e-3 * float(sc.pos_r[:, 3].min()), dx.max()


def test_sphere_rests_on_a_grid_plane(gg):
    r = F32(0.005)
    k, j, i = np.meshgrid(np.arange(9), np.arange(9), np.arange(9), indexing="ij")
    vals = (-0.0625 + k / 64.0).astype(F32)       # samples of z on a dyadic grid
    ground = S.Body(kind=S.GRID, grid=S.Grid(vals, (-0.0625, -0.0625, -0.0625), 1.0 / 64))
    psi0 = 1e-6
    z0 = F32(float(r) - psi0)
    p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=20)
    sim = gg.Sim(np.array([[0.01, -0.02, z0, r]], F32), np.zeros((1, 3), F32), np.array([0.01], F32), p)
    sim.set_bodies([ground])
    a = float(F32(0.2))
    psi = float(r) - float(z0)
    for kk in range(1, 6):
        sim.step(1)
        want = (1.0 - a) ** kk * psi
        got = float(r) - float(sim.pos()[0, 2])
        assert abs(got - want) < 4e-9, (kk, got, want)   # float32 positions near z = 5 mm


def test_grid_body_arguments(gg):
    p = S.Params(dt=1e-4)
    sim = gg.Sim(np.array([[0, 0, 0.1, 0.01]], F32), None, None, p)
    grid = S.Grid(np.zeros((2, 2, 2), F32), (0.0, 0.0, 0.0), 0.1)
    sim.set_bodies([S.Body(kind=S.PLANE)])
    with pytest.raises(gg.GGError):       # not a GRID body
        sim.set_body_grid(0, grid)
    with pytest.raises(gg.GGError) as e:  # free GRID bodies are not supported
        sim.set_bodies([S.Body(kind=S.GRID, is_free=1, mass=1.0, inertia=(1, 1, 1))])
    assert e.value.status == gg.ERR_UNSUPPORTED
    sim.set_bodies([S.Body(kind=S.GRID)])
    with pytest.raises(gg.GGError):       # spacing must be positive
        sim.set_body_grid(0, S.Grid(np.zeros((2, 2, 2), F32), (0.0, 0.0, 0.0), -1.0))
    sim.step(2)                           # a GRID body without samples touches nothing
    sim.sync()


# --------------------------------------------------------------------------- #
# the adjoint with a gridded tool
# --------------------------------------------------------------------------- #

T_STEPS = 8


@pytest.fixture(scope="module")
def grid_tool_scene():
    import oracle
    sc = S.diff_scene(n=512, n_steps=T_STEPS)
    scoop = sc.bodies[1]
    r_max = float(sc.pos_r[:, 3].max())
    ha = np.array(scoop.shape[0:3])
    g = S.bake_grid(S.box_minus_box_sdf(scoop.shape12()), -ha - 2 * r_max, ha + 2 * r_max, 0.5e-3)
    tool = dataclasses.replace(scoop, kind=S.GRID, shape=(0.0,) * 12, grid=g)
    bodies = [sc.bodies[0], tool]
    o = oracle.Sim(sc.pos_r, sc.vel, sc.mass, bodies, sc.params, twist={}, n_threads=8)
    o.step(600)
    pos_r = np.empty_like(sc.pos_r)
    pos_r[:, :3] = o.x
    pos_r[:, 3] = sc.pos_r[:, 3]
    return S.Scene("diff_grid_512", pos_r, o.v.astype(F32), sc.mass, bodies, sc.params, T_STEPS,
                   twist={1: sc.twist[1]}, info=dict(sc.info, scoop_shape=scoop.shape12()))


def test_adjoint_with_grid_tool_matches_oracle_gradient(torch, grid_tool_scene):
    import oracle
    from paper_2306_01369_gb300.autograd import rollout, scoop_mass
    sc = grid_tool_scene
    dev = torch.device("cuda", 0)
    shape = sc.info["scoop_shape"]
    tw = torch.tensor(sc.twist[1], device=dev, requires_grad=True)
    mu = torch.tensor(float(sc.params.mu), device=dev, requires_grad=True)
    pos, vel, pose = rollout(tw, mu, sc, 1, 4)
    L = scoop_mass(pos, torch.tensor(sc.mass, device=dev), pose, shape, sc.info["eps"])
    L.backward()
    g_tw = tw.grad.cpu().numpy().astype(np.float64)

    def loss(twv, muv):
        p = dataclasses.replace(sc.params, mu=muv)
        o = oracle.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, p, twist={1: twv}, n_threads=4)
        o.step(twv.shape[0])
        b = o.bodies[1]          # the tool at its final pose; the loss measures the closed-form cavity
        b.kind = S.BOX_MINUS_BOX
        for a, v in enumerate(shape):
            b.shape[a] = float(F32(v))
        return o.scoop_loss(1, sc.info["eps"])

    tw0 = sc.twist[1].astype(F32)
    mu0 = float(F32(sc.params.mu))
    L_orc = loss(tw0, mu0)
    assert abs(float(L.detach()) - L_orc) < 1e-4 * L_orc
    want = np.zeros_like(g_tw)
    for k in range(T_STEPS):
        for c in range(6):
            h = 1e-5 if c < 3 else 1e-4
            tp, tm = tw0.copy(), tw0.copy()
            tp[k, c] = F32(float(tw0[k, c]) + h)
            tm[k, c] = F32(float(tw0[k, c]) - h)
            want[k, c] = (loss(tp, mu0) - loss(tm, mu0)) / (float(tp[k, c]) - float(tm[k, c]))
    assert np.abs(want).max() > 0
    cos = float((g_tw * want).sum() / (np.linalg.norm(g_tw) * np.linalg.norm(want)))
    rel = float(np.abs(g_tw - want).max() / np.abs(want).max())
    assert cos > 0.999 and rel < 1e-2, (cos, rel)


# --------------------------------------------------------------------------- #
# the gear tower: tube wall, gears at random orientations, cyclic vertical boundary
# --------------------------------------------------------------------------- #

@pytest.fixture(scope="module")
def tower_scene():
    return S.gear_tower(n=4096, n_gears=3)


def test_tower_contacts_and_dynamics_lockstep(gg, tower_scene):
    sim, o, sc = lockstep_pair(gg, tower_scene, 1500)
    want = o.contacts()
    sim.step(1)
    sim.sync()
    assert_contacts_equal(sim.contacts(), want)
    assert int((want["bc_b"] >= 1).sum()) > 10       # contacts with the gears
    o.step(1)
    check_vel(sim.vel(), o.v, sc, want)


def test_tube_wall_contacts_and_dynamics(gg, orc):
    """Spheres pressed slightly into the tube's wall (and into each other): contact
    sets bit-exact, one-step velocities within tolerance."""
    rng = np.random.default_rng(8)
    n, R, r = 600, 0.06, 0.002
    ang = rng.uniform(0, 2 * np.pi, n)
    rho = R - r + rng.uniform(0.0, 0.3 * r, n)
    pr = np.stack([rho * np.cos(ang), rho * np.sin(ang), rng.uniform(0.0, 0.1, n), np.full(n, r)], 1).astype(F32)
    vel = (rng.normal(size=(n, 3)) * 0.05).astype(F32)
    sc = S.Scene("tube_wall", pr, vel, S.sphere_mass(pr[:, 3]), [S.Body(kind=S.TUBE, shape=(R,))],
                 S.Params(dt=1e-4, mu=0.5, pja_iters=20), 1)
    sim = gg.Sim.from_scene(sc)
    o = orc.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params)
    want = o.contacts()
    sim.step(1)
    sim.sync()
    assert int(want["stats"]["n_body"]) > 300
    assert_contacts_equal(sim.contacts(), want)
    o.step(1)
    check_vel(sim.vel(), o.v, sc, want)


def test_cyclic_boundary_wraps_like_the_oracle(gg, orc):
    """Spheres falling through the bottom of the period re-enter at the top with their
    velocity; positions agree with the oracle to float32 rounding over many wraps."""
    p = S.Params(dt=1e-3, mu=0.5, pja_iters=5, cyclic_z=(0.0, 0.0625))
    rng = np.random.default_rng(5)
    pr = np.zeros((64, 4), F32)
    pr[:, 0] = rng.uniform(-1, 1, 64) * 0.5
    pr[:, 1] = rng.uniform(-1, 1, 64) * 0.5
    pr[:, 2] = rng.uniform(0.0, 0.06, 64)
    pr[:, 3] = 0.001
    sim = gg.Sim(pr, np.zeros((64, 3), F32), np.full(64, 1e-3, F32), p)
    o = orc.Sim(pr, np.zeros((64, 3), F32), np.full(64, 1e-3, F32), [], p)
    sim.step(300)
    o.step(300)
    x = sim.pos()[:, :3].astype(np.float64)
    assert np.all((x[:, 2] >= 0.0) & (x[:, 2] < 0.0625))
    assert np.abs(sim.vel() - o.v).max() < 1e-5 * np.abs(o.v).max()
    dz = np.abs(x[:, 2] - o.x[:, 2])
    assert dz.max() < 1e-5, dz.max()


# --------------------------------------------------------------------------- #
# binning by linked lists (Alg. 2) against the counting sort
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("which", ["gear_bed", "scoop", "batched"])
def test_list_binning_gives_identical_results(gg, which, gear_scene):
    if which == "gear_bed":
        sc = gear_scene
    elif which == "scoop":
        sc = S.scoop_bed(n=4096, n_steps=60, dims=(16, 16, 16))
    else:
        sc = S.batched_beds(n_envs=6, n_steps=40, n_min=1024, n_max=4096)
    out = []
    for binning in (1, 2):
        sim = gg.Sim.from_scene(sc, binning=binning)    # the autotuner picks a set of that binning
        sim.step(30)
        assert ("lists" in sim.tuning_flags) == (binning == 2)
        out.append((sim.pos(), sim.vel(), sim.cell_keys(), sim.contacts(), sim.sort_perm(), sim.cell_start()))
        sim.close()
    (p0, v0, k0, c0, s0, t0), (p1, v1, k1, c1, s1, t1) = out
    assert np.array_equal(k0, k1)
    assert np.array_equal(s0, s1) and np.array_equal(t0, t1)   # lists: the keys sorted on demand
    assert_contacts_equal(c1, c0)
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
