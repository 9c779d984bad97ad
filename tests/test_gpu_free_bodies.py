"""Free rigid bodies that take contact reactions (two-way coupling; the paper's
bodies are kinematic, Sec. V lists two-way coupling as future work): closed forms
and oracle lockstep."""
import numpy as np
import pytest

from gpu_helpers import F32, assert_contacts_equal, check_vel, lockstep_pair, need_gpu
from paper_2306_01369_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    need_gpu()
    from paper_2306_01369_gb300 import gg
    return gg


def _params(**kw):
    p = S.Params(dt=1e-4, gravity=(0.0, 0.0, 0.0), mu=0.5, alpha=0.2, pja_iters=20)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_central_hit_is_perfectly_inelastic(gg):
    M = 2.0
    cube = S.Body(kind=S.BOX, shape=(0.25, 0.25, 0.25), pos=(0.75, 0.0, 0.0), is_free=1, mass=M,
                  inertia=(M * 0.25 / 6,) * 3)
    sim = gg.Sim(np.array([[0.0, 0.0, 0.0, 0.5]], F32), np.array([[1.0, 0, 0]], F32), np.array([1.0], F32),
                 _params(cell_size=1.2), max_free_bodies=1)
    sim.set_bodies([cube])
    sim.step(1)
    vc = 1.0 / (1.0 + M)
    assert abs(float(sim.vel()[0, 0]) - vc) < 1e-6
    bs = sim.body_state()[0]
    assert np.allclose(bs[7:13], [vc, 0, 0, 0, 0, 0], atol=1e-6)


def test_free_box_rests_on_its_corners(gg):
    M, hs = 0.5, 0.05
    cube = S.Body(kind=S.BOX, shape=(hs, hs, hs), pos=(0.0, 0.0, hs), is_free=1, mass=M,
                  inertia=(M * (2 * hs) ** 2 / 6,) * 3)
    p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=200)
    sim = gg.Sim(np.zeros((0, 4), F32), None, None, p, max_free_bodies=1, wrench_history=1)
    sim.set_bodies([S.Body(kind=S.PLANE), cube])
    sim.step(1)
    bs = sim.body_state()[1]
    g = 9.81
    assert np.abs(bs[7:13]).max() < 1e-6 * g
    w = sim.wrench()[-1]
    assert abs(w[0, 2] + M * g) < 1e-4 * M * g


def test_frictionless_hits_conserve_momenta(gg):
    M = 3.0
    h = (0.3, 0.2, 0.25)
    I = tuple(M / 3.0 * (h[(k + 1) % 3] ** 2 + h[(k + 2) % 3] ** 2) for k in range(3))
    q = S._quat_from_rotvec((0.2, -0.3, 0.1))
    cube = S.Body(kind=S.BOX, shape=h, pos=(0.0, 0.0, 0.0), quat=q, is_free=1, mass=M, inertia=I)
    pr = np.array([[0.25, 0.1, 0.4, 0.2], [-0.35, 0.05, -0.1, 0.15]], F32)
    vel = np.array([[0.0, -0.2, -1.0], [1.0, 0.3, 0.0]], F32)
    m = np.array([0.5, 0.7], F32)
    sim = gg.Sim(pr, vel, m, _params(mu=0.0, alpha=0.0, cell_size=1.0), max_free_bodies=1)
    sim.set_bodies([cube])
    st0 = sim.body_state()[0].astype(np.float64)
    sim.step(1)
    st1 = sim.body_state()[0].astype(np.float64)
    v = sim.vel().astype(np.float64)
    mm = m.astype(np.float64)[:, None]
    P0 = (mm * vel).sum(0)
    P1 = (mm * v).sum(0) + M * st1[7:10]
    assert np.abs(P1 - P0).max() < 1e-5
    # angular momentum about the origin, at the pre-step positions and orientation
    qq = st0[3:7] / np.linalg.norm(st0[3:7])
    a, b, c, d = qq
    R = np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]])
    Iw = R @ np.diag(I) @ R.T
    x0 = pr[:, :3].astype(np.float64)
    L0 = np.cross(x0, mm * vel).sum(0)
    L1 = np.cross(x0, mm * v).sum(0) + np.cross(st0[0:3], M * st1[7:10]) + Iw @ st1[10:13]
    assert np.abs(L1 - L0).max() < 1e-5
    assert np.abs(st1[10:13]).max() > 1e-3


@pytest.mark.parametrize("k", [0, 500])
def test_excavation_with_free_cubes_lockstep(gg, k):
    """Small excavation scene (16,384-sphere bed, container, scoop, two free 3 cm cubes):
    contact lists bit-exact, one-step particle velocities and cube twists within tolerance."""
    sc = S.excavation(n=16384, n_steps=800)
    sim, o, s32 = lockstep_pair(gg, sc, k, wrench_history=2)
    want = o.contacts()
    if k:   # the cubes have landed on the settling bed
        assert all(int((want["bc_b"] == b).sum()) >= 5 for b in (2, 3))
    sim.step(1)
    o.step(1)
    assert_contacts_equal(sim.contacts(), want)
    assert want["stats"]["n_body"] > 50
    check_vel(sim.vel(), o.v, s32, want)
    bs = sim.body_state()
    for b in (2, 3):   # the free cubes
        tw = o.body_twist(b)
        assert np.abs(bs[b, 7:10] - tw[:3]).max() < 1e-4 * max(1.0, np.abs(tw[:3]).max())
        assert np.abs(bs[b, 0:3] - o.body_pose(b)[:3]).max() < 1e-6
    w = sim.wrench()[-1, :4].astype(np.float64)
    scale = np.abs(o.wrench[:4]).max()
    assert np.abs(w - o.wrench[:4]).max() < 1e-3 * scale
