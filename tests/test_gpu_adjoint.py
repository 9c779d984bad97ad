"""Gradients of a task loss w.r.t. the tool's per-step twists and mu (hand-written
adjoint behind torch.autograd.Function; beyond the paper, Sec. V future work).

Scene: 512 spheres settled by the FP64 oracle around a stationary scoop (the
oracle's FP32-rounded state is the common input), then 10 steps with the scoop
on its seeded path.  Loss: the smooth mass inside the scoop's cavity.  The oracle
gradient is the central finite difference of the FP64 oracle's loss; every
difference step is checked to leave each step's contact set and each contact's
projection branch as the unperturbed run has them.
"""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import F32, need_gpu
from paper_2306_01369_gb300 import scenes as S

pytestmark = pytest.mark.gpu

T_STEPS = 10


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def scene():
    import oracle
    sc = S.diff_scene(n=512, n_steps=T_STEPS)
    o = oracle.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params, twist={}, n_threads=8)
    o.step(600)   # settle around the stationary scoop
    pos_r = np.empty_like(sc.pos_r)
    pos_r[:, :3] = o.x
    pos_r[:, 3] = sc.pos_r[:, 3]
    return S.Scene("diff_settled_512", pos_r, o.v.astype(F32), sc.mass, sc.bodies, sc.params, T_STEPS,
                   twist={1: sc.twist[1]}, info=sc.info)


def oracle_run(scene, tw, mu):
    """The FP64 oracle's loss after the T steps, and per step the contact lists and the
    branch each contact's last projection took (0 separated, 1 sticking, 2 sliding):
    what the piecewise-smooth step holds fixed."""
    import oracle
    p = dataclasses.replace(scene.params, mu=mu)
    o = oracle.Sim(scene.pos_r, scene.vel, scene.mass, scene.bodies, p, twist={1: tw}, n_threads=4)
    sets = []
    for _ in range(tw.shape[0]):
        c = o.contacts()
        lam = np.zeros((int(c["pp_off"][-1]), 3))
        blam = np.zeros((int(c["bc_off"][-1]), 3))
        geom = np.concatenate([c["pp_geom"][:, :3], c["bc_geom"][:, :3]])
        o.step(1, pp_lam=lam, bc_lam=blam)
        lm = np.concatenate([lam, blam])
        ln = (lm * geom).sum(1)
        lt = np.linalg.norm(lm - ln[:, None] * geom, axis=1)
        branch = np.where(ln <= 0.0, 0, np.where(lt >= mu * ln * (1 - 1e-9), 2, 1))
        sets.append((c["pp_off"], c["pp_j"], c["bc_off"], c["bc_b"], branch))
    return o.scoop_loss(1, scene.info["eps"]), sets


def same_sets(a, b):
    return all(all(np.array_equal(x, y) for x, y in zip(sa, sb)) for sa, sb in zip(a, b))


def oracle_loss(scene, tw, mu, ref_sets=None):
    """The oracle's loss; with ref_sets, also asserts that the contact and active sets
    of every step are those of the unperturbed run (the precondition of a central
    difference of a piecewise-smooth function)."""
    L, sets = oracle_run(scene, tw, mu)
    if ref_sets is not None:
        assert same_sets(sets, ref_sets), "a finite-difference step changed a contact or active set"
    return L


def gpu_grad(torch, scene, checkpoint_every=4):
    from paper_2306_01369_gb300.autograd import rollout, scoop_mass
    dev = torch.device("cuda", 0)
    tw = torch.tensor(scene.twist[1], device=dev, requires_grad=True)
    mu = torch.tensor(float(scene.params.mu), device=dev, requires_grad=True)
    pos, vel, pose = rollout(tw, mu, scene, 1, checkpoint_every)
    L = scoop_mass(pos, torch.tensor(scene.mass, device=dev), pose, scene.bodies[1].shape12(), scene.info["eps"])
    L.backward()
    return float(L.detach()), tw.grad.cpu().numpy().astype(np.float64), float(mu.grad)


def fd(f, x32, h):
    """Central difference of f at float32 x32 (the step actually taken after rounding)."""
    xp, xm = F32(float(x32) + h), F32(float(x32) - h)
    return (f(xp) - f(xm)) / (float(xp) - float(xm))


def test_adjoint_matches_oracle_gradient(torch, scene):
    L, g_tw, g_mu = gpu_grad(torch, scene)
    tw0 = scene.twist[1].astype(F32)
    mu0 = F32(scene.params.mu)
    L_orc, ref = oracle_run(scene, tw0, float(mu0))
    assert abs(L - L_orc) < 1e-4 * L_orc
    assert sum(int(s[0][-1]) for s in ref) > 1000 and sum(int((s[4] == 2).sum()) for s in ref) > 0
    want = np.zeros_like(g_tw)
    for k in range(T_STEPS):
        for c in range(6):
            def f(v, k=k, c=c):
                t = tw0.copy()
                t[k, c] = v
                return oracle_loss(scene, t, float(mu0), ref)
            want[k, c] = fd(f, tw0[k, c], 1e-5 if c < 3 else 1e-4)
    want_mu = fd(lambda v: oracle_loss(scene, tw0, float(v), ref), mu0, 1e-4)
    assert np.abs(want).max() > 0
    cos = float((g_tw * want).sum() / (np.linalg.norm(g_tw) * np.linalg.norm(want)))
    rel = float(np.abs(g_tw - want).max() / np.abs(want).max())
    # the GPU runs the forward and the adjoint in FP32: measured max rel 1.2e-3 (twists)
    # at cos 0.9999986, and 0.9 % on dL/dmu, against the FP64 oracle's central differences
    assert cos > 0.99999, (cos, rel, g_mu, want_mu)
    assert rel < 2e-3, (cos, rel, g_mu, want_mu)
    assert abs(g_mu - want_mu) <= 2e-2 * max(abs(want_mu), 1e-3 * np.abs(want).max()), (g_mu, want_mu, cos, rel)


def test_adjoint_invariant_to_checkpoint_interval(torch, scene):
    ref = gpu_grad(torch, scene, checkpoint_every=1)
    for K in (3, 10):
        got = gpu_grad(torch, scene, checkpoint_every=K)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and got[2] == ref[2]


def test_adjoint_matches_gpu_directional_derivative(torch, scene):
    """Central difference of the GPU's own FP32 forward along the gradient direction
    and along a random direction: g . d must match (L(tw + h d) - L(tw - h d)) / 2h.
    (Single components are too small against the FP32 rounding of the final state;
    along a whole direction the signal adds up.)"""
    from paper_2306_01369_gb300.autograd import rollout, scoop_mass
    L, g_tw, _ = gpu_grad(torch, scene)
    dev = torch.device("cuda", 0)
    mass = torch.tensor(scene.mass, device=dev)

    def loss(tw):
        with torch.no_grad():
            pos, vel, pose = rollout(torch.tensor(tw, device=dev), torch.tensor(float(scene.params.mu), device=dev),
                                     scene, 1, 10)
            return float(scoop_mass(pos.double(), mass.double(), pose.double(), scene.bodies[1].shape12(),
                                    scene.info["eps"]))

    tw0 = scene.twist[1].astype(np.float64)
    rng = np.random.default_rng(4)
    for d in (g_tw / np.linalg.norm(g_tw), rng.normal(size=g_tw.shape)):
        d = d / np.linalg.norm(d)
        h = 1e-3
        tp = (tw0 + h * d).astype(F32)
        tm = (tw0 - h * d).astype(F32)
        step = (tp.astype(np.float64) - tm.astype(np.float64))
        want = float((g_tw * step).sum())        # first-order change for the step actually taken
        got = loss(tp) - loss(tm)
        scale = np.linalg.norm(g_tw) * 2 * h
        assert abs(got - want) < 0.05 * scale, (got, want, scale)


def test_backward_and_later_steps_identical_under_both_binnings(torch, scene):
    """The taped steps of the backward pass bin like any step; with linked-list binning
    the lists they fill must be emptied before the next push (else the next step's lists
    would be cut short or cycle).  Gradients and the steps after the backward must be
    bit-identical to the counting-sort binning."""
    from paper_2306_01369_gb300 import gg
    rng = np.random.default_rng(11)
    dpos = rng.normal(size=(scene.n, 3)).astype(F32)
    out = []
    for binning in (1, 2):
        sim = gg.Sim(scene.pos_r, scene.vel, scene.mass, scene.params, binning=binning)
        sim.set_bodies(scene.bodies)
        sim.set_trajectory(1, scene.twist[1].astype(F32))
        sim.tape_reserve(T_STEPS, 4)
        sim.step_taped(1, T_STEPS)
        assert ("lists" in sim.tuning_flags) == (binning == 2)
        g_tw, g_mu = sim.backward(dpos)
        sim.step(5)
        sim.sync()
        out.append((g_tw, g_mu, sim.pos(), sim.vel()))
        sim.close()
    (g0, m0, p0, v0), (g1, m1, p1, v1) = out
    assert np.array_equal(g0, g1) and m0 == m1
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)


def test_repeated_taped_runs_on_one_simulation_are_identical(torch, scene):
    """A kept simulation reused the way a training loop reuses it: back to the start
    state, taped forward, backward, three times.  The second and third passes reuse the
    tape, the checkpoints and the per-slot graphs the first one captured; gradients and
    the final state are bit-identical every time."""
    from paper_2306_01369_gb300 import gg
    rng = np.random.default_rng(12)
    dpos = rng.normal(size=(scene.n, 3)).astype(F32)
    sim = gg.Sim(scene.pos_r, scene.vel, scene.mass, scene.params)
    sim.set_bodies(scene.bodies)
    sim.set_trajectory(1, scene.twist[1].astype(F32))
    sim.tape_reserve(T_STEPS, 4)
    st0 = sim.state()
    out = []
    for _ in range(3):
        sim.set_state(st0)
        sim.step_taped(1, T_STEPS)
        sim.sync()
        fin = (sim.pos(), sim.vel())
        g_tw, g_mu = sim.backward(dpos)
        out.append((g_tw, g_mu, fin))
    sim.close()
    for g_tw, g_mu, fin in out[1:]:
        assert np.array_equal(g_tw, out[0][0]) and g_mu == out[0][1]
        assert np.array_equal(fin[0], out[0][2][0]) and np.array_equal(fin[1], out[0][2][1])
