"""Depth observations on the device (the paper's Sec. III-A sky and ego cameras)
against the oracle, from the same float32 state."""
import math

import numpy as np
import pytest

from gpu_helpers import F32, fp32_scene, need_gpu, oracle_advanced
from paper_2306_01369_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    need_gpu()
    from paper_2306_01369_gb300 import gg
    return gg


@pytest.fixture(scope="module")
def scoop_state():
    sc = S.scoop_bed(n=4096, n_steps=200, dims=(16, 16, 16))
    return fp32_scene(sc, oracle_advanced(sc, 150))


def _both(gg, orc, sc, cam):
    sim = gg.Sim.from_scene(sc)
    got = sim.render(cam)
    want = orc.render(cam, sc.pos_r[:, :3].astype(np.float64), sc.pos_r[:, 3].astype(np.float64), sc.bodies)
    sim.close()
    return got, want


def test_sky_camera_matches_oracle(gg, orc, scoop_state):
    sc = scoop_state
    foot = sc.info["side"] * sc.info["pitch"]
    cam = S.Camera(kind=S.HEIGHT_CAMERA, width=72, height=36, pos=(0.0, 0.0, 0.0), extent=(1.1 * foot, 0.55 * foot),
                   empty=-1.0)
    got, want = _both(gg, orc, sc, cam)
    assert np.array_equal(got == -1.0, want == -1.0)          # coverage decided identically (FP32)
    cov = want != -1.0
    assert cov.sum() > 1000
    err = np.abs(got[cov] - want[cov])
    # float32 vs float64 of z + sqrt(r^2 - d^2); at a sphere's rim sqrt amplifies rounding
    assert np.percentile(err, 99) < 2e-7 and err.max() < 2e-5, (np.percentile(err, 99), err.max())


def test_ego_camera_matches_oracle(gg, orc, scoop_state):
    """Perspective depth of the bed, the container and the scoop (sphere tracing)."""
    sc = scoop_state
    pose = (0.0, -0.12, 0.12)
    look = S._quat_from_rotvec((-2.2, 0.0, 0.0))             # tilted down towards the bed
    cam = S.Camera(kind=S.DEPTH_CAMERA, width=36, height=36, pos=pose, quat=look, fov_y=1.2, near=0.01, far=0.6,
                   march_steps=96, march_eps=1e-5)
    got, want = _both(gg, orc, sc, cam)
    assert np.array_equal(got == F32(0.6), want == float(F32(0.6)))
    hit = want < float(F32(0.6))
    assert hit.sum() > 600
    err = np.abs(got[hit] - want[hit])
    # rays grazing a sphere are ill-conditioned (d t / d disc = 1 / (2 sqrt(disc)))
    assert np.percentile(err, 99) < 2e-6 and err.max() < 1e-3, (np.percentile(err, 99), err.max())


def test_ego_camera_sees_grid_bodies(gg, orc):
    sc = S.gear_bed(n=4096)
    down = S._quat_from_rotvec((math.pi, 0.0, 0.0))
    cam = S.Camera(kind=S.DEPTH_CAMERA, width=36, height=36, pos=(0.0, 0.0, 0.08), quat=down, fov_y=1.0, near=0.005,
                   far=0.3, march_steps=128, march_eps=1e-5, body_mask=0b10)   # the gear alone (no container)
    sim = gg.Sim.from_scene(sc)
    got = sim.render(cam)
    empty = S.Scene("gear_only", np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), sc.bodies,
                    sc.params, 1)
    want = orc.render(cam, np.zeros((0, 3)), np.zeros(0), sc.bodies)
    got_only = gg.Sim.from_scene(empty).render(cam)
    assert np.array_equal(got_only, want.astype(F32))          # bodies alone: identical FP32 tracing
    hit = want < float(F32(0.3))
    assert hit.sum() > 100
    sim.close()


def test_render_arguments(gg):
    sim = gg.Sim(np.array([[0, 0, 0.1, 0.01]], F32), None, None, S.Params(dt=1e-4))
    for bad in (S.Camera(kind=S.DEPTH_CAMERA, fov_y=0.0), S.Camera(kind=S.DEPTH_CAMERA, near=0.5, far=0.1),
                S.Camera(kind=S.HEIGHT_CAMERA, extent=(0.0, 1.0)), S.Camera(kind=5), S.Camera(width=0)):
        with pytest.raises(gg.GGError):
            sim.render(bad)
