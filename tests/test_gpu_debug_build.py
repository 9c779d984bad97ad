"""The checked build (-DGG_DEBUG, libgg_debug.so): every device-side index check
(bucket keys, list links, partner and body indices of the sweeps, scratch entries of
the half-stencil pass, the adjoint's twin and partner gathers) passes on the test
scenes, and the checks change no result: positions, velocities and gradients equal the
release library's bit for bit.  It runs in a child process (GG_DEBUG=1 selects the
library at import)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# each case: (scene, tuning set, steps); the last one adds a backward pass
SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2306_01369_gb300 import gg, scenes as S
out = {}
bed = S.scoop_bed(n=4096, n_steps=40, dims=(16, 16, 16))
for tuning in (1, 9, 11, 13):
    sim = gg.Sim.from_scene(bed, tuning=tuning)
    sim.step(30)
    sim.sync()   # raises on GG_ERR_INTERNAL
    out[f"bed{tuning}"] = np.concatenate([sim.pos().ravel(), sim.vel().ravel()]).tobytes().hex()
    sim.close()
b = S.batched_beds(n_envs=4, n_steps=20, n_min=1024, n_max=2048)
sim = gg.Sim.from_scene(b, binning=2)
sim.step(15)
sim.sync()
out["batched"] = np.concatenate([sim.pos().ravel(), sim.vel().ravel()]).tobytes().hex()
sim.close()
sim = gg.Sim(bed.pos_r, bed.vel, bed.mass, bed.params, binning=2)
sim.set_bodies(bed.bodies)
sim.set_trajectory(1, bed.twist[1][:10].astype(np.float32))
sim.tape_reserve(10, 4)
sim.step_taped(1, 10)
g, gm = sim.backward(np.ones((bed.n, 3), np.float32))
sim.sync()
out["grad"] = np.asarray(g, np.float32).tobytes().hex() + "/" + repr(float(gm))
sim.close()
print(json.dumps(out))
"""


def run(debug):
    env = dict(os.environ, GG_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_passes_and_changes_nothing():
    need_gpu()
    from paper_2306_01369_gb300 import _build
    _build.build(debug=True)
    checked, release = run(True), run(False)
    assert checked.keys() == release.keys()
    for k in checked:
        assert checked[k] == release[k], k
