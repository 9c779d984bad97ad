"""The one-step velocity tolerance of the GPU parity tests (reading g21), checked on the
CPU on hand-made contact lists: it is the documented formula, it grows only near body
contacts, and it never exceeds the body-frame floor it starts from."""
import numpy as np

from gpu_helpers import EPS32, vel_tol
from paper_2306_01369_gb300 import scenes as S


def _chain(n, body_at_first=True):
    """n equal spheres in a row along x, each touching its neighbours; the first also
    touches a plane body 0.1 m away from the plane's origin."""
    r = 0.002
    pos_r = np.zeros((n, 4), np.float32)
    pos_r[:, 0] = 0.1 + 2 * r * np.arange(n)
    pos_r[:, 3] = r
    sc = S.Scene("chain", pos_r, np.zeros((n, 3), np.float32), np.full(n, 0.01, np.float32),
                 [S.Body(kind=S.PLANE)], S.Params(dt=1e-4, alpha=0.2, pja_iters=20), 1)
    pp_off, pp_j = [0], []
    for i in range(n):
        pp_j += [j for j in (i - 1, i + 1) if 0 <= j < n]
        pp_off.append(len(pp_j))
    bc_off = np.cumsum([0] + [1 if body_at_first and i == 0 else 0 for i in range(n)]).astype(np.uint32)
    contacts = {"pp_off": np.array(pp_off, np.uint32), "pp_j": np.array(pp_j, np.uint32),
                "bc_off": bc_off, "bc_b": np.zeros(int(bc_off[-1]), np.uint32)}
    return sc, contacts


def test_floor_formula_without_bodies():
    sc, c = _chain(6, body_at_first=False)
    v = np.zeros((6, 3))
    tol = vel_tol(sc, v, c)
    p = sc.params
    want = 1e-5 * 9.81 * p.dt + (p.alpha / p.dt) * 8 * EPS32 * 2 * float(sc.pos_r[:, 3].max())
    assert np.allclose(tol, want, rtol=1e-12)


def test_body_floor_reaches_partners_by_their_shares():
    """The sphere touching the body gets the body-frame scale |x - p| = 0.1 m; its direct
    partner the same (one hop); further along, each contact multiplies it by the
    mass-splitting share 1 / (n_i + n_j m_i / m_j) = 1/4 for equal masses with two
    contacts each (the second sphere: 1 / (2 + 2)), until it falls below 2 r_max."""
    n = 8
    sc, c = _chain(n)
    v = np.zeros((n, 3))
    p = sc.params
    base = 1e-5 * 9.81 * p.dt
    floor = (vel_tol(sc, v, c) - base) / ((p.alpha / p.dt) * 8 * EPS32)     # the scale L per sphere
    L0 = float(np.linalg.norm(sc.pos_r[0, :3].astype(np.float64)))
    assert abs(floor[0] - L0) < 1e-9 and abs(floor[1] - L0) < 1e-9
    # sphere 0 has a body contact and one pair (n = 2), the others two pairs (n = 2)
    assert abs(floor[2] - L0 / 4) < 1e-9 and abs(floor[3] - L0 / 16) < 1e-9
    two_r = 2 * float(sc.pos_r[:, 3].max())
    assert np.allclose(floor[5:], two_r)
    assert np.all(floor <= L0 + 1e-12) and np.all(np.diff(floor) <= 1e-12)
