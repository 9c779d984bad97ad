"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-derived
hash values (Eq. 6), library routines (numpy lexsort, scipy's k-d tree), brute
force, and closed-form outcomes of the contact step (Alg. 1, Eq. 1-5, Baumgarte)
on scenes small enough to solve by hand.
"""
import math
import os

import numpy as np
import pytest

from paper_2306_01369_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F32 = np.float32


def _params(**kw):
    p = S.Params(dt=1e-4, gravity=(0.0, 0.0, 0.0), mu=0.5, alpha=0.2, pja_iters=20)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# --------------------------------------------------------------------------- #
# Binning (Eq. 6)
# --------------------------------------------------------------------------- #

def test_hash_golden(orc):
    rows = 0
    with open(os.path.join(GOLDEN, "hash_cells.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k0, k1, k2, nh, want = (int(t) for t in line.split())
            assert orc.hash_cell(k0, k1, k2, nh) == want, (k0, k1, k2, nh)
            rows += 1
    assert rows >= 8


def test_cell_index_is_rounding_to_nearest(orc):
    """Away from half-integers, the FP32 cell index equals round(x / c) of the paper."""
    rng = np.random.default_rng(0)
    c = F32(0.0044)
    inv = orc.inv_cell(float(c))
    assert inv == float(F32(1.0 / float(c)))
    xs = rng.uniform(-2.0, 2.0, 4000).astype(F32)
    for x in xs:
        y = float(x) / float(c)
        if abs(y - math.floor(y) - 0.5) < 1e-4:
            continue
        assert orc.cell_index(float(x), inv) == int(math.floor(y + 0.5))


def test_cell_index_two_roundings_no_fma(orc):
    """The cell index rounds x*inv_c to FP32 before adding 0.5 (no fused multiply-add).

    Search inputs where a fused x*inv_c + 0.5 would land in another cell; numpy's
    float32 arithmetic (one rounding per operation) gives the required answer.
    """
    rng = np.random.default_rng(1)
    inv = F32(orc.inv_cell(float(F32(0.0044))))
    found = 0
    for k in range(-3000, 3000):
        base = (k + 0.5) / float(inv)
        for x in (np.nextafter(F32(base), F32(-1e9)), F32(base), np.nextafter(F32(base), F32(1e9))):
            two = np.floor(F32(F32(x) * inv) + F32(0.5))
            fused = math.floor(float(F32(float(x) * float(inv) + 0.5)))
            if int(two) != fused:
                found += 1
                assert orc.cell_index(float(x), float(inv)) == int(two)
    assert found > 0, "no FMA-sensitive input found; widen the search"


def test_sort_perm_matches_lexsort(orc):
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 50, 3000).astype(np.uint32)   # many ties
    perm = orc.sort_perm(keys)
    ref = np.lexsort((np.arange(keys.size), keys)).astype(np.uint32)
    assert np.array_equal(perm, ref)


# --------------------------------------------------------------------------- #
# Contacts (Sec. II-B, II-C)
# --------------------------------------------------------------------------- #

def _pairs(res):
    off, j = res["pp_off"], res["pp_j"]
    return [tuple(j[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


@pytest.mark.parametrize("n,hsize,overlap", [(300, 0, 1.0), (1500, 0, 0.6), (800, 7, 0.5), (500, 1, 0.5),
                                             (1200, 3001, 0.4)])
def test_cell_list_equals_brute_force(orc, n, hsize, overlap):
    pr, _ = S.random_cloud(n, seed=10 + n, box=0.06, overlap=overlap)
    p = _params(hash_size=hsize)
    a = orc.contacts(pr[:, :3], pr[:, 3], [], p, brute=False)
    b = orc.contacts(pr[:, :3], pr[:, 3], [], p, brute=True)
    assert a["stats"]["n_pp"] > 0
    assert np.array_equal(a["pp_off"], b["pp_off"])
    assert np.array_equal(a["pp_j"], b["pp_j"])
    # partners ascending by id, never self
    for i, lst in enumerate(_pairs(a)):
        assert list(lst) == sorted(lst) and i not in lst


def test_lattice_cell_list_equals_brute_force(orc):
    sc = S.settle_box(n=4096, seed=1000)
    pr = sc.pos_r.copy()
    pr[:, :3] *= F32(0.93)    # squeeze so that contacts exist
    p = sc.params
    a = orc.contacts(pr[:, :3], pr[:, 3], [], p)
    b = orc.contacts(pr[:, :3], pr[:, 3], [], p, brute=True)
    assert a["stats"]["n_pp"] > 1000
    assert np.array_equal(a["pp_j"], b["pp_j"]) and np.array_equal(a["pp_off"], b["pp_off"])


def test_contacts_match_kdtree(orc):
    """Contact pairs = pairs with |x_i - x_j| <= r_i + r_j (scipy k-d tree, FP64),
    except pairs within 1e-6 relative of touching, where FP32 decides."""
    spatial = pytest.importorskip("scipy.spatial")
    pr, _ = S.random_cloud(2000, seed=77, box=0.08, overlap=0.6)
    x = pr[:, :3].astype(np.float64)
    r = pr[:, 3].astype(np.float64)
    res = orc.contacts(x, r, [], _params())
    got = set()
    for i, lst in enumerate(_pairs(res)):
        for j in lst:
            got.add((i, int(j)))
    tree = spatial.cKDTree(x)
    want, border = set(), set()
    for i, j in tree.query_pairs(2.0 * r.max() * 1.01):
        d = float(np.linalg.norm(x[i] - x[j]))
        s = r[i] + r[j]
        if abs(d - s) < 1e-6 * s:
            border |= {(i, j), (j, i)}
        elif d <= s:
            want |= {(i, j), (j, i)}
    assert len(want) > 500
    assert (got - border) == (want - border)


def test_pair_test_sums_in_the_stated_order(orc):
    """The FP32 sphere test is ((dx^2 + dy^2) + dz^2) <= (r_i + r_j)^2, one rounding
    per operation, no fused multiply-add (Sec. II-C; reading g9 family).  Search pairs
    within a few ulps of touching on which another summation order decides the other
    way; the oracle must follow the stated order, which numpy's float32 arithmetic
    evaluates here independently."""
    rng = np.random.default_rng(4)
    p = _params(cell_size=0.01)
    found = 0
    for _ in range(6000):
        ri, rj = F32(rng.uniform(1e-3, 3e-3)), F32(rng.uniform(1e-3, 3e-3))
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        xi = rng.uniform(-0.5, 0.5, 3).astype(F32)
        rs = float(ri) + float(rj)
        for k in (-2, -1, 0, 1, 2):
            xj = (xi.astype(np.float64) + rs * (1 + k * 6e-8) * u).astype(F32)
            d = [F32(xi[a] - xj[a]) for a in range(3)]
            sq = [F32(v * v) for v in d]
            stated = F32(F32(sq[0] + sq[1]) + sq[2])
            others = (F32(sq[0] + F32(sq[1] + sq[2])), F32(F32(sq[0] + sq[2]) + sq[1]))
            r2 = F32(F32(ri + rj) * F32(ri + rj))
            if all((o <= r2) == (stated <= r2) for o in others):
                continue
            found += 1
            pr = np.array([[*xi, ri], [*xj, rj]], F32)
            c = orc.contacts(pr[:, :3], pr[:, 3], [], p)
            assert (c["pp_off"][-1] == 2) == bool(stated <= r2), (xi, xj, ri, rj)
    assert found >= 10, "too few order-sensitive pairs; widen the search"


def test_contact_geometry_antisymmetric(orc):
    pr, _ = S.random_cloud(400, seed=5, box=0.04, overlap=0.5)
    res = orc.contacts(pr[:, :3], pr[:, 3], [], _params())
    off, jj, g = res["pp_off"], res["pp_j"], res["pp_geom"]
    x = pr[:, :3].astype(np.float64)
    r = pr[:, 3].astype(np.float64)
    for i in range(0, 400, 7):
        for c in range(off[i], off[i + 1]):
            j = int(jj[c])
            d = x[i] - x[j]
            dist = np.linalg.norm(d)
            assert np.allclose(g[c, :3], d / dist, atol=1e-14)
            assert abs(g[c, 3] - (r[i] + r[j] - dist)) < 1e-15
            cj = off[j] + list(jj[off[j]:off[j + 1]]).index(i)
            assert np.array_equal(g[cj, :3], -g[c, :3]) and g[cj, 3] == g[c, 3]


def test_coincident_centres_normal(orc):
    pr = np.array([[0.01, 0.01, 0.01, 0.002], [0.01, 0.01, 0.01, 0.002]], F32)
    res = orc.contacts(pr[:, :3], pr[:, 3], [], _params())
    g = res["pp_geom"]
    assert np.allclose(g[0, :3], [0, 0, -1]) and np.allclose(g[1, :3], [0, 0, 1])


# --------------------------------------------------------------------------- #
# SDF geometry (Sec. II-C, Eq. 7)
# --------------------------------------------------------------------------- #

def _box_dist_sampled(y, h, step):
    """Distance from y to the surface of the box |y_k| <= h_k, by sampling its faces."""
    best = np.inf
    for ax in range(3):
        o = [a for a in range(3) if a != ax]
        g0 = np.arange(-h[o[0]], h[o[0]] + step / 2, step)
        g1 = np.arange(-h[o[1]], h[o[1]] + step / 2, step)
        G0, G1 = np.meshgrid(g0, g1, indexing="ij")
        for s in (-1, 1):
            P = np.zeros(G0.shape + (3,))
            P[..., ax] = s * h[ax]
            P[..., o[0]] = G0
            P[..., o[1]] = G1
            best = min(best, float(np.min(np.linalg.norm(P - y, axis=-1))))
    return best


def test_box_sdf_against_sampled_surface(orc):
    rng = np.random.default_rng(3)
    h = np.array([0.03, 0.02, 0.01])
    rv = np.array([0.3, -0.2, 0.5])
    body = S.Body(kind=S.BOX, shape=tuple(h), pos=(0.1, -0.05, 0.2), quat=S._quat_from_rotvec(rv))
    q = np.array(body.quat, np.float64)
    w, xq, yq, zq = (F32(v) for v in q)
    # rotation of the float32 quaternion the oracle uses
    qq = np.array([w, xq, yq, zq], np.float64)
    qq /= np.linalg.norm(qq)
    a, b, c, d = qq
    R = np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]])
    p = np.array([F32(v) for v in body.pos], np.float64)
    hh = np.array([F32(v) for v in h], np.float64)
    step = 2e-4
    for _ in range(25):
        y = rng.uniform(-0.05, 0.05, 3)
        xw = p + R @ y
        f, nrm = orc.sdf(body, xw)
        dist = _box_dist_sampled(y, hh, step)
        inside = np.all(np.abs(y) < hh)
        assert (f < 0) == inside
        assert abs(abs(f) - dist) < step, (y, f, dist)
        assert abs(np.linalg.norm(nrm) - 1) < 1e-12
        # the normal points along the direction in which f grows
        f2, _ = orc.sdf(body, xw + 1e-7 * nrm)
        assert f2 > f


def test_box_face_tie_takes_the_lower_axis(orc):
    """Reading g14: inside a box, a point as far from an x face as from a y face takes
    the x face (ties go to the lower axis); as far from y as from z, the y face."""
    box = S.Body(kind=S.BOX, shape=(0.02, 0.02, 0.02))
    f, n = orc.sdf(box, np.array([0.015, 0.015, 0.0]))
    assert np.allclose(n, [1, 0, 0]) and abs(f + 0.005) < 1e-9
    f, n = orc.sdf(box, np.array([0.0, -0.015, -0.015]))
    assert np.allclose(n, [0, -1, 0]) and abs(f + 0.005) < 1e-9


def test_container_floor_below_its_origin(orc):
    """Reading g16: an open box's floor is at -h_z in its frame (walls at +-h_x, +-h_y):
    with h_z = 0.05 a point 4 mm above the floor is 4 mm away, normal up."""
    box = S.Body(kind=S.OPEN_BOX, shape=(0.1, 0.1, 0.05), pos=(0.0, 0.0, 0.5))
    f, n = orc.sdf(box, np.array([0.0, 0.0, 0.5 - 0.05 + 0.004]))
    assert abs(f - 0.004) < 1e-7 and np.allclose(n, [0, 0, 1])
    pr = np.array([[0.0, 0.0, 0.5 - 0.05 + 0.0049, 0.005], [0.05, 0.0, 0.5 - 0.05 + 0.03, 0.005]], F32)
    c = orc.contacts(pr[:, :3], pr[:, 3], [box], _params(cell_size=0.011))
    assert list(np.diff(c["bc_off"].astype(np.int64))) == [1, 0]       # touching; 3 cm above: free


def test_scoop_and_container_sdf_values(orc):
    scoop = S.scoop_body(1.0)
    # inside the 6 mm floor: 5 mm from the bottom face and from the cavity floor
    f, n = orc.sdf(scoop, np.array([0.0, 0.0, -0.035]))
    assert abs(f + 0.005) < 1e-9
    # origin of the tool: 3 cm above the cavity floor (z = -0.03), nearer than any wall
    f, n = orc.sdf(scoop, np.array([0.0, 0.0, 0.0]))
    assert abs(f - 0.03) < 1e-7 and np.allclose(n, [0, 0, 1])
    # 4 mm from the cavity's +y wall (at y = 0.044), 2 cm above its floor
    f, n = orc.sdf(scoop, np.array([0.0, 0.04, -0.01]))
    assert abs(f - 0.004) < 1e-7 and np.allclose(n, [0, -1, 0])
    # 4 mm from the cavity's +x and -x walls (at x = +-0.054): normals into the cavity
    f, n = orc.sdf(scoop, np.array([0.05, 0.0, -0.01]))
    assert abs(f - 0.004) < 1e-7 and np.allclose(n, [-1, 0, 0])
    f, n = orc.sdf(scoop, np.array([-0.05, 0.0, -0.01]))
    assert abs(f - 0.004) < 1e-7 and np.allclose(n, [1, 0, 0])
    # outside next to a side wall
    f, n = orc.sdf(scoop, np.array([0.07, 0.0, 0.0]))
    assert abs(f - 0.01) < 1e-7 and np.allclose(n, [1, 0, 0])
    box = S.Body(kind=S.OPEN_BOX, shape=(0.1, 0.1, 0.0), pos=(0.1, 0.1, 0.0))
    f, n = orc.sdf(box, np.array([0.03, 0.1, 0.5]))     # 3 cm from the x = 0 wall, far above the floor
    assert abs(f - 0.03) < 1e-7 and np.allclose(n, [1, 0, 0])
    f, n = orc.sdf(box, np.array([0.1, 0.1, 0.004]))    # 4 mm above the floor
    assert abs(f - 0.004) < 1e-7 and np.allclose(n, [0, 0, 1])


# --------------------------------------------------------------------------- #
# Solver and integrator: closed forms (Alg. 1, Eq. 1-5, Baumgarte)
# --------------------------------------------------------------------------- #

def _two_spheres(orc, v0, v1, m0=1.0, m1=3.0, mu=0.5, iters=20):
    # radii 0.5 and 0.25, centres 0.75 apart: exactly touching (psi = 0) in FP32 and FP64
    pr = np.array([[0.0, 0.0, 0.0, 0.5], [0.75, 0.0, 0.0, 0.25]], F32)
    vel = np.array([v0, v1], F32)
    s = orc.Sim(pr, vel, np.array([m0, m1], F32), [], _params(mu=mu, pja_iters=iters, cell_size=1.6))
    s.step(1)
    return s


def test_body_contact_point_lies_on_the_touched_face(orc):
    """Reading g18: the contact point of a body contact is x - f n, the closest point of
    the surface.  A sphere pressing 0.1 mm into the +x face of a box turned 30 degrees
    about z: the face's outward normal is R e_x, psi = r - (n . (x - p) - h), and the
    contact point is on the face plane, f = r - psi from the centre along -n."""
    th = math.radians(30.0)
    h = 0.05
    box = S.Body(kind=S.BOX, shape=(h, h, h), pos=(0.1, 0.2, 0.3),
                 quat=(math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)))
    n_w = np.array([math.cos(th), math.sin(th), 0.0])
    t_w = np.array([-math.sin(th), math.cos(th), 0.0])
    r = 0.01
    centre = np.array(box.pos) + (h + r - 1e-4) * n_w + 0.013 * t_w + np.array([0.0, 0.0, -0.007])
    pr = np.array([[*centre, r]], F32)
    s = orc.Sim(pr, np.zeros((1, 3), F32), np.array([0.01], F32), [box], _params(cell_size=0.05))
    c = s.contacts()
    assert c["bc_off"][-1] == 1
    g = c["bc_geom"][0]
    x = pr[0, :3].astype(np.float64)
    p = np.array([float(F32(v)) for v in box.pos])
    qf = np.array([float(F32(v)) for v in box.quat])
    n_f = _quat_matrix(qf)[:, 0]                                        # R e_x of the stored pose
    f = float(n_f @ (x - p)) - float(F32(h))
    assert np.allclose(g[:3], n_f, atol=1e-12)
    assert abs(g[3] - (float(F32(r)) - f)) < 1e-12
    assert np.allclose(g[4:7], x - f * n_f, atol=1e-12)
    assert abs(float(n_f @ (g[4:7] - p)) - float(F32(h))) < 1e-12         # on the face plane


def test_two_sphere_head_on_inelastic(orc):
    s = _two_spheres(orc, (1.0, 0, 0), (-0.5, 0, 0))
    vc = (1.0 * 1.0 + 3.0 * -0.5) / 4.0
    assert np.allclose(s.v[:, 0], vc, atol=1e-14, rtol=0)
    assert np.all(s.v[:, 1:] == 0)
    s.step(1)   # still touching, no approach: nothing changes
    assert np.allclose(s.v[:, 0], vc, atol=1e-14, rtol=0)


def test_two_sphere_oblique_sticks(orc):
    s = _two_spheres(orc, (1.0, 0.1, 0), (0, 0, 0))
    vcm = np.array([1.0, 0.1, 0.0], F32).astype(np.float64) * 1.0 / 4.0
    assert np.allclose(s.v, vcm[None, :], atol=1e-14)


def test_two_sphere_oblique_slides_at_mu(orc):
    mu = 0.5
    s = _two_spheres(orc, (1.0, 0.8, 0), (0, 0, 0), mu=mu)
    m = np.array([1.0, 3.0])
    dv = s.v - np.array([[1.0, 0.8, 0.0], [0.0, 0.0, 0.0]], F32).astype(np.float64)
    p_n = dv[:, 0] * m          # normal impulses
    p_t = dv[:, 1] * m          # tangential impulses
    assert abs(s.v[0, 0] - s.v[1, 0]) < 1e-14              # normal relative velocity removed
    assert np.allclose(np.abs(p_t), mu * np.abs(p_n), rtol=1e-12)
    assert s.v[0, 1] - s.v[1, 1] > 0                      # still sliding the same way


def test_resting_sphere_baumgarte_decay(orc):
    r = F32(0.005)
    for psi0 in (1e-6, 0.0):
        z0 = F32(float(r) - psi0)
        pr = np.array([[0.0, 0.0, z0, r]], F32)
        p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=20)
        s = orc.Sim(pr, np.zeros((1, 3), F32), np.array([0.01], F32), [S.Body(kind=S.PLANE)], p)
        a = float(F32(0.2))
        psi = float(r) - float(z0)
        for k in range(1, 9):
            s.step(1)
            want = (1.0 - a) ** k * psi
            assert abs((float(r) - s.x[0, 2]) - want) < 1e-15, (k, psi0)
        # the plane carries the sphere's weight once the correction has decayed
        if psi0 == 0.0:
            g = float(F32(9.81))
            m32 = float(F32(0.01))
            assert abs(s.wrench[0, 2] + m32 * g) < 1e-12 * m32 * g
            assert np.allclose(s.wrench[0, [0, 1]], 0.0, atol=1e-18)


def test_resting_sphere_torque_about_the_body_origin(orc):
    """The wrench's torque is taken about the body's position, with the lever arm from
    there to the contact point x - f n (Sec. III-C force readback; readings g18, g19):
    a sphere resting at (dx, dy) on a plane through the origin presses on it with
    F = (0, 0, -m g) at (dx, dy, 0), so tau = (dx, dy, 0) x F = (-m g dy, m g dx, 0).
    A lever arm taken the other way round, or the product in the other order, flips
    both signs."""
    r = F32(0.005)
    dx, dy = F32(0.03), F32(-0.02)
    pr = np.array([[dx, dy, r, r]], F32)
    p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=20)
    s = orc.Sim(pr, np.zeros((1, 3), F32), np.array([0.01], F32), [S.Body(kind=S.PLANE)], p)
    s.step(3)
    mg = float(F32(0.01)) * float(F32(9.81))
    want = np.array([0.0, 0.0, -mg, -mg * float(dy), mg * float(dx), 0.0])
    assert np.allclose(s.wrench[0], want, rtol=0, atol=1e-12 * mg)


def test_sphere_sticks_to_a_moving_plate(orc):
    """A kinematic body's surface velocity at a contact is v_b + w_b x (x_c - p_b)
    (reading g18, world-frame twist): a sphere resting at (dx, dy) on a plate through
    the origin that translates at v_b and spins at w_b about z is carried, after one
    step, at exactly that velocity, as long as friction can hold it (|v_s| < mu g dt:
    the first iteration removes the relative velocity, the cone keeps the impulse).
    A lever arm or a cross product the other way round, or a dropped v_b, fails it."""
    r = F32(0.005)
    dx, dy = F32(0.03), F32(-0.02)
    vb, wz = F32(1e-4), F32(0.005)
    pr = np.array([[dx, dy, r, r]], F32)
    p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=20)
    plate = S.Body(kind=S.PLANE, lin_vel=(float(vb), 0.0, 0.0), ang_vel=(0.0, 0.0, float(wz)))
    s = orc.Sim(pr, np.zeros((1, 3), F32), np.array([0.01], F32), [plate], p)
    s.step(1)
    want = np.array([float(vb) - float(wz) * float(dy), float(wz) * float(dx), 0.0])
    assert np.linalg.norm(want) < 0.5 * float(F32(9.81)) * float(F32(1e-4))   # inside the cone
    assert np.allclose(s.v[0], want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dtheta_deg", [-2.0, 2.0])
def test_block_on_incline_threshold(orc, dtheta_deg):
    """Sliding threshold tan(theta) = mu and a = g (sin theta - mu cos theta) above it."""
    mu = 0.5
    theta = math.atan(mu) + math.radians(dtheta_deg)
    quat = (math.cos(theta / 2), math.sin(theta / 2), 0.0, 0.0)   # tilt about x
    plane = S.Body(kind=S.PLANE, quat=quat)
    r = 0.005
    nrm = np.array([0.0, -math.sin(theta), math.cos(theta)])
    x0 = (r - 1e-9) * nrm          # tiny overlap so that FP32 sees the contact
    pr = np.array([[x0[0], x0[1], x0[2], r]], F32)
    p = S.Params(dt=1e-4, mu=mu, alpha=0.0, pja_iters=20)
    s = orc.Sim(pr, np.zeros((1, 3), F32), np.array([0.02], F32), [plane], p)
    s.step(1)
    # the oracle's plane normal comes from the float32 quaternion
    qf = np.array([F32(v) for v in quat], np.float64)
    qf /= np.linalg.norm(qf)
    th = 2 * math.atan2(qf[1], qf[0])
    g = float(F32(9.81))
    dt = float(F32(1e-4))
    mu32 = float(F32(mu))
    n32 = np.array([0.0, -math.sin(th), math.cos(th)])
    vt = s.v[0] - np.dot(s.v[0], n32) * n32
    assert abs(np.dot(s.v[0], n32)) < 1e-15
    if dtheta_deg < 0:
        assert np.linalg.norm(vt) < 1e-15
    else:
        want = dt * g * (math.sin(th) - mu32 * math.cos(th))
        assert abs(np.linalg.norm(vt) - want) < 1e-12 * want


def test_momentum_conserved_without_gravity(orc):
    pr, vel = S.random_cloud(300, seed=9, box=0.03, overlap=0.5, vel_scale=0.3)
    m = S.sphere_mass(pr[:, 3])
    s = orc.Sim(pr, vel, m, [], _params(mu=0.4, pja_iters=20))
    mm = s.m[:, None]
    p0 = (mm * s.v).sum(0)
    scale = (mm * np.abs(s.v)).sum()
    res = s.contacts()
    npp = int(res["pp_off"][-1])
    assert npp > 100
    lam = np.zeros((npp, 3))
    s.step(1, pp_lam=lam)
    # equal and opposite impulses on the two copies of each pair, bit for bit
    off, jj = res["pp_off"], res["pp_j"]
    for i in range(300):
        for c in range(off[i], off[i + 1]):
            j = int(jj[c])
            cj = off[j] + list(jj[off[j]:off[j + 1]]).index(i)
            assert np.array_equal(lam[cj], -lam[c])
    for _ in range(4):
        s.step(1)
    p1 = (mm * s.v).sum(0)
    assert np.all(np.abs(p1 - p0) < 1e-12 * scale)


def test_ncp_residual_decreases_with_iterations(orc):
    """The iteration's fixed point is the NCP of Eq. 1-3: the residual shrinks as I grows."""
    sc = S.settle_box(n=125, seed=1000)
    pr = S.jittered_lattice((5, 5, 5), 125, 5e-3, 0.1, 1000, origin=(0.075, 0.075, 0.0),
                            pitch=2 * 5.5e-3 * 0.985)[0]   # slightly overlapping pile
    res = []
    for it in (5, 50, 500, 5000):
        p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=it)
        s = orc.Sim(pr, np.zeros((125, 3), F32), S.sphere_mass(pr[:, 3]), sc.bodies, p)
        s.step(1)
        res.append(s.stats.ncp_residual)
    assert all(b < a for a, b in zip(res, res[1:])), res
    assert res[-1] < 1e-6, res


def test_kinematic_body_pose_closed_form(orc):
    w = 3.0
    body = S.Body(kind=S.BOX, shape=(0.01, 0.01, 0.01), pos=(0.0, 0.0, 1.0), lin_vel=(0.5, 0.0, -0.25),
                  ang_vel=(0.0, 0.0, w))
    s = orc.Sim(np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), [body], _params())
    n = 37
    s.step(n)
    dt = float(F32(1e-4))
    ang = n * dt * float(F32(w))
    pose = s.body_pose(0)
    assert np.allclose(pose[:3], [n * dt * 0.5, 0.0, 1.0 - n * dt * 0.25], atol=1e-14)
    assert np.allclose(pose[3:], [math.cos(ang / 2), 0, 0, math.sin(ang / 2)], atol=1e-14)


def test_kinematic_body_follows_its_twist_table_row_by_row(orc):
    """Reading g17: step k of a driven body uses row k of its per-step world twist table
    (its own twist once the table ends).  Rows that grow with k make the pose after n
    steps the sum of the first n rows times dt; a table read one row early or late
    moves the body by a different amount."""
    n, dt = 12, float(F32(1e-4))
    k = np.arange(n + 4, dtype=np.float64)
    tab = np.zeros((n + 4, 6), np.float32)
    tab[:, 0] = (1e-3 * (k + 1)).astype(np.float32)       # x velocity of row k
    tab[:, 5] = (0.5 * (k + 1)).astype(np.float32)        # rotation rate about z
    body = S.Body(kind=S.BOX, shape=(0.01, 0.01, 0.01), pos=(0.0, 0.0, 1.0))
    s = orc.Sim(np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), [body], _params(), twist={0: tab})
    s.step(n)
    pose = s.body_pose(0)
    x = dt * float(tab[:n, 0].astype(np.float64).sum())
    ang = dt * float(tab[:n, 5].astype(np.float64).sum())
    assert abs(pose[0] - x) < 1e-14 and abs(pose[2] - 1.0) < 1e-14
    assert np.allclose(pose[3:], [math.cos(ang / 2), 0, 0, math.sin(ang / 2)], atol=1e-14)


def _quat_mul(a, b):
    """Hamilton product a (x) b of (w, x, y, z) quaternions."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw])


def _quat_matrix(q):
    q = np.asarray(q, np.float64) / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("omega", [(0.0, 0.0, 30.0), (10.0, -20.0, 5.0)])
def test_kinematic_pose_world_frame_twist_from_tilted_start(orc, omega):
    """Sec. II: a driven body's twist lives in se(3) with its angular part in the world
    frame.  A body tilted 90 degrees about x that spins at a constant world omega has,
    after k steps, the orientation exp(k dt omega / 2) (x) q0 exactly (one axis, so the
    increments commute).  The frame mistake q0 (x) exp(...) gives another rotation
    here, which scipy's independent rotation composition tells apart."""
    from scipy.spatial.transform import Rotation
    q0 = (math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0)
    body = S.Body(kind=S.BOX, shape=(0.01, 0.01, 0.01), pos=(0.0, 0.0, 1.0), quat=q0, ang_vel=omega)
    s = orc.Sim(np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), [body], _params())
    k = 53
    s.step(k)
    dt = float(F32(1e-4))
    th = k * dt * np.array([float(F32(w)) for w in omega])
    q0f = np.array([float(F32(v)) for v in q0])
    r0 = Rotation.from_quat([q0f[1], q0f[2], q0f[3], q0f[0]])          # scipy: (x, y, z, w)
    want_world = (Rotation.from_rotvec(th) * r0).as_matrix()            # world-frame increment
    want_body = (r0 * Rotation.from_rotvec(th)).as_matrix()             # body-frame increment
    got = _quat_matrix(s.body_pose(0)[3:])
    assert np.abs(got - want_world).max() < 1e-12
    assert np.abs(want_body - want_world).max() > 1e-3                 # the two frames differ here
    # and the closed form in quaternions: exp(k dt omega / 2) (x) q0, up to sign
    ang = float(np.linalg.norm(th))
    e = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * th / ang])
    qk = _quat_mul(e, q0f / np.linalg.norm(q0f))
    assert abs(abs(float(np.dot(qk, s.body_pose(0)[3:]))) - 1.0) < 1e-12


@pytest.mark.parametrize("iters,want_a,want_b", [(1, -0.5, -1.0), (2, -5.0 / 12.0, -5.0 / 6.0)])
def test_stacked_spheres_on_a_plane_mass_split_iterates(orc, iters, want_a, want_b):
    """Mass splitting counts a body contact in n_i too (reading g3).  Sphere A rests on a
    plane, sphere B on A (both touching exactly, at rest, gravity on; equal masses).
    First sweep: the plane contact of A (n_A = 2) takes w = m / 2 of A's approach
    g dt, the A-B pair sees no relative velocity: U_A = -g dt / 2, U_B = -g dt.  Second
    sweep: the plane contact grows to 3/4 m g dt, the pair (w = 1 / (2/m + 1/m) = m/3)
    closes the relative velocity g dt / 2 by a third of it: U_A = -5/12 g dt,
    U_B = -5/6 g dt.  A body-contact weight without the count gives U_A = 0 after one
    sweep."""
    r = F32(2.0 ** -8)                                # exact: the contacts touch exactly
    pr = np.array([[0.0, 0.0, r, r], [0.0, 0.0, 3 * r, r]], F32)
    p = S.Params(dt=1e-4, gravity=(0.0, 0.0, -9.81), mu=0.5, alpha=0.2, pja_iters=iters)
    s = orc.Sim(pr, np.zeros((2, 3), F32), np.array([0.01, 0.01], F32), [S.Body(kind=S.PLANE)], p)
    s.step(1)
    gdt = float(F32(9.81)) * float(F32(1e-4))
    assert np.allclose(s.v[:, :2], 0.0, atol=1e-18)
    assert abs(s.v[0, 2] - want_a * gdt) < 1e-15 and abs(s.v[1, 2] - want_b * gdt) < 1e-15


def test_free_box_hit_from_both_sides_counts_its_contacts(orc):
    """A free body's share of the mass splitting counts its contacts this step (reading
    for free bodies: n_b (1/M + ...)).  Two equal spheres hit a free cube through its
    centre from opposite sides (gravity off, one sweep, levers parallel to the normals):
    w = 1 / (1/m + 2/M), each sphere keeps s (1 - w/m) = s/2 for M = 2m, and the cube,
    pushed equally both ways, stays at rest.  Counting one contact gives s/3."""
    h, r = 2.0 ** -5, F32(2.0 ** -8)
    m, M = 0.01, 0.02
    cube = S.Body(kind=S.BOX, shape=(h, h, h), pos=(0.0, 0.0, 0.0), is_free=1, mass=M,
                  inertia=(M * (2 * h) ** 2 / 6,) * 3)
    x0 = F32(h) + r
    pr = np.array([[-x0, 0.0, 0.0, r], [x0, 0.0, 0.0, r]], F32)
    sp = 0.2
    vel = np.array([[sp, 0.0, 0.0], [-sp, 0.0, 0.0]], F32)
    s = orc.Sim(pr, vel, np.array([m, m], F32), [cube], _params(pja_iters=1))
    s.step(1)
    sp32 = float(F32(sp))
    assert np.allclose(s.v, [[sp32 / 2, 0, 0], [-sp32 / 2, 0, 0]], rtol=0, atol=1e-15)
    assert np.allclose(s.body_twist(0), 0.0, atol=1e-15)


def test_free_body_central_hit_inelastic(orc):
    """A sphere hitting a free box through its centre: both end with m v / (m + M)."""
    M = 2.0
    cube = S.Body(kind=S.BOX, shape=(0.25, 0.25, 0.25), pos=(0.75, 0.0, 0.0), is_free=1, mass=M,
                  inertia=(M * 0.25 / 6,) * 3)
    pr = np.array([[0.0, 0.0, 0.0, 0.5]], F32)      # touching the face x = 0.5
    m = 1.0
    s = orc.Sim(pr, np.array([[1.0, 0, 0]], F32), np.array([m], F32), [cube], _params(cell_size=1.2))
    s.step(1)
    vc = m * 1.0 / (m + M)
    assert abs(s.v[0, 0] - vc) < 1e-14
    assert np.allclose(s.body_twist(0), [vc, 0, 0, 0, 0, 0], atol=1e-14)


def test_scoop_loss_limits(orc):
    """Reading g18 (loss): sum_i m_i sigmoid(-f_B(y_i) / eps) over the cavity box B
    (half extents 0.054, 0.044, 0.04 about z = 0.01 in the tool frame).  Deep inside the
    cavity a particle counts fully, far outside not at all, on the cavity's +x wall
    (f_B = 0) by half, and 5 mm below the cavity's open top (f_B = -0.005) by
    1 / (1 + e^-5); the four masses tell the terms apart."""
    scoop = S.scoop_body(1.0, pos=(0.0, 0.0, 0.0))
    pr = np.array([[0.0, 0.0, 0.01, 0.002], [0.5, 0.5, 0.5, 0.002], [0.054, 0.0, 0.01, 0.002],
                   [0.0, 0.0, 0.045, 0.002]], F32)
    s = orc.Sim(pr, np.zeros((4, 3), F32), np.array([1.0, 2.0, 4.0, 8.0], F32), [scoop], _params())
    L = s.scoop_loss(0, eps=1e-3)
    assert abs(L - (1.0 + 0.5 * 4.0 + 8.0 / (1.0 + math.exp(-5.0)))) < 1e-4


def test_mass_splitting_weight_three_in_a_row(orc):
    """Three equal touching spheres on a line, outer ones approaching the middle at v.

    One Jacobi iteration with w = 1 / (n_i/m_i + n_j/m_j) = m/3 (the middle sphere
    has two contacts) leaves the middle at rest and the outer ones at 2v/3."""
    pr = np.array([[-1.0, 0, 0, 0.5], [0.0, 0, 0, 0.5], [1.0, 0, 0, 0.5]], F32)
    vel = np.array([[1.0, 0, 0], [0, 0, 0], [-1.0, 0, 0]], F32)
    s = orc.Sim(pr, vel, np.full(3, 2.0, F32), [], _params(pja_iters=1, cell_size=2.2))
    s.step(1)
    assert np.allclose(s.v[:, 0], [2.0 / 3.0, 0.0, -2.0 / 3.0], atol=1e-15)


@pytest.mark.parametrize("iters", [1, 2, 3, 4, 5])
def test_literal_alg1_weight_two_spheres_oscillate(orc, iters):
    """Alg. 1 as printed (pja_weight = 1): each particle adds the whole projected
    correction to its own velocity (w = m_i), whatever the masses.  For two touching
    spheres approaching head-on (psi = 0, gravity off) the first iteration makes each
    take the other's normal velocity; the next finds them separating and takes the
    impulse back to zero, so the iterates alternate: after an odd number of
    iterations the velocities are exchanged, after an even number unchanged.  (With
    mass splitting they stick at the momentum-weighted mean.)"""
    pr = np.array([[0.0, 0.0, 0.0, 0.5], [1.0, 0.0, 0.0, 0.5]], F32)
    vel = np.array([[0.75, 0.1, 0.0], [-0.25, 0.0, 0.0]], F32)
    m = np.array([1.0, 3.0], F32)
    s = orc.Sim(pr, vel, m, [], _params(pja_iters=iters, pja_weight=1, mu=0.0, cell_size=1.2))
    s.step(1)
    want = vel.astype(np.float64)
    if iters % 2:
        want[0, 0], want[1, 0] = want[1, 0], want[0, 0]      # normal components exchanged
    assert np.abs(s.v - want).max() < 1e-14, (iters, s.v)


@pytest.mark.parametrize("iters", [1, 3])
def test_literal_alg1_weight_three_in_a_row(orc, iters):
    """Alg. 1 as printed on three equal touching spheres in a row, the outer ones
    approaching the middle at v: each outer sphere removes its whole approach speed
    (stops), the middle takes +v from one side and -v from the other (stays): all at
    rest after the first iteration, and later iterations find nothing to correct.
    (Mass splitting gives 2v/3, 0, -2v/3 after one iteration.)"""
    pr = np.array([[-1.0, 0, 0, 0.5], [0.0, 0, 0, 0.5], [1.0, 0, 0, 0.5]], F32)
    vel = np.array([[1.0, 0, 0], [0, 0, 0], [-1.0, 0, 0]], F32)
    s = orc.Sim(pr, vel, np.full(3, 2.0, F32), [], _params(pja_iters=iters, pja_weight=1, cell_size=2.2))
    s.step(1)
    assert np.abs(s.v).max() < 1e-15


@pytest.mark.parametrize("iters", [1, 2])
def test_literal_alg1_weight_body_contact(orc, iters):
    """Alg. 1 as printed with a body: the particle takes the whole correction of its
    body contact too (w = m_i).  A sphere touching a plane (psi = 0) and touching a
    second, equal sphere on top, at rest with gravity on: each sweep the bottom sphere
    cancels its plane approach g dt in full and the pair sees no relative velocity in
    the first sweep: after one sweep U_bottom = 0, U_top = -g dt.  In the second the
    pair's approach g dt is corrected in full by each side (the bottom moves down by
    g dt, the top up by g dt), and the plane contact keeps its impulse: U_bottom = -g dt,
    U_top = 0."""
    r = F32(2.0 ** -8)
    pr = np.array([[0.0, 0.0, r, r], [0.0, 0.0, 3 * r, r]], F32)
    p = S.Params(dt=1e-4, gravity=(0.0, 0.0, -9.81), mu=0.5, alpha=0.2, pja_iters=iters, pja_weight=1)
    s = orc.Sim(pr, np.zeros((2, 3), F32), np.array([0.01, 0.01], F32), [S.Body(kind=S.PLANE)], p)
    s.step(1)
    gdt = float(F32(9.81)) * float(F32(1e-4))
    want = (0.0, -gdt) if iters == 1 else (-gdt, 0.0)
    assert abs(s.v[0, 2] - want[0]) < 1e-15 and abs(s.v[1, 2] - want[1]) < 1e-15


def test_literal_alg1_weight_rejects_free_bodies(orc):
    cube = S.Body(kind=S.BOX, shape=(0.25, 0.25, 0.25), pos=(0.75, 0.0, 0.0), is_free=1, mass=2.0,
                  inertia=(0.1,) * 3)
    s = orc.Sim(np.array([[0.0, 0.0, 0.0, 0.5]], F32), np.zeros((1, 3), F32), np.array([1.0], F32), [cube],
                _params(pja_weight=1, cell_size=1.2))
    with pytest.raises(RuntimeError):
        s.step(1)


def test_free_body_angular_momentum_frictionless(orc):
    """Off-centre frictionless hits on a free box conserve linear and angular momentum
    (impulses act along the normal through both contact points)."""
    M = 3.0
    h = (0.3, 0.2, 0.25)
    I = tuple(M / 3.0 * (h[(k + 1) % 3] ** 2 + h[(k + 2) % 3] ** 2) for k in range(3))
    q = S._quat_from_rotvec((0.2, -0.3, 0.1))
    cube = S.Body(kind=S.BOX, shape=h, pos=(0.0, 0.0, 0.0), quat=q, is_free=1, mass=M, inertia=I)
    pr = np.array([[0.25, 0.1, 0.4, 0.2], [-0.35, 0.05, -0.1, 0.15]], F32)
    vel = np.array([[0.0, -0.2, -1.0], [1.0, 0.3, 0.0]], F32)
    m = np.array([0.5, 0.7], F32)
    s = orc.Sim(pr, vel, m, [cube], _params(mu=0.0, alpha=0.0, cell_size=1.0))
    assert s.contacts()["bc_off"][-1] == 2

    def momenta():
        o = s.bodies[0]
        R = _rot(np.array(list(o.quat)))
        Iw = R @ np.diag(list(o.inertia)) @ R.T
        P = (s.m[:, None] * s.v).sum(0) + M * np.array(list(o.lin_vel))
        L = (np.cross(s.x, s.m[:, None] * s.v)).sum(0) + np.cross(np.array(list(o.pos)), M * np.array(list(o.lin_vel)))
        L = L + Iw @ np.array(list(o.ang_vel))
        return P, L

    P0, L0 = momenta()
    s.step(1)
    # the integrator moved x and p with the new velocities: compare momenta of the
    # post-solve velocities at the pre-step positions instead
    o = s.bodies[0]
    s.x -= float(F32(1e-4)) * s.v
    p_new = np.array(list(o.pos)) - float(F32(1e-4)) * np.array(list(o.lin_vel))
    R = _rot(np.array(list(o.quat)))
    # orientation change of one step rotates the inertia by ~dt*omega; undo it exactly
    q_prev = np.array(list(cube.quat), F32).astype(np.float64)
    Rp = _rot(q_prev)
    Iw = Rp @ np.diag(list(o.inertia)) @ Rp.T
    P1 = (s.m[:, None] * s.v).sum(0) + M * np.array(list(o.lin_vel))
    L1 = (np.cross(s.x, s.m[:, None] * s.v)).sum(0) + np.cross(p_new, M * np.array(list(o.lin_vel)))
    L1 = L1 + Iw @ np.array(list(o.ang_vel))
    assert np.abs(P1 - P0).max() < 1e-13
    assert np.abs(L1 - L0).max() < 1e-13
    assert np.abs(np.array(list(o.ang_vel))).max() > 1e-3     # the hits did spin the box


def _rot(q):
    q = q / np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]])


def test_free_box_rests_on_plane(orc):
    """A free box whose four bottom corners touch a plane: the corner contacts carry
    its weight (the solve converges to zero velocity and the plane feels M g)."""
    M = 0.5
    hs = 0.05
    cube = S.Body(kind=S.BOX, shape=(hs, hs, hs), pos=(0.0, 0.0, hs), is_free=1, mass=M,
                  inertia=(M * (2 * hs) ** 2 / 6,) * 3)
    s = orc.Sim(np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), [S.Body(kind=S.PLANE), cube],
                S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=200))
    s.step(1)
    g = float(F32(9.81))
    assert s.stats.n_corner == 4
    assert np.abs(s.body_twist(1)).max() < 1e-9 * g
    assert abs(s.wrench[0, 2] + float(F32(M)) * g) < 1e-9 * M * g


def test_tilted_free_box_on_its_lowest_edge(orc):
    """A free box turned 30 degrees about x stands on the plane with its two lowest
    corners (those at -y, -z in its frame: world y = h (sin - cos), z = 0).  Those two
    corners, and only they, are the corner contacts; after the solve their velocities
    do not point into the plane (the contact condition), whatever the box does about
    the edge."""
    M, h, th = 0.5, 0.05, math.radians(30.0)
    q = (math.cos(th / 2), math.sin(th / 2), 0.0, 0.0)
    box = S.Body(kind=S.BOX, shape=(h, h, h), pos=(0.0, 0.0, h * (math.sin(th) + math.cos(th))), quat=q,
                 is_free=1, mass=M, inertia=(M * (2 * h) ** 2 / 6,) * 3)
    s = orc.Sim(np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), [S.Body(kind=S.PLANE), box],
                S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=200))
    pose0 = s.body_pose(1)
    s.step(1)
    assert s.stats.n_corner == 2
    R = _quat_matrix(pose0[3:])
    tw = s.body_twist(1)
    for sx in (-1.0, 1.0):
        rc = R @ np.array([sx * h, -h, -h])
        assert abs(pose0[2] + rc[2]) < 1e-6                    # on the plane
        vc = tw[:3] + np.cross(tw[3:], rc)
        assert vc[2] > -1e-9, vc                               # not moving into it


def test_free_box_corners_ignore_other_free_boxes(orc):
    """Reading for free bodies: box corners are tested as points against the bodies that
    are not free; a free box's corner inside another free box makes no contact."""
    M, h = 0.5, 0.05
    inert = (M * (2 * h) ** 2 / 6,) * 3
    a = S.Body(kind=S.BOX, shape=(h, h, h), pos=(0.0, 0.0, 0.0), is_free=1, mass=M, inertia=inert)
    b = S.Body(kind=S.BOX, shape=(h, h, h), pos=(0.09, 0.09, 0.09), is_free=1, mass=M, inertia=inert)
    s = orc.Sim(np.zeros((0, 4), F32), np.zeros((0, 3), F32), np.zeros(0, F32), [a, b], _params())
    s.step(1)
    assert s.stats.n_corner == 0
    assert np.allclose(s.body_twist(0), 0.0) and np.allclose(s.body_twist(1), 0.0)


def test_fast_remainder_identity():
    """The step kernels compute Eq. 6's `mod n_h` without a division (Lemire, Kaser &
    Kurz 2019): low = magic * x mod 2^64, result = high 64 bits of low * d, with
    magic = floor((2^64 - 1) / d) + 1.  The identity is exact for all 32-bit x, d."""
    rng = np.random.default_rng(11)
    M64 = (1 << 64) - 1
    for d in [1, 2, 3, 7, 97, 4096, 524288, 1000003, 14_000_000, (1 << 31) + 11, (1 << 32) - 1] + \
            [int(v) for v in rng.integers(1, 1 << 32, 200)]:
        magic = (M64 // d + 1) & M64
        for x in [0, 1, d - 1, d, (1 << 32) - 1] + [int(v) for v in rng.integers(0, 1 << 32, 50)]:
            x &= (1 << 32) - 1
            low = (magic * x) & M64
            assert (low * d) >> 64 == x % d, (x, d)


# --------------------------------------------------------------------------- #
# gridded SDF (Sec. II-C: samples on a regular grid, trilinear interpolation)
# --------------------------------------------------------------------------- #

def _grid_body(f, origin, h, dims, pos=(0.0, 0.0, 0.0), quat=(1.0, 0.0, 0.0, 0.0)):
    """GRID body sampling f (body frame, vectorised over (..., 3)) at origin + h (i, j, k)."""
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    y = np.stack([origin[0] + h * i, origin[1] + h * j, origin[2] + h * k], axis=-1)
    vals = f(y).astype(F32)
    return S.Body(kind=S.GRID, pos=pos, quat=quat, grid=S.Grid(vals, origin, h))


def test_grid_sdf_exact_on_linear_fields(orc):
    """Trilinear interpolation reproduces a linear function exactly (dyadic samples,
    exact in float32), and its unit gradient is the field's direction."""
    rng = np.random.default_rng(11)
    for a, c in (((0.25, -0.5, 0.75), 0.125), ((0.0, 0.0, 1.0), -0.0625), ((-1.0, 0.5, 0.0), 0.25)):
        a = np.array(a)
        body = _grid_body(lambda y: y @ a + c, (-0.5, -0.25, -0.125), 1.0 / 64, (65, 33, 17))
        for _ in range(40):
            y = rng.uniform([-0.49, -0.24, -0.12], [0.49, 0.24, 0.124])
            f, n = orc.sdf(body, y)
            assert abs(f - (y @ a + c)) < 1e-12, (y, f)
            assert np.allclose(n, a / np.linalg.norm(a), atol=1e-12)


def test_grid_sdf_interpolates_its_samples(orc):
    """At the sample points the interpolant equals the samples, which for a baked box
    are the box's closed-form SDF rounded to float32; a rotated, translated body is
    queried in its own frame."""
    h = 1.0 / 128
    half = np.array([0.03, 0.02, 0.01])

    def box(y):
        q = np.abs(y) - half
        return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(q.max(axis=-1), 0.0)

    origin = (-0.0625, -0.046875, -0.03125)
    dims = (17, 13, 9)
    rv = np.array([0.2, -0.1, 0.3])
    body = _grid_body(box, origin, h, dims, pos=(0.25, -0.125, 0.5), quat=S._quat_from_rotvec(rv))
    qq = np.array([F32(v) for v in body.quat], np.float64)
    qq /= np.linalg.norm(qq)
    a_, b_, c_, d_ = qq
    R = np.array([[1 - 2 * (c_ * c_ + d_ * d_), 2 * (b_ * c_ - a_ * d_), 2 * (b_ * d_ + a_ * c_)],
                  [2 * (b_ * c_ + a_ * d_), 1 - 2 * (b_ * b_ + d_ * d_), 2 * (c_ * d_ - a_ * b_)],
                  [2 * (b_ * d_ - a_ * c_), 2 * (c_ * d_ + a_ * b_), 1 - 2 * (b_ * b_ + c_ * c_)]])
    p = np.array([F32(v) for v in body.pos], np.float64)
    rng = np.random.default_rng(12)
    for _ in range(30):
        i, j, k = rng.integers(0, dims[0]), rng.integers(0, dims[1]), rng.integers(0, dims[2])
        y = np.array([origin[0] + h * i, origin[1] + h * j, origin[2] + h * k])
        f, _ = orc.sdf(body, p + R @ y)
        assert abs(f - float(body.grid.values[k, j, i])) < 1e-9
        assert abs(f - box(y)) < 1e-7


def test_grid_sdf_error_within_trilinear_bound(orc):
    """For f with bounded second derivatives the trilinear interpolant errs by at most
    (h^2 / 8) (|f_xx| + |f_yy| + |f_zz|); for a sphere's SDF |y| - R that is
    3 h^2 / (8 rho) at distance rho >= rho_min from the centre.  Halving h must cut the
    error by about four."""
    Rs = 0.05

    def sph(y):
        return np.linalg.norm(y, axis=-1) - Rs

    rng = np.random.default_rng(13)
    pts = rng.normal(size=(300, 3))
    pts = pts / np.linalg.norm(pts, axis=1)[:, None] * rng.uniform(0.04, 0.07, (300, 1))
    errs, nerrs = [], []
    for h in (1.0 / 64, 1.0 / 128):
        n = int(round(0.16 / h)) + 1
        body = _grid_body(sph, (-0.08, -0.08, -0.08), h, (n, n, n))
        e = ne = 0.0
        for y in pts:
            f, nrm = orc.sdf(body, y)
            rho = np.linalg.norm(y)
            err = abs(f - sph(y))
            assert err <= 3 * h * h / (8 * 0.03) + 1e-7, (h, err)   # cell corners within 0.03 of the centre at most
            e = max(e, err)
            ne = max(ne, np.linalg.norm(nrm - y / rho))
        errs.append(e)
        nerrs.append(ne)
    assert errs[1] < errs[0] / 3.0          # second order in h
    assert nerrs[1] < nerrs[0] / 1.7        # the normal: first order
    assert nerrs[1] < 0.15


def test_grid_sdf_on_its_last_samples(orc):
    """The last cell along an axis ends on the last sample: a point exactly on the top
    corner of the sampled box, or on its upper faces, takes the last cell (i = n - 2,
    t = 1) and returns the sample there."""
    a, c = np.array([0.25, -0.5, 0.75]), 0.125
    o, h, dims = (-0.5, -0.25, -0.125), 1.0 / 64, (65, 33, 17)
    body = _grid_body(lambda y: y @ a + c, o, h, dims)
    top = np.array([o[k] + h * (dims[k] - 1) for k in range(3)])
    for y in (top, np.array([top[0], 0.0, 0.0]), np.array([0.0, top[1], 0.0]), np.array([0.0, 0.0, top[2]])):
        f, n = orc.sdf(body, y)
        assert abs(f - (y @ a + c)) < 1e-12, y
        assert np.allclose(n, a / np.linalg.norm(a), atol=1e-12), y     # the last cell's own gradient


def test_grid_outside_the_samples_is_not_in_contact(orc):
    body = _grid_body(lambda y: y[..., 2], (-0.09375, -0.09375, -0.09375), 1.0 / 32, (7, 7, 7))
    f, _ = orc.sdf(body, np.array([0.0, 0.0, 0.0]))
    assert abs(f) < 1e-12
    for y in ([0.2, 0.0, 0.0], [0.0, -0.11, 0.0], [0.0, 0.0, 0.095]):
        f, _ = orc.sdf(body, np.array(y))
        assert f == math.inf


def test_sphere_rests_on_a_grid_plane(orc):
    """A sphere resting on a GRID body that samples the plane z = 0 behaves as on the
    closed-form plane: penetration decays as (1 - alpha)^k (Baumgarte, Sec. II-A)."""
    r = F32(0.005)
    ground = _grid_body(lambda y: y[..., 2], (-0.0625, -0.0625, -0.0625), 1.0 / 64, (9, 9, 9))
    psi0 = 1e-6
    z0 = F32(float(r) - psi0)
    pr = np.array([[0.01, -0.02, z0, r]], F32)
    p = S.Params(dt=1e-4, mu=0.5, alpha=0.2, pja_iters=20)
    s = orc.Sim(pr, np.zeros((1, 3), F32), np.array([0.01], F32), [ground], p)
    a = float(F32(0.2))
    psi = float(r) - float(z0)
    for k in range(1, 9):
        s.step(1)
        want = (1.0 - a) ** k * psi
        assert abs((float(r) - s.x[0, 2]) - want) < 1e-13, k


def test_cyclic_vertical_boundary_free_fall(orc):
    """Cyclic boundary of the gear tower (Sec. III): a free-falling sphere leaving
    through the bottom re-enters at the top with the same velocity.  Symplectic Euler
    from rest: v_k = -k g dt, z_k = z_0 - g dt^2 k (k + 1) / 2, then wrapped into the
    period [lo, hi)."""
    lo, hi = 0.0, 0.0625
    p = S.Params(dt=1e-3, mu=0.5, pja_iters=5, cyclic_z=(lo, hi))
    z0 = F32(0.05)
    s = orc.Sim(np.array([[0.0, 0.0, z0, 0.001]], F32), np.zeros((1, 3), F32), np.array([1e-3], F32), [], p)
    g, dt = float(F32(9.81)), float(F32(1e-3))
    wrapped = 0
    z = float(z0)
    for k in range(1, 301):
        s.step(1)
        v = -k * g * dt
        z = z + dt * v
        if z < lo:
            z += hi - lo
            wrapped += 1
        assert abs(s.v[0, 2] - v) < 1e-12
        assert abs(s.x[0, 2] - z) < 1e-12, (k, s.x[0, 2], z)
    assert wrapped >= 3


def test_tube_sdf_values(orc):
    """Inside of a vertical cylinder of radius R (the gear tower's wall): f = R - rho,
    normal towards the axis, independent of height."""
    tube = S.Body(kind=S.TUBE, shape=(0.0625,), pos=(0.25, -0.125, 0.0))
    for y, want in (((0.0, 0.0, 0.3), 0.0625), ((0.05, 0.0, -1.0), 0.0125), ((0.0, -0.06, 0.0), 0.0025),
                    ((0.03, 0.04, 0.7), 0.0125)):
        x = np.array(y) + np.array([0.25, -0.125, 0.0])
        f, n = orc.sdf(tube, x)
        assert abs(f - want) < 1e-12
        rho = math.hypot(y[0], y[1])
        if rho > 0:
            assert np.allclose(n, [-y[0] / rho, -y[1] / rho, 0.0], atol=1e-12)


def test_tube_contacts_only_at_the_wall(orc):
    """The FP32 contact test of the tube wall (f = R - rho <= r): a sphere touching the
    wall from inside has one body contact, normal towards the axis; spheres near the axis
    or half a radius from the wall have none."""
    R = 0.0625
    tube = S.Body(kind=S.TUBE, shape=(R,))
    r = 0.004
    pr = np.array([[R - 0.9 * r, 0.0, 0.1, r], [0.0, 0.0, 0.2, r], [0.0, -(R - 1.5 * r), 0.3, r]], F32)
    c = orc.contacts(pr[:, :3], pr[:, 3], [tube], _params(cell_size=0.009))
    assert list(np.diff(c["bc_off"].astype(np.int64))) == [1, 0, 0]
    assert np.allclose(c["bc_geom"][0, :3], [-1, 0, 0], atol=1e-12)
    assert abs(c["bc_geom"][0, 3] - (float(F32(r)) - (R - float(F32(R - 0.9 * r))))) < 1e-12


# --------------------------------------------------------------------------- #
# depth observations (Sec. III-A sky and ego cameras)
# --------------------------------------------------------------------------- #

def test_height_camera_single_sphere(orc):
    """Orthographic height map of one sphere: z + sqrt(r^2 - d^2) at the pixel centres
    it covers (d = horizontal distance), `empty` elsewhere."""
    cam = S.Camera(kind=S.HEIGHT_CAMERA, width=16, height=8, pos=(0.0, 0.0, 0.0), extent=(0.032, 0.016),
                   empty=-1.0)
    x = np.array([[0.0011, -0.0007, 0.02]])
    r = np.array([0.005])
    img = orc.render(cam, x, r, [])
    covered = 0
    for v in range(8):
        for u in range(16):
            # pixel centres are float32 values (the camera's sample points)
            px = float(F32(F32(-0.016) + F32(F32(u + 0.5) * F32(F32(0.032) / F32(16)))))
            py = float(F32(F32(-0.008) + F32(F32(v + 0.5) * F32(F32(0.016) / F32(8)))))
            d2 = (x[0, 0] - px) ** 2 + (x[0, 1] - py) ** 2
            if d2 < r[0] ** 2 * (1 - 1e-5):
                assert abs(img[v, u] - (0.02 + math.sqrt(r[0] ** 2 - d2))) < 1e-9
                covered += 1
            elif d2 > r[0] ** 2 * (1 + 1e-5):
                assert img[v, u] == -1.0
    assert covered > 10


def test_height_camera_pixel_pitch_per_axis(orc):
    """Non-square pixels (0.002 m wide, 0.001 m tall): a sphere of 1.5 mm radius at
    (0.0001, 0.0045) over a 16 x 16 map of a 0.032 x 0.016 rectangle (pixel centres
    x = -0.015 + 0.002 u, y = -0.0075 + 0.001 v) covers the two columns u = 7, 8
    (x = -0.001, 0.001: 1.1 and 0.9 mm away) and in them the rows whose centre is
    within sqrt(r^2 - dx^2) (1.02 and 1.2 mm) of y = 0.0045: v = 11, 12, 13."""
    cam = S.Camera(kind=S.HEIGHT_CAMERA, width=16, height=16, pos=(0.0, 0.0, 0.0), extent=(0.032, 0.016),
                   empty=-1.0)
    img = orc.render(cam, np.array([[0.0001, 0.0045, 0.02]]), np.array([0.0015]), [])
    rows = sorted({v for v in range(16) for u in range(16) if img[v, u] != -1.0})
    assert rows == [11, 12, 13]
    assert all(sorted(u for u in range(16) if img[v, u] != -1.0) == [7, 8] for v in rows)


def test_height_camera_takes_the_highest_surface(orc):
    cam = S.Camera(kind=S.HEIGHT_CAMERA, width=4, height=4, pos=(0.0, 0.0, 0.0), extent=(0.008, 0.008))
    x = np.array([[0.001, 0.001, 0.01], [0.001, 0.001, 0.013], [0.001, 0.001, 0.004]])
    r = np.array([0.002, 0.002, 0.002])
    img = orc.render(cam, x, r, [])
    assert abs(img[2, 2] - (0.013 + 0.002)) < 1e-12   # pixel centre (0.001, 0.001): right above all three


def test_depth_camera_sphere_and_plane(orc):
    """Pinhole camera 0.5 m above a floor plane looking straight down: per pixel the
    ray distance to the plane is 0.5 / (d . -z); a sphere on the axis shows its near
    surface 0.5 - z_c - r away at the centre pixels; a distance beyond `far` clips."""
    down = S._quat_from_rotvec((math.pi, 0.0, 0.0))   # camera z (forward) -> world -z
    cam = S.Camera(kind=S.DEPTH_CAMERA, width=12, height=10, pos=(0.0, 0.0, 0.5), quat=down, fov_y=0.8,
                   near=0.01, far=2.0, march_steps=200, march_eps=1e-6)
    floor = S.Body(kind=S.PLANE)
    img = orc.render(cam, np.zeros((0, 3)), np.zeros(0), [floor])
    f = 0.5 * 10 / math.tan(0.4)
    for v in range(10):
        for u in range(12):
            dx, dy = (u + 0.5 - 6) / f, (v + 0.5 - 5) / f
            t = 0.5 * math.sqrt(dx * dx + dy * dy + 1.0)   # the ray's z component is -1/|(dx, dy, 1)|
            assert abs(img[v, u] - t) < 2e-6, (u, v, img[v, u], t)
    img = orc.render(cam, np.array([[0.0, 0.0, 0.1]]), np.array([0.05]), [floor])
    # a sphere below the camera: ray (dx, -dy, -1) / n from (0, 0, 0.5) meets the sphere
    # of radius 0.05 about (0, 0, 0.1) at t = b - sqrt(b^2 - 0.4^2 + 0.05^2), b = 0.4 / n
    hits = 0
    for v in range(10):
        for u in range(12):
            dx, dy = (u + 0.5 - 6) / f, (v + 0.5 - 5) / f
            nrm = math.sqrt(dx * dx + dy * dy + 1.0)
            b = 0.4 / nrm
            disc = b * b - 0.4 ** 2 + 0.05 ** 2
            if disc > 1e-6:
                assert abs(img[v, u] - (b - math.sqrt(disc))) < 1e-6
                hits += 1
            elif disc < -1e-6:
                assert abs(img[v, u] - 0.5 * nrm) < 2e-6
    assert hits >= 4
    far = S.Camera(kind=S.DEPTH_CAMERA, width=4, height=4, pos=(0.0, 0.0, 5.0), quat=down, fov_y=0.5, far=2.0)
    assert np.all(orc.render(far, np.zeros((0, 3)), np.zeros(0), [floor]) == 2.0)


def test_depth_camera_axes_and_near_clip(orc):
    """Reading g25: camera x right, y down, z forward.  With the camera frame equal to
    the world's, a sphere at world +y (camera down) lands in the lower rows and one at
    world +x in the right columns; a sphere whose near surface is closer than `near`
    is not seen."""
    cam = S.Camera(kind=S.DEPTH_CAMERA, width=20, height=20, fov_y=0.8, near=0.01, far=2.0)
    f = 0.5 * 20 / math.tan(0.4)
    img = orc.render(cam, np.array([[0.0, 0.15, 1.0]]), np.array([0.05]), [])
    rows = {v for v in range(20) for u in range(20) if img[v, u] < 2.0}
    assert rows and min(rows) >= 10 and abs(np.mean(sorted(rows)) - (10 + f * 0.15)) < 1.5
    img = orc.render(cam, np.array([[0.15, 0.0, 1.0]]), np.array([0.05]), [])
    cols = {u for v in range(20) for u in range(20) if img[v, u] < 2.0}
    assert cols and min(cols) >= 10
    img = orc.render(cam, np.array([[0.0, 0.0, 0.03]]), np.array([0.025]), [])
    assert np.all(img == 2.0)                      # near surface 5 mm away: clipped


def test_depth_camera_traces_a_box_and_a_grid_box_alike(orc):
    """Sphere tracing a closed-form box and the same box baked onto a grid (outside the
    samples the tracing steps by the distance to the sampled box) gives the same face
    distance, 0.3 - 0.05 along the optical axis."""
    half = (0.05, 0.04, 0.03)
    box = S.Body(kind=S.BOX, shape=half)

    def f(y):
        q = np.abs(y) - np.array(half)
        return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(q.max(axis=-1), 0.0)

    grid = S.Body(kind=S.GRID, grid=S.bake_grid(f, (-0.0625, -0.0625, -0.0625), (0.0625, 0.0625, 0.0625), 1.0 / 256))
    look = S._quat_from_rotvec((0.0, -math.pi / 2, 0.0))  # camera z (forward) -> world -x
    cam = S.Camera(kind=S.DEPTH_CAMERA, width=6, height=6, pos=(0.3, 0.0, 0.0), quat=look, fov_y=0.2,
                   march_steps=300, march_eps=1e-6)
    a = orc.render(cam, np.zeros((0, 3)), np.zeros(0), [box])
    b = orc.render(cam, np.zeros((0, 3)), np.zeros(0), [grid])
    fz = 0.5 * 6 / math.tan(0.1)
    dx = 0.5 / fz
    want = 0.25 * math.sqrt(1 + 2 * dx * dx)   # pixel (2, 2)/(3, 3): the rays next to the axis hit x = 0.05
    assert abs(a[2, 2] - want) < 1e-5 and abs(a[3, 3] - want) < 1e-5
    assert np.allclose(a, b, atol=1e-5)
