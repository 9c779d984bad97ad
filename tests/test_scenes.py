"""Seeded input generators: shapes and recipes of the workloads (no GPU)."""
import numpy as np

from paper_2306_01369_gb300 import scenes as S


def test_splitmix64_reference_values():
    # splitmix64 seeded with 0: first outputs from the published algorithm (Steele et al. 2014)
    z = S.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_lattice_has_no_initial_overlap():
    pr, pitch = S.jittered_lattice((8, 8, 8), 512, 2e-3, 0.15, 7)
    x = pr[:, :3].astype(np.float64)
    r = pr[:, 3].astype(np.float64)
    d = np.linalg.norm(x[:, None] - x[None], axis=-1) - (r[:, None] + r[None])
    np.fill_diagonal(d, 1.0)
    assert d.min() > 0
    assert r.min() >= 2e-3 * 0.85 - 1e-9 and r.max() <= 2e-3 * 1.15 + 1e-9


def test_batched_scene_recipe():
    sc = S.batched_beds(n_envs=256, n_steps=2)
    ne = np.diff(sc.env_offsets.astype(np.int64))
    assert len(ne) == 256 and ne.min() >= 8192 and ne.max() <= 65536
    assert 6.0e6 < sc.n < 8.5e6
    assert len(sc.body_offsets) == 257 and len(sc.bodies) == 512


def test_column_recipe():
    sc = S.column_collapse(n_steps=1)
    assert sc.n == 262144 and sc.info["dims"] == (40, 40, 164)
    assert abs(sc.info["pitch"] - 4.488e-3) < 1e-9
    assert sc.params.dt == 5e-5 and sc.params.pja_iters == 20 and sc.params.mu == 0.6


def test_pile_statistics_recovers_a_cone():
    """The repose-angle measure of the long-run statistics test, on a solid cone of
    known base angle filled uniformly with points.  Below a surface of height H(r) the
    95th percentile of z is 0.95 H(r), so the measure must return atan(0.95 tan(angle));
    the centre of mass must sit h/4 above the base (closed form)."""
    from paper_2306_01369_gb300.stats import pile_statistics
    rng = np.random.default_rng(7)
    for deg in (10.0, 25.0, 35.0):
        R = 0.2
        h = R * np.tan(np.radians(deg))
        p = rng.uniform([-R, -R, 0], [R, R, h], (400000, 3))
        p = p[p[:, 2] <= h * (1 - np.hypot(p[:, 0], p[:, 1]) / R)]
        angle, com, nb = pile_statistics(p, np.ones(len(p)), 0.002)
        assert nb >= 10
        want = np.degrees(np.arctan(0.95 * np.tan(np.radians(deg))))
        assert abs(angle - want) < 0.3, (angle, want)
        assert abs(com[2] - h / 4) < 0.01 * h


def test_pile_column_members_differ_by_one_ulp():
    base = S.pile_column(-1, n=2048, dims=(8, 8, 32))
    for k in (0, 5):
        m = S.pile_column(k, n=2048, dims=(8, 8, 32))
        sel = np.arange(base.n) % 8 == k
        assert np.array_equal(m.pos_r[~sel], base.pos_r[~sel])
        assert np.array_equal(m.pos_r[sel, 1:], base.pos_r[sel, 1:])
        assert np.array_equal(m.pos_r[sel, 0], np.nextafter(base.pos_r[sel, 0], np.float32(np.inf)))
    assert base.params.mu == np.float32(0.2) or abs(base.params.mu - 0.2) < 1e-7
