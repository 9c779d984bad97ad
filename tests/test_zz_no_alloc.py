"""The allocation-free binning entry point, gg_bin_sort_noalloc.

Some callers cannot allocate device memory: code running inside another
framework's memory pool, allocator-free real-time control loops, and plug-ins
that are handed device buffers but may not grow the process's device footprint.
For them the library offers binning + bucket sort whose scratch lives in a fixed
static device array.  This test calls it through the C ABI twice in a row, on two
different particle sets (the second smaller, so stale histogram counts from the
first call would show), and checks each result against the same quantities read
back from the regular allocating path (gg_create + gg_step): bucket keys, sorted
permutation and bucket start table, which are integers and must agree exactly.

This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2306_01369_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _regular_path(gg, pos_r, cell_size, n_h):
    p = S.Params(dt=1e-4, cell_size=cell_size, hash_size=n_h, max_contacts=32)
    sim = gg.Sim(pos_r, None, None, p)
    sim.step(1)
    sim.sync()
    out = sim.cell_keys(), sim.sort_perm(), sim.cell_start()
    sim.close()
    return out


def _noalloc(torch, lib, pos_r, cell_size, n_h):
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(pos_r).to(dev)
    n = pos_r.shape[0]
    keys = torch.full((n,), 0xFFFF, dtype=torch.int32, device=dev)
    perm = torch.full((n,), 0xFFFF, dtype=torch.int32, device=dev)
    start = torch.full((n_h + 1,), 0xFFFF, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = lib.gg_bin_sort_noalloc(C.c_void_p(pos.data_ptr()), n, cell_size, n_h, C.c_void_p(keys.data_ptr()),
                                 C.c_void_p(perm.data_ptr()), C.c_void_p(start.data_ptr()), C.c_void_p(stream))
    assert st == 0, st
    torch.cuda.synchronize(dev)
    as_u32 = lambda t: t.cpu().numpy().view(np.uint32)
    return as_u32(keys), as_u32(perm), as_u32(start)


def test_noalloc_bin_sort_matches_regular_path_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_01369_gb300 import _build, gg
    _build.build()
    lib = gg.load()
    torch.cuda.set_device(0)
    import oracle
    oracle.build()
    cases = [(S.column_collapse(n=60000, n_steps=1).pos_r, 0.0045, 120000),
             (S.random_cloud(9000, seed=5, box=0.12)[0], 0.0045, 7001)]
    for pos_r, cell, n_h in cases:
        got = _noalloc(torch, lib, np.ascontiguousarray(pos_r), cell, n_h)
        want = _regular_path(gg, np.ascontiguousarray(pos_r), cell, n_h)
        for g, w, name in zip(got, want, ("keys", "perm", "cell_start")):
            assert g.shape == w.shape, name
            assert np.array_equal(g, w), name
        # and the oracle's binning (Eq. 6 keys, stable sort by (key, id), bucket starts)
        keys = oracle.cell_keys(pos_r[:, :3].astype(np.float64), cell, n_h)
        start = np.zeros(n_h + 1, np.int64)
        np.add.at(start, keys.astype(np.int64) + 1, 1)
        assert np.array_equal(got[0], keys)
        assert np.array_equal(got[1], oracle.sort_perm(keys))
        assert np.array_equal(got[2], np.cumsum(start).astype(np.uint32))


def test_noalloc_crowded_bucket_stays_a_permutation():
    """A cell far larger than the spheres crowds 3,000 of them into one bucket, above
    GG_NOALLOC_MAX_OCCUPANCY: keys and bucket starts stay exact (the oracle's), and the
    crowded bucket's slots hold exactly its members, in an unspecified order."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_01369_gb300 import gg
    import oracle
    oracle.build()
    lib = gg.load()
    torch.cuda.set_device(0)
    pr = np.concatenate([S.random_cloud(3000, seed=12, box=0.05)[0],
                         S.random_cloud(2000, seed=14, box=0.5)[0] + np.array([2.0, 2.0, 2.0, 0.0], np.float32)])
    n_h = 4099
    for _ in range(2):
        keys, perm, start = _noalloc(torch, lib, np.ascontiguousarray(pr), 1.0, n_h)
        want = oracle.cell_keys(pr[:, :3].astype(np.float64), 1.0, n_h)
        assert np.array_equal(keys, want)
        cnt = np.zeros(n_h + 1, np.int64)
        np.add.at(cnt, want.astype(np.int64) + 1, 1)
        assert np.array_equal(start, np.cumsum(cnt).astype(np.uint32))
        assert (np.diff(start.astype(np.int64)) > 1024).any()
        assert np.array_equal(np.sort(perm), np.arange(pr.shape[0], dtype=np.uint32))
        ref = oracle.sort_perm(want)
        for b in range(n_h):
            seg = slice(int(start[b]), int(start[b + 1]))
            if start[b + 1] - start[b] <= 1024:
                assert np.array_equal(perm[seg], ref[seg])
            else:
                assert np.array_equal(np.sort(perm[seg]), np.sort(ref[seg]))


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_01369_gb300 import gg
    lib = gg.load()
    big = (1 << 20) + 1
    assert lib.gg_bin_sort_noalloc(None, big, 0.01, 16, None, None, None, None) == gg.ERR_INVALID_ARG
    assert lib.gg_bin_sort_noalloc(None, 0, 0.01, (1 << 21) + 1, None, None, None, None) == gg.ERR_INVALID_ARG
