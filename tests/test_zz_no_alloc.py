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
    cases = [(S.column_collapse(n=60000, n_steps=1).pos_r, 0.0045, 120000),
             (S.random_cloud(9000, seed=5, box=0.12)[0], 0.0045, 7001)]
    for pos_r, cell, n_h in cases:
        got = _noalloc(torch, lib, np.ascontiguousarray(pos_r), cell, n_h)
        want = _regular_path(gg, np.ascontiguousarray(pos_r), cell, n_h)
        for g, w, name in zip(got, want, ("keys", "perm", "cell_start")):
            assert g.shape == w.shape, name
            assert np.array_equal(g, w), name


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_01369_gb300 import gg
    lib = gg.load()
    big = (1 << 20) + 1
    assert lib.gg_bin_sort_noalloc(None, big, 0.01, 16, None, None, None, None) == gg.ERR_INVALID_ARG
    assert lib.gg_bin_sort_noalloc(None, 0, 0.01, (1 << 21) + 1, None, None, None, None) == gg.ERR_INVALID_ARG
