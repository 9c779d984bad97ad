"""C ABI checks that need no GPU: the library builds, loads, and exports every
function include/gg.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2306_01369_gb300 import _build, gg
    _build.build()
    return gg.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "gg.h")).read()
    return sorted(set(re.findall(r"^GG_API[^;]*?\b(gg_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_api():
    names = _declared()
    for n in ("gg_create", "gg_create_batch", "gg_set_bodies", "gg_step", "gg_readback", "gg_destroy"):
        assert n in names
    assert len(names) >= 16


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2306_01369_gb300 import gg
    assert set(_declared()) == set(gg.SIGNATURES), "binding and header disagree"


def test_library_exports_nothing_else():
    from paper_2306_01369_gb300 import gg
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", gg.LIB_PATH], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert syms == set(_declared())


def test_host_only_calls(lib):
    assert lib.gg_abi_version() == 2
    assert lib.gg_status_string(0) == b"ok"
    assert lib.gg_status_string(4) == b"contact capacity overflow"
    assert lib.gg_tuning_count() >= 2
    assert lib.gg_tuning_flags(0) == 0 and lib.gg_tuning_flags(lib.gg_tuning_count() + 1) == 0
    assert lib.gg_last_error(None) == b"null simulation"
    lib.gg_destroy(None)   # no-op


def test_tuning_sets_cover_every_variant():
    """Each launch variant exists with both binnings, so the autotuner can pick any
    combination the binning restriction allows."""
    from paper_2306_01369_gb300 import gg
    sets = [gg.tuning_flags(k) for k in range(1, gg.load().gg_tuning_count() + 1)]
    assert {"lists"} in sets and set() in sets
    for v in ("lean", "half"):
        assert {v} in sets and {v, "lists"} in sets
    assert {"fused"} in sets
    assert {"detect"} in sets and {"detect", "lists"} in sets
    assert {"serp", "preload"} in sets and {"serp", "lists", "preload"} in sets
    assert {"serp", "lists", "half", "preload"} in sets and {"serp", "lists", "half", "lean"} in sets
    assert {"oneloop"} in sets and {"oneloop", "lists"} in sets


def test_struct_sizes_match_header():
    """The ctypes mirrors must have the C layout (4-byte fields and arrays)."""
    from paper_2306_01369_gb300 import gg
    assert ctypes.sizeof(gg.GGParams) == 4 * 26
    assert ctypes.sizeof(gg.GGBody) == 4 * (2 + 12 + 3 + 4 + 3 + 3 + 1 + 3)
    assert ctypes.sizeof(gg.GGStats) == 8 + 4 * 8   # 7 four-byte fields, padded to 8
    assert ctypes.sizeof(gg.GGCamera) == 4 * 20


def test_create_rejects_bad_params_before_touching_a_device(lib):
    """Invalid parameter structs are rejected by argument checks (no CUDA call needed)."""
    from paper_2306_01369_gb300 import gg
    p = gg.GGParams()
    p.struct_size = 3   # wrong version
    h = ctypes.c_void_p()
    assert lib.gg_create(ctypes.byref(p), 0, None, None, None, 0, ctypes.byref(h)) == gg.ERR_INVALID_ARG
    assert lib.gg_create(None, 0, None, None, None, 0, ctypes.byref(h)) == gg.ERR_INVALID_ARG


def test_checked_build_exports_the_same_symbols():
    """libgg_debug.so (-DGG_DEBUG, device-side index checks) builds without a GPU and
    exports exactly the release library's ABI."""
    import subprocess
    from paper_2306_01369_gb300 import _build

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
        return {l.split()[-1] for l in out.splitlines() if " T " in l}

    assert exported(_build.build(debug=True)) == exported(_build.build()) == set(_declared())


def test_no_device_fails_loudly(lib):
    """Without a CUDA device the library reports it (GG_ERR_NO_DEVICE) instead of
    computing anything on the host: creating a simulation raises, and the
    allocation-free binning call returns the status without touching its buffers."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import numpy as np
    from paper_2306_01369_gb300 import gg, scenes as S
    pr = np.array([[0.0, 0.0, 0.0, 0.01], [0.05, 0.0, 0.0, 0.01]], np.float32)
    with pytest.raises(gg.GGError) as e:
        gg.Sim(pr, None, None, S.Params())
    assert e.value.status == gg.ERR_NO_DEVICE
    keys = (ctypes.c_uint32 * 2)()
    assert lib.gg_bin_sort_noalloc(ctypes.c_void_p(pr.ctypes.data), 2, ctypes.c_float(0.02), 4, keys, keys, keys,
                                   None) == gg.ERR_NO_DEVICE
