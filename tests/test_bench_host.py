"""Host logic of bench.py that needs no GPU: the kernels a launch-shape set runs, the
profile lookup (digest match), the algorithmic byte counts, the hash-table option."""
import argparse

import bench


def test_stage_kernels_follow_the_tuning_flags():
    assert bench.stage_kernels(set()) == ("k_pja", "k_contacts")
    assert bench.stage_kernels({"lists", "half"}) == ("k_pja", "k_pairs_half+k_pairs_finish")
    assert bench.stage_kernels({"lean"})[0] == "k_pja_lean"
    assert bench.stage_kernels({"fused"})[0] == "k_pja_fused"
    assert bench.stage_kernels({"detect", "lists"}) == ("k_detect_sweeps", "k_detect_sweeps")
    assert bench.stage_kernels({"oneloop", "lists"}) == ("k_oneloop", "k_contacts")
    assert bench.stage_kernels({"lists", "lean", "half", "serp"}) == ("k_pja_lean", "k_pairs_half+k_pairs_finish")
    assert bench.profile_traffic("k_pja", "column_pile", "x") is None     # no profile kept for it


def test_profile_traffic_needs_the_current_digest(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_pja_column_collapse.txt").write_text("# c\nkernel_digest: abc\ndram_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("k_pja", "column", "abc") == 1234.0
    assert bench.profile_traffic("k_pja", "column", "other") is None
    assert bench.profile_traffic("k_pja", "excavation", "abc") is None   # no such file


def test_algorithmic_bytes():
    assert bench.pja_bytes(10, 0, 0) == 520
    assert bench.pja_bytes(0, 1, 1) == 44 + 60
    assert bench.contacts_bytes(10, 2, 1, 20) == 600 + 80 + 64 + 48


def test_hash_option():
    assert bench.hash_kw(argparse.Namespace(hash_factor=0)) == {"hash_tune": 1}
    assert bench.hash_kw(argparse.Namespace(hash_factor=2)) == {"hash_factor": 2}


def test_committed_profiles_are_readable_and_name_their_command():
    """Every kernel summary under profiles/ gives the command that made it (with the
    clocks left alone) and, where it carries DRAM traffic, the kernel digest it was
    taken on; bench.py reads the traffic back for its own kernel and workload names."""
    import glob
    import os
    files = sorted(glob.glob(os.path.join(bench.ROOT, "profiles", "*.txt")))
    assert files
    for path in files:
        text = open(path).read()
        assert ("command" in text and "--clock-control none" in text) or "same report" in text, path
        kv = dict(line.split(":", 1) for line in text.splitlines() if ":" in line and not line.startswith("#"))
        if "dram_bytes_per_launch" in kv:
            assert float(kv["dram_bytes_per_launch"]) > 0 and len(kv["kernel_digest"].strip()) == 16, path
            stem, workload = os.path.basename(path)[:-4], None
            for w, name in bench.PROFILE_WORKLOAD.items():
                if stem.endswith("_" + name):
                    workload, kernel = w, stem[: -len(name) - 1]
            assert workload is not None, path
            assert bench.profile_traffic(kernel, workload, kv["kernel_digest"].strip()) == \
                float(kv["dram_bytes_per_launch"])
