"""bench.py's host-side arithmetic (no device): the traffic figure is taken from an ncu summary
only while the kernel source still has the hash the counters were taken on, the whole-job
rate, and the algorithmic bytes of the roofline."""
import os
import re

import numpy as np

import bench
import synth


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2012_03119_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_x.cu").write_text("// kernel source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_sha("k_x.cu")
    summary = tmp_path / "profiles" / "k_x__w.md"
    summary.write_text(f"dram_bytes_per_launch_full: 1.25e+09\nsource_sha256_16: {sha}\n")
    assert bench.profiled_traffic("k_x.cu", "k_x__w.md") == 1.25e9
    (csrc / "k_x.cu").write_text("// kernel source, changed\n")  # counters no longer describe it
    assert bench.profiled_traffic("k_x.cu", "k_x__w.md") is None
    summary.write_text(f"dram_bytes_per_launch_full: null\nsource_sha256_16: {bench.kernel_source_sha('k_x.cu')}\n")
    assert bench.profiled_traffic("k_x.cu", "k_x__w.md") is None
    assert bench.profiled_traffic("k_x.cu", "missing.md") is None


def test_committed_summaries_are_well_formed():
    """Each committed summary that gives a traffic line also names the source hash and gives
    the command it came from."""
    d = os.path.join(bench.ROOT, "profiles")
    seen = 0
    for name in sorted(os.listdir(d)):
        text = open(os.path.join(d, name)).read()
        m = re.search(r"dram_bytes_per_launch_full:\s*(\S+)", text)
        if not m:
            continue
        seen += 1
        assert m.group(1) == "null" or float(m.group(1)) > 0, name
        assert re.search(r"source_sha256_16:\s*[0-9a-f]{16}\b", text), name
        assert "ncu " in text or "k_pack__" in text, name  # the command, or a pointer to it
    assert seen >= 4


def test_whole_job_rate_and_algorithmic_bytes():
    # 4 ranks x 1e9 units per step x 10 steps in 2 s = 20 G units/s
    assert abs(bench.whole_job_rate(10 ** 9, 4, 10, 2.0) - 20.0) < 1e-12
    inst = synth.tiny()
    m, L, V, N = inst.n_clauses, inst.n_lits, inst.n_vars, inst.n_assign
    W = (N + 31) // 32
    R = 1234
    b = bench.algorithmic_bytes(inst, R)
    assert b["test"] == 4 * (m + 1) + 4 * L + 8 * V * W + 12 * R
    assert b["pack"] == N * V + 8 * V * W
    assert np.isclose(bench.max_over_ranks(3.5), 3.5)
