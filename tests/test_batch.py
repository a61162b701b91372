"""Batches: every instance's records equal the oracle's, through one graph-launched batched run."""
import numpy as np
import pytest

import oracle
import paper_2012_03119_gb300 as gss
import synth
from gpu_util import check_records

pytestmark = pytest.mark.gpu


def small_batch(n=10, scale=0.01, seed=None):
    return [synth.batch_instance(s) for s in synth.batch_specs(n, seed=seed, scale=scale)]


def load_batch(b, insts, device_codes=False):
    import torch
    for I in insts:
        i = b.add_instance(I.n_vars, I.offsets, I.lits, max_assignments=max(I.n_assign, 32),
                           report_capacity=I.n_clauses * ((I.n_assign + 31) // 32) + 1024)
        b.set_assignments(i, torch.from_numpy(I.codes).cuda() if device_codes else I.codes)


def check_all(b, insts, mode=gss.GSS_MODE_ALLF):
    for i, I in enumerate(insts):
        rec = b.fetch_reports(i)
        check_records(rec, I.n_clauses, I.n_assign)
        assert np.array_equal(gss.expand_reports(rec), oracle.pairs(I.offsets, I.lits, I.codes, mode)), f"instance {i}"


@pytest.mark.parametrize("device_codes", [False, True])
def test_uneven_batch_matches_oracle(device_codes):
    insts = small_batch(12)
    with gss.Batch() as b:
        load_batch(b, insts, device_codes)
        b.test()
        check_all(b, insts)
        info = b.info()
        assert info["n_instances"] == 12 and info["n_groups"] == 1 and info["tiles_per_steal"][0] >= 1


def test_graph_replay_and_new_assignments():
    insts = small_batch(6, seed=77)
    with gss.Batch() as b:
        load_batch(b, insts)
        b.test()
        b.test()  # replay of the same graph
        check_all(b, insts)
        for I in insts:  # new contents, same sizes: the captured graph stays valid
            I.codes = synth.assign_trail(I.n_vars, I.n_assign, 0.3, 0.7, int(I.params["seed"]) + 1)
        for i, I in enumerate(insts):
            b.set_assignments(i, I.codes)
        b.test()
        check_all(b, insts)
        assert b.info()["runs"] == 3


def test_mixed_row_widths_and_trigger():
    insts = small_batch(4, seed=5)
    big = synth.single(scale=0.002, n_assign=2048)  # N > 1024: a second launch group
    insts.append(big)
    for mode in (gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER):
        with gss.Batch(mode=mode) as b:
            load_batch(b, insts)
            b.test()
            assert b.info()["n_groups"] == 2
            check_all(b, insts, mode)


def test_bad_instance_is_isolated():
    insts = small_batch(4, seed=9)
    with gss.Batch() as b:
        load_batch(b, insts)
        bad = insts[2].codes.copy()
        bad[0, 0] = 7
        b.set_assignments(2, bad)
        b.test()
        with pytest.raises(gss.GssError) as ei:
            b.fetch_reports(2)
        assert ei.value.code == gss.GSS_E_INVAL
        for i in (0, 1, 3):
            I = insts[i]
            assert np.array_equal(gss.expand_reports(b.fetch_reports(i)), oracle.allf_pairs(I.offsets, I.lits, I.codes))


def test_empty_instances_and_state_errors():
    insts = small_batch(3, seed=3)
    with gss.Batch() as b:
        with pytest.raises(gss.GssError) as ei:
            b.test()
        assert ei.value.code == gss.GSS_E_STATE
        load_batch(b, insts)
        i = b.add_instance(10, np.zeros(1, np.uint64), np.zeros(0, np.uint32))  # no clauses
        b.set_assignments(i, np.zeros((40, 10), np.uint8))
        j = b.add_instance(10, np.array([0, 1], np.uint64), np.array([0], np.uint32))
        with pytest.raises(gss.GssError) as ei:
            b.test()  # instance j has no assignment set
        assert ei.value.code == gss.GSS_E_STATE
        b.set_assignments(j, np.zeros((0, 10), np.uint8))  # an empty set
        b.test()
        check_all(b, insts)
        assert len(b.fetch_reports(i)) == 0 and len(b.fetch_reports(j)) == 0


def test_autotune_cache_file(tmp_path):
    """With GSS_AUTOTUNE_CACHE set, the first process tunes and writes its choices; the second
    takes them from the file (no timing) and gives the same records."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, oracle, synth
import paper_2012_03119_gb300 as gss
insts = [synth.batch_instance(s) for s in synth.batch_specs(5, scale=0.01, seed=77)]
with gss.Batch() as b:
    for I in insts:
        b.set_assignments(b.add_instance(I.n_vars, I.offsets, I.lits, max_assignments=I.n_assign,
                                         report_capacity=1 << 20), I.codes)
    b.test()
    same = all(np.array_equal(gss.expand_reports(b.fetch_reports(i)), oracle.allf_pairs(I.offsets, I.lits, I.codes))
               for i, I in enumerate(insts))
    info = b.info()
print(json.dumps({"same": same, "tuned_us": info["tuned_test_us"], "grab": info["tiles_per_steal"],
                  "cpw": info["clauses_per_tile"]}))
"""
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, GSS_AUTOTUNE_CACHE=str(cache))
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", script, root], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert runs[0]["same"] and runs[1]["same"]
    assert runs[0]["tuned_us"] > 0 and runs[1]["tuned_us"] == 0
    assert runs[1]["grab"] == runs[0]["grab"] and runs[1]["cpw"] == runs[0]["cpw"]
    assert len(cache.read_text().split("\n")) >= 2
    # the cache file also fixes the tile shape: both shapes give the oracle's records
    lines = [l.split() for l in cache.read_text().splitlines() if l.strip()]
    for cpw in (16, 32):
        cache.write_text("".join(f"{k} {g} {d} {cpw}\n" for k, g, d, _ in lines))
        r = subprocess.run([sys.executable, "-c", script, root], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        out = json.loads(r.stdout.strip().splitlines()[-1])
        assert out["same"] and out["tuned_us"] == 0 and set(out["cpw"]) == {cpw}
