"""Parity at the benchmark's full sizes, in the launch configuration bench.py times."""
import numpy as np
import pytest

import oracle
import paper_2012_03119_gb300 as gss
import synth
from gpu_util import check_records

pytestmark = pytest.mark.gpu


def test_single_instance_full_size():
    """1M vars, 4M clauses (L ~ 131M), 1024 trail assignments: the oracle runs in full."""
    inst = synth.single(scale=1.0)
    with gss.Context(inst.n_vars, report_capacity=1 << 25) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        rec = ctx.run(inst.codes)
    check_records(rec, inst.n_clauses, inst.n_assign)
    got = gss.expand_reports(rec)
    want = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes)
    assert got.shape == want.shape and np.array_equal(got, want)
    s = set(map(tuple, got.tolist()))
    assert all(tuple(p) in s for p in inst.planted.tolist())


def test_structured_full_size_sampled():
    """10M vars, 10M clauses (L ~ 660M), 1024 assignments: the oracle checks a 64-assignment
    sample in full, and every GPU pair of a further random sample one by one."""
    inst = synth.structured(scale=1.0)
    with gss.Context(inst.n_vars, report_capacity=1 << 26) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        rec = ctx.run(inst.codes)
    check_records(rec, inst.n_clauses, inst.n_assign)
    got = gss.expand_reports(rec)
    s = set(map(tuple, got.tolist()))
    assert all(tuple(p) in s for p in inst.planted.tolist())
    lo, hi = 480, 544  # two whole 32-assignment groups
    want = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, a_range=(lo, hi))
    sub = got[(got[:, 1] >= lo) & (got[:, 1] < hi)]
    assert np.array_equal(sub, want)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(got), size=min(2000, len(got)), replace=False):
        c, a = got[i]
        assert oracle.pair(inst.offsets, inst.lits, inst.codes[a], int(c))
