"""Failure handling without a GPU fault: the n-th device allocation of a process is made to
fail on the host (GSS_FAULT_ALLOC_AT=n).  The call that hit it returns GSS_E_NOMEM, the
context stays usable, and repeating the call gives the oracle's records."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle, synth
import paper_2012_03119_gb300 as gss

inst = synth.tiny()
failed = []

def attempt(name, fn):
    try:
        return fn()
    except gss.GssError as e:  # the injected failure: record it, then the same call again
        failed.append([name, e.code])
        return fn()

ctx = attempt("create", lambda: gss.Context(inst.n_vars, report_capacity=1 << 20, max_assignments=64))
attempt("add_clauses", lambda: ctx.add_clauses(inst.offsets, inst.lits))
attempt("set_assignments", lambda: ctx.set_assignments(inst.codes))
ctx.test()
rec = ctx.fetch_reports()
same = bool(np.array_equal(gss.expand_reports(rec), oracle.allf_pairs(inst.offsets, inst.lits, inst.codes)))
ctx.close()
print(json.dumps({"failed": failed, "same": same}))
"""


@pytest.mark.gpu
@pytest.mark.parametrize("n", list(range(1, 16)))
def test_injected_allocation_failure(n):
    env = dict(os.environ, GSS_FAULT_ALLOC_AT=str(n))
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["same"], out
    assert len(out["failed"]) <= 1
    for name, code in out["failed"]:
        assert code == -2, (name, code)  # GSS_E_NOMEM


@pytest.mark.gpu
def test_injection_reaches_every_stage():
    """Some n lands in each of creation, ingest and staging (the loop above is not vacuous)."""
    seen = set()
    for n in range(1, 16):
        env = dict(os.environ, GSS_FAULT_ALLOC_AT=str(n))
        r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        seen |= {name for name, _ in json.loads(r.stdout.strip().splitlines()[-1])["failed"]}
    assert {"create", "add_clauses", "set_assignments"} <= seen, seen
