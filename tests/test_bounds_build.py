"""The bounds-checked build (GSS_DEBUG_BOUNDS=1): the same results as the oracle on every path
(plain test in both modes and both tile shapes, wide sets in both modes, batch, serving with
and without a reduction, activity and deletion),
with no out-of-range gather counted.  Runs in a subprocess that builds and loads the checked
library, so the rest of the suite keeps the release build."""
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
from paper_2012_03119_gb300 import _build
assert _build.BOUNDS and _build.LIB.endswith("libgss_bounds.so")
_build.build()
gss.gss_debug_bounds(reset=True)
ok = {}
inst = synth.tiny()
for mode in (gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER):
    with gss.Context(inst.n_vars, mode=mode, report_capacity=1 << 20, max_assignments=64) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        got = gss.expand_reports(ctx.run(inst.codes))
    ok["plain%d" % mode] = bool(np.array_equal(got, oracle.pairs(inst.offsets, inst.lits, inst.codes, mode)))
insts = [synth.batch_instance(s) for s in synth.batch_specs(6, scale=0.005)]
with gss.Batch() as b:
    for I in insts:
        b.set_assignments(b.add_instance(I.n_vars, I.offsets, I.lits, max_assignments=I.n_assign,
                                         report_capacity=1 << 20), I.codes)
    b.test()
    ok["batch"] = all(np.array_equal(gss.expand_reports(b.fetch_reports(i)), oracle.allf_pairs(I.offsets, I.lits, I.codes))
                      for i, I in enumerate(insts))
w = synth.serve_workload(scale=0.005, n_batches=2)
snap = synth.serve_snapshots(w.n_vars, 1, seed=3)[0]
with gss.Server(w.n_vars, max_clauses=len(w.offsets), max_lits=int(w.offsets[-1]) + 1, slots=4, lanes=2) as srv:
    srv.add_clauses(*w.csr(0, w.n_initial))
    rec, info = srv.wait(srv.submit(snap, wait_us=10_000_000))
off = w.offsets[: info["watermark"] + 1]
ok["serve"] = bool(np.array_equal(gss.expand_reports(rec), oracle.allf_pairs(off, w.lits[: int(off[-1])], snap)))
with gss.Context(inst.n_vars, report_capacity=1 << 20, max_assignments=64) as ctx:
    ctx.set_activity(0.9)
    ctx.add_clauses(inst.offsets, inst.lits)
    ctx.run(inst.codes)
    ctx.reduce_db(0.5)
    ids = ctx.clause_ids()
    got = gss.expand_reports(ctx.run(inst.codes))
full = oracle.pairs(inst.offsets, inst.lits, inst.codes)
keep = np.isin(full[:, 0], ids)
ok["reduce"] = bool(np.array_equal(got, full[keep]))
wsizes = synth.clause_sizes(600, "geom", 1 / 7, 0, 30, 400, 5)
woff = synth.offsets_from_sizes(wsizes)
wlits = synth.clause_lits(woff, 400, 5)
wcodes = synth.assign_trail(400, 5000, 0.3, 0.7, 5, group=1024, flip_frac=0.1)
for mode in (gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER):  # more than 4096 assignments: the level-2 path
    with gss.Context(400, mode=mode, report_capacity=1 << 20, max_assignments=5000) as ctx:
        ctx.add_clauses(woff, wlits)
        got = gss.expand_reports(ctx.run(wcodes))
    ok["wide%d" % mode] = bool(np.array_equal(got, oracle.pairs(woff, wlits, wcodes, mode)))
# the 16-clause tile shape (two lanes per clause), long clauses with CSR tails
lsizes = synth.clause_sizes(900, "lognormal", 20.0, 1.0, 120, 500, 8)
loff = synth.offsets_from_sizes(lsizes)
llits = synth.clause_lits(loff, 500, 8)
lcodes = synth.assign_trail(500, 200, 0.3, 0.7, 8)
for mode in (gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER):
    with gss.Context(500, mode=mode, report_capacity=1 << 20, max_assignments=200, clauses_per_tile=16) as ctx:
        ctx.add_clauses(loff, llits)
        got = gss.expand_reports(ctx.run(lcodes))
    ok["cpw16_%d" % mode] = bool(np.array_equal(got, oracle.pairs(loff, llits, lcodes, mode)))
# serving with activity and a reduction, then a request on the compacted database
with gss.Server(w.n_vars, max_clauses=len(w.offsets), max_lits=int(w.offsets[-1]) + 1, slots=4, lanes=2) as srv:
    srv.set_activity(0.9)
    srv.add_clauses(*w.csr(0, w.n_initial))
    srv.wait(srv.submit(snap, wait_us=10_000_000))
    srv.reduce(0.5)
    kept = srv.clause_ids()
    rec, info = srv.wait(srv.submit(snap, wait_us=10_000_000))
off = w.offsets[: w.n_initial + 1]
sfull = oracle.allf_pairs(off, w.lits[: int(off[-1])], snap)
ok["serve_reduce"] = bool(np.array_equal(gss.expand_reports(rec), sfull[np.isin(sfull[:, 0], kept)]))
enabled, errors = gss.gss_debug_bounds()
print(json.dumps({"ok": ok, "enabled": enabled, "errors": errors}))
"""


@pytest.mark.gpu
def test_bounds_checked_build_runs_clean():
    env = dict(os.environ, GSS_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["enabled"] and out["errors"] == 0, out
    assert all(out["ok"].values()), out


def test_release_build_reports_no_bounds_checking():
    """Host-only: the release library says it is not the checked build (no device needed)."""
    import paper_2012_03119_gb300 as gss
    from paper_2012_03119_gb300 import _build
    if _build.BOUNDS:
        pytest.skip("running under the checked build")
    assert "gss_debug_bounds" in gss.SIGNATURES
