"""Parity at the benchmark's full sizes, in the launch configuration bench.py times."""
import numpy as np
import pytest

import oracle
import paper_2012_03119_gb300 as gss
import synth
from gpu_util import check_records, contains_all

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
    assert contains_all(got, inst.planted)


def test_structured_full_size():
    """10M vars in 1,000 communities, 10M clauses (L ~ 660M), 1024 assignments: the whole set
    against the oracle (10.2 G pair tests on the host cores)."""
    inst = synth.structured(scale=1.0)
    with gss.Context(inst.n_vars, report_capacity=1 << 26) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        rec = ctx.run(inst.codes)
    check_records(rec, inst.n_clauses, inst.n_assign)
    got = gss.expand_reports(rec)
    assert contains_all(got, inst.planted)
    want = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes)
    assert got.shape == want.shape and np.array_equal(got, want)


def test_batch_full_size():
    """The 64-instance batching workload at full size (18.6M clauses, 12.5 G pair tests) in one
    graph run: every instance equals the oracle in full."""
    insts = [synth.batch_instance(sp) for sp in synth.batch_specs(64)]
    with gss.Batch() as b:
        for I in insts:
            cap = I.n_clauses * ((I.n_assign + 31) // 32) // 4 + 65536
            i = b.add_instance(I.n_vars, I.offsets, I.lits, max_assignments=I.n_assign, report_capacity=cap)
            b.set_assignments(i, I.codes)
        b.test()
        got = [gss.expand_reports(b.fetch_reports(i)) for i in range(len(insts))]
    for I, g in zip(insts, got):
        assert contains_all(g, I.planted), I.name
        want = oracle.allf_pairs(I.offsets, I.lits, I.codes)
        assert g.shape == want.shape and np.array_equal(g, want), I.name


def test_serve_full_size():
    """The serving workload at full size: 1M vars, the database grows from 2M to 6M clauses in
    80 batches of 50k, with the bench's server shape.  Requests admitted along the way, and
    three at the final 6M-clause watermark, equal the oracle on the database prefix their
    watermark names."""
    w = synth.serve_workload(scale=1.0)
    snaps = synth.serve_snapshots(w.n_vars, 4, seed=synth.seed_for(4, 1))
    final = len(w.offsets) - 1
    with gss.Server(w.n_vars, max_clauses=final + 1, max_lits=int(w.offsets[-1]) + 1, slots=64, lanes=3,
                    lane_report_capacity=1 << 23) as srv:
        srv.add_clauses(*w.csr(0, w.n_initial))
        ids = [(srv.submit(snaps[0], wait_us=10_000_000), 0)]
        for b in range(w.n_batches):
            srv.add_clauses(*w.csr(*w.batch_range(b)))
            if b % 20 == 19:
                ids.append((srv.submit(snaps[(b + 1) % 4], wait_us=10_000_000), (b + 1) % 4))
        for k in range(3):  # at the final watermark
            ids.append((srv.submit(snaps[k + 1], wait_us=10_000_000), k + 1))
        results = [(srv.wait(rid), k) for rid, k in ids]
    seen = []
    for (rec, info), k in results:
        wm = info["watermark"]
        assert w.n_initial <= wm <= final
        off = w.offsets[: wm + 1]
        want = oracle.allf_pairs(off, w.lits[: int(off[-1])], snaps[k])
        assert np.array_equal(gss.expand_reports(rec), want)
        seen.append(wm)
    assert final == 6_000_000 and seen.count(final) >= 3
    assert len(set(seen)) >= 4  # requests saw different database sizes
