"""Clause activity and activity-based deletion on the GPU (Section 3.6) against the oracle's
float32 statement: activities bit-exact after every test, the same clauses removed, and the
records of later tests carrying the surviving clauses' ids."""
import numpy as np
import pytest

import oracle
import synth
from oracle.activity import ActivityOracle
import paper_2012_03119_gb300 as gss

pytestmark = pytest.mark.gpu


def _db(n_vars, m, seed):
    sizes = synth.clause_sizes(m, "geom", 1 / 7, 0, 30, n_vars, seed)
    sizes[:: 7] = np.minimum(sizes[:: 7], 2)  # plenty of binary clauses, which are always kept
    off = synth.offsets_from_sizes(sizes)
    return off, synth.clause_lits(off, n_vars, seed)


def _codes(n_vars, n, seed):
    return synth.assign_trail(n_vars, n, 0.3, 0.7, seed)


def _check(ctx, ora):
    assert np.array_equal(ctx.clause_ids(), ora.ids)
    got = ctx.activity()
    assert got.dtype == np.float32 and np.array_equal(got.view(np.uint32), ora.act.view(np.uint32))


@pytest.mark.parametrize("mode", [gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER])
def test_activity_bumps_decay_reduce_and_ids(mode):
    n_vars = 300
    ora = ActivityOracle(0.8)
    with gss.Context(n_vars, mode=mode, report_capacity=1 << 20, max_assignments=96) as ctx:
        ctx.set_activity(0.8)
        off, lits = _db(n_vars, 4000, 21)
        assert ctx.add_clauses(off, lits) == ora.add(off, lits) == 0
        _check(ctx, ora)
        for step in range(9):
            codes = _codes(n_vars, 32 + 8 * step, 100 + step)
            pairs = gss.expand_reports(ctx.run(codes))
            want = ora.pairs(codes, mode)
            assert np.array_equal(pairs, want)
            ora.after_test(want[:, 0])
            _check(ctx, ora)
            if step == 3:
                off2, lits2 = _db(n_vars, 500, 31)
                assert ctx.add_clauses(off2, lits2) == ora.add(off2, lits2)
                _check(ctx, ora)
            if step in (4, 7):
                assert ctx.reduce_db(0.5) == ora.reduce(0.5) > 0
                _check(ctx, ora)
        st = ctx.stats()
        assert st["clauses_removed"] == ora.next_id - ora.n_clauses
        assert st["next_clause_id"] == ora.next_id


def test_rescale_matches_oracle():
    """decay 0.25 multiplies inc by 4 per test: past 1e20 after 34 tests, then every activity is
    scaled by 1e-20 on both sides, bit for bit."""
    n_vars = 200
    ora = ActivityOracle(0.25)
    with gss.Context(n_vars, report_capacity=1 << 20, max_assignments=64) as ctx:
        ctx.set_activity(0.25)
        off, lits = _db(n_vars, 1500, 41)
        ctx.add_clauses(off, lits)
        ora.add(off, lits)
        for step in range(40):
            codes = _codes(n_vars, 64, 200 + step)
            rec = ctx.run(codes)
            ora.after_test(gss.expand_reports(rec)[:, 0])
        assert ora.inc < np.float32(1e20)
        _check(ctx, ora)
        assert ctx.reduce_db(0.3) == ora.reduce(0.3)
        _check(ctx, ora)
        codes = _codes(n_vars, 64, 999)
        assert np.array_equal(gss.expand_reports(ctx.run(codes)), ora.pairs(codes))


def test_reduce_edge_cases():
    n_vars = 100
    with gss.Context(n_vars, report_capacity=1 << 16, max_assignments=32) as ctx:
        with pytest.raises(gss.GssError) as ei:  # activity off
            ctx.reduce_db(0.5)
        assert ei.value.code == gss.GSS_E_STATE
        with pytest.raises(gss.GssError):
            ctx.set_activity(0.0)
        ctx.set_activity(1.0)
        assert ctx.reduce_db(0.5) == 0  # empty database
        off, lits = _db(n_vars, 300, 51)
        ctx.add_clauses(off, lits)
        assert ctx.reduce_db(0.0) == 0
        with pytest.raises(gss.GssError):
            ctx.reduce_db(1.5)
        n_long = int((np.diff(off) > 2).sum())
        # all activities equal: ties go to the smaller id, so the oldest long clauses leave first
        assert ctx.reduce_db(1.0) == n_long
        ids = ctx.clause_ids()
        assert np.array_equal(ids, np.nonzero(np.diff(off) <= 2)[0].astype(np.uint32))
        codes = _codes(n_vars, 32, 7)
        ora = ActivityOracle(1.0)
        ora.add(off, lits)
        ora.reduce(1.0)
        assert np.array_equal(gss.expand_reports(ctx.run(codes)), ora.pairs(codes))


def test_larger_database_reduce_is_exact():
    """A 200k-clause database with activities spread over many values: the GPU's radix select
    removes exactly the oracle's clauses."""
    inst = synth.single(scale=0.05, n_assign=256)
    ora = ActivityOracle(0.95)
    with gss.Context(inst.n_vars, report_capacity=1 << 22, max_assignments=256) as ctx:
        ctx.set_activity(0.95)
        ctx.add_clauses(inst.offsets, inst.lits)
        ora.add(inst.offsets, inst.lits)
        for step in range(6):
            codes = synth.assign_trail(inst.n_vars, 256, 0.3, 0.7, 300 + step)
            rec = ctx.run(codes)
            ora.after_test(gss.expand_reports(rec)[:, 0])
        _check(ctx, ora)
        assert ctx.reduce_db(0.5) == ora.reduce(0.5)
        _check(ctx, ora)
        codes = inst.codes[:256]
        assert np.array_equal(gss.expand_reports(ctx.run(codes)), ora.pairs(codes))


@pytest.mark.parametrize("layout", [gss.GSS_LAYOUT_IDENTITY, gss.GSS_LAYOUT_FREQUENCY])
def test_export_rebuilds_the_database(layout):
    """The export gives the resident clauses in the caller's numbering (the frequency layout's
    renaming undone) with their ids; a context built from it reports the same pairs."""
    n_vars = 400
    ora = ActivityOracle(0.9)
    off, lits = _db(n_vars, 3000, 61)
    with gss.Context(n_vars, layout=layout, report_capacity=1 << 20, max_assignments=64) as ctx:
        ctx.set_activity(0.9)
        ctx.add_clauses(off, lits)
        ora.add(off, lits)
        e_off, e_lits, e_ids = ctx.export_clauses()
        assert np.array_equal(e_off, off) and np.array_equal(e_lits, lits)
        assert np.array_equal(e_ids, np.arange(len(off) - 1, dtype=np.uint32))
        for step in range(3):
            codes = _codes(n_vars, 64, 500 + step)
            ora.after_test(gss.expand_reports(ctx.run(codes))[:, 0])
        ctx.reduce_db(0.5)
        ora.reduce(0.5)
        e_off, e_lits, e_ids = ctx.export_clauses()
        assert np.array_equal(e_off, ora.offsets) and np.array_equal(e_lits, ora.lits)
        assert np.array_equal(e_ids, ora.ids)
        codes = _codes(n_vars, 64, 600)
        want = gss.expand_reports(ctx.run(codes))
    with gss.Context(n_vars, layout=layout, report_capacity=1 << 20, max_assignments=64) as ctx2:
        ctx2.add_clauses(e_off, e_lits)
        got = gss.expand_reports(ctx2.run(codes))
    got[:, 0] = e_ids[got[:, 0]]  # the rebuilt context numbers clauses from 0
    order = np.lexsort((got[:, 1], got[:, 0]))
    assert np.array_equal(got[order], want)


def test_record_and_overflow_counters():
    import ctypes
    inst = synth.tiny()
    with gss.Context(inst.n_vars, report_capacity=100, max_assignments=64) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.set_assignments(inst.codes)
        ctx.test()
        cnt = ctypes.c_uint64()
        for _ in range(2):  # reading twice counts once
            assert gss.load().gss_report_count(ctx.ptr, ctypes.byref(cnt)) == gss.GSS_E_OVERFLOW
        n = cnt.value
        st = ctx.stats()
        assert n > 100 and st["records"] == n and st["overflows"] == 1
        ctx.set_report_capacity(n)
        ctx.test()
        assert ctx.report_count() == n
        st = ctx.stats()
        assert st["records"] == 2 * n and st["overflows"] == 1
