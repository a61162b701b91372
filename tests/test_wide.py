"""Sets of more than 4096 assignments: stage A on the level-2 aggregates (one bit per
1024-assignment super-group), then the 32-assignment groups of Section 4.2, then the exact
test -- the aggregate of aggregates that Section 7 proposes.  Records must equal the oracle
bit for bit, and each filter level must let through exactly the (clause, group) pairs whose
aggregate test (Section 4.2, with groups of 1024 and of 32) is positive."""
import numpy as np
import pytest

import oracle
import paper_2012_03119_gb300 as gss
import synth
from gpu_util import check_records
from oracle.activity import ActivityOracle

pytestmark = pytest.mark.gpu

ALLF, TRIG = gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER


def wide_instance(n_assign, n_vars=1500, n_clauses=1500, seed=23, units=40):
    """Geometric clause sizes (2 + Geom(1/7), at most 30), Zipf(1.1) variables; assignments as
    trail-prefix groups of 1024 (one simulated solver thread each), 30-70 % assigned with the
    last 10 % of each prefix re-decided; some unit clauses (which trigger wherever their
    variable is U) and planted all-F pairs."""
    sizes = synth.clause_sizes(n_clauses, "geom", 1 / 7, 0, 30, n_vars, seed)
    off = synth.offsets_from_sizes(sizes)
    lits = synth.clause_lits(off, n_vars, seed)
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2 * n_vars, size=units).astype(np.uint32)
    off = np.concatenate([off, off[-1] + np.arange(1, units + 1, dtype=np.uint64)])
    lits = np.concatenate([lits, u])
    codes = synth.assign_trail(n_vars, n_assign, 0.3, 0.7, seed, group=1024, flip_frac=0.1)
    pl = synth.plant(off, lits, codes, 60, seed)
    return synth.Instance(f"wide(N={n_assign})", n_vars, off, lits, codes, pl)


def run(inst, mode, cap=None):
    N = inst.codes.shape[0]
    cap = cap or inst.n_clauses * ((N + 31) // 32)
    with gss.Context(inst.n_vars, mode=mode, report_capacity=cap, max_assignments=N) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        rec = ctx.run(inst.codes)
        st = gss.gss_get_stats(ctx.ptr)
    check_records(rec, inst.n_clauses, N)
    return gss.expand_reports(rec), st


@pytest.mark.parametrize("N", [4097, 8192, 9000, 32768])
@pytest.mark.parametrize("mode", [ALLF, TRIG])
def test_wide_parity(N, mode):
    inst = wide_instance(N)
    got, st = run(inst, mode)
    want = oracle.pairs(inst.offsets, inst.lits, inst.codes, mode)
    assert got.shape == want.shape, f"{len(got)} GPU pairs vs {len(want)} oracle pairs"
    assert np.array_equal(got, want)
    assert len(want) >= len(inst.planted) > 0
    supers = -(-N // 1024)
    assert 0 < st["super_pairs"] < inst.n_clauses * supers, "the level-2 test filtered nothing or everything"


@pytest.mark.parametrize("N,mode", [(8192, ALLF), (8192, TRIG), (32768, ALLF)])
def test_wide_filter_levels_match_oracle(N, mode):
    """super_pairs = (clause, super-group) pairs with a positive aggregate test over 1024
    assignments; candidate_pairs = (clause, group) pairs with a positive test over 32, as on
    a narrow set: the level-2 filter only skips groups whose own test is negative."""
    inst = wide_instance(N, n_clauses=700, seed=31)
    got, st = run(inst, mode)
    want2 = oracle.aggregate_pairs(inst.offsets, inst.lits, inst.codes, group=1024, mode=mode)
    want1 = oracle.aggregate_pairs(inst.offsets, inst.lits, inst.codes, group=32, mode=mode)
    assert st["super_pairs"] == len(want2)
    assert st["candidate_pairs"] == len(want1)
    assert st["group_pairs"] == inst.n_clauses * ((N + 31) // 32)
    assert np.array_equal(got, oracle.pairs(inst.offsets, inst.lits, inst.codes, mode))


def test_wide_then_narrow_activity_and_ids():
    """One context with clause activity on takes wide and narrow sets in turn, and a reduction
    in between: records (with the surviving clauses' ids), activities and the level-2 counter
    as the oracle's float32 statement gives them, bit for bit."""
    inst = wide_instance(8192, n_clauses=900, seed=41)
    narrow = np.ascontiguousarray(inst.codes[:1000])
    ora = ActivityOracle(0.9)
    with gss.Context(inst.n_vars, report_capacity=1 << 22, max_assignments=8192) as ctx:
        ctx.set_activity(0.9)
        assert ctx.add_clauses(inst.offsets, inst.lits) == ora.add(inst.offsets, inst.lits) == 0
        for step, codes in enumerate((inst.codes, narrow, inst.codes, inst.codes, narrow)):
            got = gss.expand_reports(ctx.run(codes))
            want = ora.pairs(codes, ALLF)
            assert np.array_equal(got, want)
            ora.after_test(want[:, 0])
            st = gss.gss_get_stats(ctx.ptr)
            assert (st["super_pairs"] > 0) == (codes.shape[0] > gss.GSS_MAX_NARROW_ASSIGNMENTS)
            assert np.array_equal(ctx.clause_ids(), ora.ids)
            a = ctx.activity()
            assert np.array_equal(a.view(np.uint32), ora.act.view(np.uint32))
            if step == 2:
                assert ctx.reduce_db(0.5) == ora.reduce(0.5) > 0


def test_wide_limits():
    """N above GSS_MAX_ASSIGNMENTS is refused; batch instances keep the narrow limit."""
    with pytest.raises(gss.GssError):
        gss.Context(100, max_assignments=gss.GSS_MAX_ASSIGNMENTS + 1)
    with gss.Batch() as b:
        with pytest.raises(gss.GssError) as ei:
            b.add_instance(100, np.array([0, 1], np.uint64), np.array([0], np.uint32), max_assignments=4097)
        assert ei.value.code == gss.GSS_E_INVAL
