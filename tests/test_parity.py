"""CUDA path vs the oracle, bit-exact as sorted (clause, assignment) pair sets."""
import numpy as np
import pytest

import oracle
import paper_2012_03119_gb300 as gss
import synth
from gpu_util import check_records, gpu_pairs, gpu_records

pytestmark = pytest.mark.gpu

ALLF, TRIG = gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER


def small_instance(n_vars=500, n_clauses=3000, n_assign=64, seed=11, trail=True, law="geom", cap=30):
    if law == "geom":
        sizes = synth.clause_sizes(n_clauses, "geom", 1 / 7, 0, cap, n_vars, seed)
    else:
        sizes = synth.clause_sizes(n_clauses, "lognormal", 20.0, 1.0, cap, n_vars, seed)
    off = synth.offsets_from_sizes(sizes)
    lits = synth.clause_lits(off, n_vars, seed)
    codes = (synth.assign_trail(n_vars, n_assign, 0.3, 0.7, seed) if trail
             else synth.assign_indep(n_vars, n_assign, 0.5, seed))
    pl = synth.plant(off, lits, codes, min(50, n_clauses), seed) if n_assign else np.zeros((0, 2), np.uint32)
    return synth.Instance("small", n_vars, off, lits, codes, pl)


def assert_parity(inst, mode=ALLF, **kw):
    got = gpu_pairs(inst, mode=mode, **kw)
    codes = kw.get("codes", inst.codes)
    want = oracle.pairs(inst.offsets, inst.lits, codes, mode)
    assert got.shape == want.shape, f"{len(got)} GPU pairs vs {len(want)} oracle pairs"
    assert np.array_equal(got, want)
    return got


@pytest.mark.parametrize("mode", [ALLF, TRIG])
def test_tiny(tiny_instance, mode):
    got = assert_parity(tiny_instance, mode)
    if mode == ALLF:
        s = set(map(tuple, got.tolist()))
        assert all(tuple(p) in s for p in tiny_instance.planted.tolist())


@pytest.mark.parametrize("mode", [ALLF, TRIG])
def test_single_scaled(mode):
    assert_parity(synth.single(scale=0.02), mode)  # 20k vars, 80k clauses, N = 1024


def test_structured_scaled():
    assert_parity(synth.structured(scale=0.003))  # 3 communities, 30k clauses, sizes up to 1000


@pytest.mark.parametrize("n_assign", [1, 31, 32, 33, 100, 128, 129, 513, 1000, 1025, 2049, 4096])
def test_ragged_assignment_counts(n_assign):
    inst = small_instance(n_assign=n_assign, seed=100 + n_assign)
    assert_parity(inst, ALLF, max_assignments=max(n_assign, 1024))


@pytest.mark.parametrize("n_assign", [33, 1000, 2049])
def test_ragged_trigger(n_assign):
    inst = small_instance(n_assign=n_assign, seed=200 + n_assign)
    assert_parity(inst, TRIG, max_assignments=max(n_assign, 1024))


def test_independent_assignments_many_hits():
    inst = small_instance(n_vars=60, n_clauses=5000, n_assign=256, trail=False, seed=5)
    assert len(assert_parity(inst)) > 10000


@pytest.mark.parametrize("cpw", [16, 32])
@pytest.mark.parametrize("mode", [ALLF, TRIG])
@pytest.mark.parametrize("law", ["geom", "lognormal"])
def test_tile_shapes(cpw, mode, law):
    """Both test tile shapes (a lane per clause; two lanes per clause, whose segment results
    compose) give the oracle's pairs and the oracle's aggregate-test count: short and long
    clauses (CSR tails of several 16-literal rounds), a ragged last tile (3001 clauses), a
    ragged last group (200 assignments)."""
    inst = small_instance(n_vars=700, n_clauses=3001, n_assign=200, seed=21, law=law, cap=200)
    assert_parity(inst, mode, clauses_per_tile=cpw)
    with gss.Context(inst.n_vars, mode=mode, report_capacity=1 << 20, max_assignments=200,
                     clauses_per_tile=cpw) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.run(inst.codes)
        st = gss.gss_get_stats(ctx.ptr)
    assert st["candidate_pairs"] == len(oracle.aggregate_pairs(inst.offsets, inst.lits, inst.codes, mode=mode))


@pytest.mark.parametrize("cpw", [16, 32])
def test_tile_shapes_around_head_width(cpw):
    test_sizes_around_head_width_and_tautologies(cpw)


def test_sizes_around_head_width_and_tautologies(cpw=0):
    V, rng = 40, np.random.default_rng(1)
    clauses = []
    for s in list(range(1, 21)) * 30:
        vs = rng.choice(V, size=s, replace=False)
        clauses.append(list(2 * vs + rng.integers(0, 2, s)))
    for s in (2, 7, 8, 9, 16):  # tautologies at every head boundary
        for _ in range(20):
            vs = rng.choice(V, size=s - 1, replace=False)
            c = list(2 * vs + rng.integers(0, 2, s - 1))
            clauses.append(c + [c[0] ^ 1])
    off = np.zeros(len(clauses) + 1, np.uint64)
    off[1:] = np.cumsum([len(c) for c in clauses])
    lits = np.array([l for c in clauses for l in c], np.uint32)
    codes = synth.assign_trail(V, 512, 0.5, 1.0, 9)
    inst = synth.Instance("heads", V, off, lits, codes, np.zeros((0, 2), np.uint32))
    assert_parity(inst, ALLF, clauses_per_tile=cpw)
    assert_parity(inst, TRIG, clauses_per_tile=cpw)


def test_all_u_assignments():
    inst = small_instance(n_assign=0)
    codes = np.zeros((96, inst.n_vars), np.uint8)
    assert len(gpu_pairs(inst, codes=codes)) == 0
    # Definition "triggers": a unit clause triggers when its literal is U; longer clauses never do
    units = synth.Instance("units", 10, np.arange(0, 11, dtype=np.uint64), np.arange(0, 20, 2, dtype=np.uint32),
                           np.zeros((96, 10), np.uint8), np.zeros((0, 2), np.uint32))
    got = gpu_pairs(units, mode=TRIG)
    assert len(got) == 10 * 96
    assert_parity(inst, TRIG, codes=codes)


def test_empty_database_and_empty_set():
    inst = small_instance()
    with gss.Context(inst.n_vars) as ctx:
        ctx.set_assignments(inst.codes)
        ctx.test()
        assert len(ctx.fetch_reports()) == 0
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.set_assignments(np.zeros((0, inst.n_vars), np.uint8))
        ctx.test()
        assert len(ctx.fetch_reports()) == 0


def test_single_variable():
    off = np.array([0, 1, 2, 4], np.uint64)
    lits = np.array([0, 1, 0, 1], np.uint32)  # v, not v, (v or not v)
    codes = np.array([[0], [1], [2]] * 20, np.uint8)
    inst = synth.Instance("v1", 1, off, lits, codes, np.zeros((0, 2), np.uint32))
    got = assert_parity(inst)
    assert len(got) == 40  # clause 0 on every F, clause 1 on every T, the tautology never
    assert_parity(inst, TRIG)


def test_report_overflow_then_rerun():
    inst = small_instance(n_vars=60, n_clauses=5000, n_assign=256, trail=False, seed=5)
    want = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes)
    with gss.Context(inst.n_vars, report_capacity=100, max_assignments=256) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.set_assignments(inst.codes)
        ctx.test()
        with pytest.raises(gss.GssError) as ei:
            ctx.fetch_reports()
        assert ei.value.code == gss.GSS_E_OVERFLOW
        with pytest.raises(gss.GssError):
            ctx.report_count()
        ctx.set_report_capacity(1 << 20)
        ctx.test()
        rec = ctx.fetch_reports()
        check_records(rec, inst.n_clauses, 256)
        assert np.array_equal(gss.expand_reports(rec), want)
        # a caller buffer smaller than the record count
        small = np.empty(10, gss.REPORT_DTYPE)
        with pytest.raises(gss.GssError) as ei:
            ctx.fetch_reports(small)
        assert ei.value.code == gss.GSS_E_OVERFLOW


def test_invalid_inputs_leave_state_unchanged():
    inst = small_instance()
    with gss.Context(inst.n_vars, max_assignments=64) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        before = ctx.run(inst.codes)
        bad = inst.lits.copy()
        bad[5] = 2 * inst.n_vars  # literal out of range
        with pytest.raises(gss.GssError) as ei:
            ctx.add_clauses(inst.offsets, bad)
        assert ei.value.code == gss.GSS_E_INVAL
        with pytest.raises(gss.GssError) as ei:  # empty clause
            ctx.add_clauses(np.array([0, 2, 2, 3], np.uint64), np.array([0, 2, 4], np.uint32))
        assert ei.value.code == gss.GSS_E_INVAL
        with pytest.raises(gss.GssError) as ei:  # offsets[0] != 0
            ctx.add_clauses(np.array([1, 2], np.uint64), np.array([0, 2], np.uint32))
        assert ei.value.code == gss.GSS_E_INVAL
        assert ctx.stats()["n_clauses"] == inst.n_clauses
        with pytest.raises(gss.GssError) as ei:  # too many assignments
            ctx.set_assignments(np.zeros((65, inst.n_vars), np.uint8))
        assert ei.value.code == gss.GSS_E_INVAL
        codes = inst.codes.copy()
        codes[3, 7] = 3  # value code outside {0, 1, 2}
        ctx.set_assignments(codes)
        ctx.test()
        with pytest.raises(gss.GssError) as ei:
            ctx.fetch_reports()
        assert ei.value.code == gss.GSS_E_INVAL
        after = ctx.run(inst.codes)
        assert np.array_equal(gss.expand_reports(before), gss.expand_reports(after))


@pytest.mark.parametrize("layout", [gss.GSS_LAYOUT_FREQUENCY, gss.GSS_LAYOUT_IDENTITY])
def test_assignments_before_the_first_clauses(layout):
    """An assignment set given before any clause: the frequency layout's numbering, fixed by
    the first clause batch, applies to it as well."""
    inst = small_instance()
    with gss.Context(inst.n_vars, max_assignments=inst.n_assign, layout=layout) as ctx:
        ctx.set_assignments(inst.codes)
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.test()
        got = gss.expand_reports(ctx.fetch_reports())
    assert np.array_equal(got, oracle.allf_pairs(inst.offsets, inst.lits, inst.codes))


def test_test_before_assignments():
    with gss.Context(10) as ctx:
        with pytest.raises(gss.GssError) as ei:
            ctx.test()
        assert ei.value.code == gss.GSS_E_STATE
        with pytest.raises(gss.GssError) as ei:
            ctx.fetch_reports()
        assert ei.value.code == gss.GSS_E_STATE


def test_incremental_database_growth():
    inst = synth.single(scale=0.005)  # 20k clauses in uneven batches, forcing several reallocations
    want = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes)
    with gss.Context(inst.n_vars) as ctx:
        cuts = [0, 1, 700, 701, 5000, 12000, inst.n_clauses]
        for a, b in zip(cuts[:-1], cuts[1:]):
            off = inst.offsets[a:b + 1] - inst.offsets[a]
            first = ctx.add_clauses(off, inst.lits[int(inst.offsets[a]):int(inst.offsets[b])])
            assert first == a
        got = gss.expand_reports(ctx.run(inst.codes))
    assert np.array_equal(got, want)


def test_device_codes_and_torch_stream():
    import torch
    inst = small_instance(n_vars=501, n_assign=100)  # odd V: unaligned rows take the copy path
    want = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes)
    s = torch.cuda.Stream()
    with gss.Context(inst.n_vars, stream=s, max_assignments=100) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        d = torch.from_numpy(inst.codes).cuda()
        torch.cuda.synchronize()
        ctx.set_assignments(d)
        ctx.test()
        assert np.array_equal(gss.expand_reports(ctx.fetch_reports()), want)
        wide = torch.zeros((100, 512), dtype=torch.uint8, device="cuda")  # pitch 512 > V, aligned
        wide[:, :501] = d
        wide[:, 501:] = 2  # bytes past V must be ignored
        torch.cuda.synchronize()
        gss.gss_set_assignments_device(ctx.ptr, wide.data_ptr(), 512, 100)
        ctx.test()
        assert np.array_equal(gss.expand_reports(ctx.fetch_reports()), want)


def test_repeatable():
    inst = synth.single(scale=0.01)
    with gss.Context(inst.n_vars) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.set_assignments(inst.codes)
        a = gss.expand_reports(ctx.run(inst.codes))
        ctx.test()
        b = gss.expand_reports(ctx.fetch_reports())
    assert np.array_equal(a, b)


def test_long_planted_clause():
    V = 3000
    rng = np.random.default_rng(4)
    lits = (2 * rng.choice(V, size=1000, replace=False) + rng.integers(0, 2, 1000)).astype(np.uint32)
    off = np.array([0, 1000], np.uint64)
    codes = synth.assign_trail(V, 1024, 0.3, 0.7, 4)
    for a in (0, 517, 1023):
        codes[a, lits >> 1] = np.where(lits & 1, 1, 2)
    inst = synth.Instance("long", V, off, lits, codes, np.zeros((0, 2), np.uint32))
    got = assert_parity(inst)
    assert {0, 517, 1023} <= set(got[:, 1].tolist())


@pytest.mark.parametrize("mode", [ALLF, TRIG])
def test_layouts_agree(mode):
    """The internal variable numbering changes memory layout only, never results."""
    inst = synth.single(scale=0.01)
    out = []
    for layout in (gss.GSS_LAYOUT_IDENTITY, gss.GSS_LAYOUT_FREQUENCY):
        with gss.Context(inst.n_vars, mode=mode, layout=layout, report_capacity=1 << 22) as ctx:
            ctx.add_clauses(inst.offsets, inst.lits)
            out.append(gss.expand_reports(ctx.run(inst.codes)))
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(out[0], oracle.pairs(inst.offsets, inst.lits, inst.codes, mode))


@pytest.mark.parametrize("mode", [ALLF, TRIG])
@pytest.mark.parametrize("layout", [gss.GSS_LAYOUT_IDENTITY, gss.GSS_LAYOUT_FREQUENCY])
def test_aggregate_candidates_match_oracle(mode, layout):
    """Stage A is the aggregate test of Section 4.2 (Listing aggregateTrigger, all-F or
    trigger): the number of (clause, group) pairs it lets through equals the oracle's count of
    pairs whose aggregate test is positive, including a ragged last group."""
    inst = small_instance(n_vars=400, n_clauses=2500, n_assign=80, seed=5)
    with gss.Context(inst.n_vars, mode=mode, layout=layout, report_capacity=1 << 20, max_assignments=80) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.run(inst.codes)
        st = gss.gss_get_stats(ctx.ptr)
    want = oracle.aggregate_pairs(inst.offsets, inst.lits, inst.codes, mode=mode)
    assert st["group_pairs"] == inst.n_clauses * 3
    assert st["candidate_pairs"] == len(want)
    assert 0 < len(want) < st["group_pairs"]
