"""The oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle
import synth
from pins import (pin_aggregate_brute_force, pin_aggregate_theorem, pin_brute_force, pin_golden, pin_invariants,
                  pin_monotone)

GOLDEN = ["sec33_trigger_example.txt", "sec36_two_thread_example.txt", "sec42_aggregate_examples.txt"]


@pytest.mark.parametrize("name", GOLDEN)
def test_golden_examples(name):
    assert pin_golden(name) == []


@pytest.mark.parametrize("n_vars", [1, 2, 3, 4])
def test_brute_force_closed_forms(n_vars):
    assert pin_brute_force(n_vars) == []


def test_invariants_tiny(tiny_instance):
    assert pin_invariants(tiny_instance) == []


def test_invariants_trail_assignments():
    inst = synth.single(scale=0.002)  # 2,000 vars, 8,000 clauses, 1024 trail assignments
    assert pin_invariants(inst) == []


def test_monotone(tiny_instance):
    assert pin_monotone(tiny_instance) == []


@pytest.mark.parametrize("mode", [oracle.MODE_ALLF, oracle.MODE_TRIGGER])
def test_aggregate_theorem(tiny_instance, mode):
    assert pin_aggregate_theorem(tiny_instance, mode, group=8) == []


@pytest.mark.parametrize("mode", [oracle.MODE_ALLF, oracle.MODE_TRIGGER])
def test_aggregate_of_aggregates(mode):
    """Section 7's aggregate of aggregates, which the test of sets above 4096 assignments
    filters with: the aggregate of a 1024-assignment super-group is the union of its 32
    groups' aggregates (value sets), and by the Theorem of Section 4.2 applied to it, every
    (clause, group) pair whose aggregate test passes lies in a super-group whose test passes.
    Ragged last group and super-group included."""
    V, N, m = 150, 2 * 1024 + 100, 300
    sizes = synth.clause_sizes(m, "geom", 1 / 7, 0, 30, V, 9)
    off = synth.offsets_from_sizes(sizes)
    lits = synth.clause_lits(off, V, 9)
    codes = synth.assign_trail(V, N, 0.3, 0.7, 9, group=1024, flip_frac=0.1)
    a32, a1024 = oracle.aggregate(codes, 32), oracle.aggregate(codes, 1024)
    assert a1024.shape == (3, V) and a32.shape == (68, V)
    for s in range(3):
        assert np.array_equal(a1024[s], np.bitwise_or.reduce(a32[32 * s: 32 * s + 32], axis=0))
    p32 = oracle.aggregate_pairs(off, lits, codes, group=32, mode=mode)
    p1024 = oracle.aggregate_pairs(off, lits, codes, group=1024, mode=mode)
    sup = set(map(tuple, p1024.tolist()))
    assert all((c, g // 32) in sup for c, g in p32.tolist())
    assert 0 < len(p1024) < 3 * m and len(p32) > 0


def test_pair_matches_pairs(tiny_instance):
    I = tiny_instance
    R = set(map(tuple, oracle.allf_pairs(I.offsets, I.lits, I.codes).tolist()))
    rng = np.random.default_rng(3)
    for c, a in zip(rng.integers(0, I.n_clauses, 500), rng.integers(0, I.n_assign, 500)):
        assert oracle.pair(I.offsets, I.lits, I.codes[a], int(c)) == ((int(c), int(a)) in R)


def test_empty_inputs():
    off = np.zeros(1, np.uint64)
    assert oracle.allf_pairs(off, np.zeros(0, np.uint32), np.zeros((5, 3), np.uint8)).shape == (0, 2)
    off = np.array([0, 2], np.uint64)
    assert oracle.allf_pairs(off, np.array([0, 2], np.uint32), np.zeros((0, 3), np.uint8)).shape == (0, 2)


# Deliberately wrong oracle builds: each must be rejected by at least one pin.
MUTANTS = {1: "wrong sign convention", 2: "drops last literal", 3: "treats U as F",
           4: "skips first literal", 5: "exists instead of for-all", 6: "trigger threshold off by one",
           7: "aggregate all-F takes F or U in G(l)", 8: "aggregate trigger threshold off by one"}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_reject_mutant(mutant, tiny_instance):
    fails = []
    for name in GOLDEN:
        fails += pin_golden(name, mutant=mutant)
    fails += pin_brute_force(3, mutant=mutant)
    fails += pin_aggregate_brute_force(2, mutant=mutant)
    if mutant != 6:
        fails += pin_invariants(tiny_instance, mutant=mutant)
    assert fails, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"


@pytest.mark.parametrize("mutant,mode", [(7, 0), (8, 1)])
def test_aggregate_mutant_is_caught_by_the_set_pin_alone(mutant, mode):
    """Mutants 7 and 8 loosen only an aggregate test (all-F, trigger), which the Theorem of
    Section 4.2 cannot see (it only rules out false negatives): the two-sided pin rejects each
    by itself, while the Theorem still holds for it."""
    inst = synth.tiny()
    m = oracle.MODE_ALLF if mode == 0 else oracle.MODE_TRIGGER
    assert pin_aggregate_theorem(inst, m, group=8, mutant=mutant, max_clauses=500) == []
    assert pin_aggregate_brute_force(2, mutant=mutant) != []


# ---------------------------------------------------------------- clause activity (Section 3.6)
from oracle.activity import ActivityOracle  # noqa: E402


def _csr(sizes, n_vars, seed):
    off = synth.offsets_from_sizes(np.asarray(sizes, np.uint32))
    return off, synth.clause_lits(off, n_vars, seed)


def test_activity_without_decay_counts_reports():
    """decay = 1: every clause ends at 1 + (number of tests that reported it), exactly."""
    rng = np.random.default_rng(1)
    a = ActivityOracle(1.0)
    a.add(*_csr(rng.integers(1, 6, 50), 40, 1))
    counts = np.zeros(50, np.int64)
    for _ in range(30):
        rep = rng.choice(50, size=rng.integers(0, 20), replace=True)  # repeats: one bump per test
        counts[np.unique(rep)] += 1
        a.after_test(rep.astype(np.uint32))
    assert np.array_equal(a.act, (1 + counts).astype(np.float32))


def test_activity_decay_half_is_a_sum_of_powers_of_two():
    """decay = 1/2 doubles inc after each test: a clause added before test 0 and reported in
    tests S holds 1 + sum of 2^t over t in S, and a later report outweighs all earlier ones."""
    rng = np.random.default_rng(2)
    a = ActivityOracle(0.5)
    a.add(*_csr(rng.integers(1, 6, 40), 30, 2))
    want = [1] * 40
    for t in range(20):
        rep = np.nonzero(rng.random(40) < 0.3)[0]
        for c in rep:
            want[c] += 2 ** t
        a.after_test(rep.astype(np.uint32))
    assert [int(x) for x in a.act] == want
    assert a.inc == np.float32(2.0 ** 20)


def test_activity_rescale_keeps_the_order():
    """70 tests at decay 1/2 push inc past 1e20: activities and inc are scaled by 1e-20 and the
    ranking of clauses equals the ranking of the exact integer sums."""
    rng = np.random.default_rng(3)
    a = ActivityOracle(0.5)
    a.add(*_csr(rng.integers(1, 6, 60), 50, 3))
    exact = [1] * 60
    scaled = False
    for t in range(70):
        rep = np.nonzero(rng.random(60) < 0.2)[0]
        for c in rep:
            exact[c] += 2 ** t
        before = a.inc
        a.after_test(rep.astype(np.uint32))
        scaled |= a.inc < before
    assert scaled and a.inc <= np.float32(1e20)
    order_f = sorted(range(60), key=lambda c: (float(a.act[c]), c))
    order_x = sorted(range(60), key=lambda c: (exact[c], c))
    # equal exact sums stay equal; float rounding never swaps two clauses whose sums differ by more than a factor 2^-20
    for i, j in zip(order_f, order_x):
        assert i == j or exact[i] == exact[j] or abs(exact[i] - exact[j]) < max(exact[i], exact[j]) >> 20


def test_reduce_matches_brute_force_and_keeps_short_clauses():
    rng = np.random.default_rng(4)
    a = ActivityOracle(0.9)
    sizes = rng.integers(1, 9, 300)
    a.add(*_csr(sizes, 100, 4))
    for _ in range(12):
        a.after_test(np.nonzero(rng.random(300) < 0.25)[0].astype(np.uint32))
    act_before, ids_before = a.act.copy(), a.ids.copy()
    long_ids = [int(i) for i, s in zip(ids_before, sizes) if s > 2]
    n_remove = int(0.4 * len(long_ids))
    gone = set(sorted(long_ids, key=lambda i: (float(act_before[i]), i))[:n_remove])  # brute force
    assert a.reduce(0.4) == n_remove
    assert set(a.ids.tolist()) == set(range(300)) - gone
    assert all(i in set(a.ids.tolist()) for i, s in zip(ids_before, sizes) if s <= 2)
    assert np.all(np.diff(a.ids.astype(np.int64)) > 0)
    assert np.array_equal(np.diff(a.offsets), sizes[a.ids])
    assert np.array_equal(a.act, act_before[a.ids])


def test_reduce_removes_exactly_the_pairs_of_deleted_clauses():
    inst = synth.tiny()
    a = ActivityOracle(0.95)
    a.add(inst.offsets, inst.lits)
    full = oracle.pairs(inst.offsets, inst.lits, inst.codes)
    a.after_test(full[:, 0])
    a.reduce(0.5)
    kept = set(a.ids.tolist())
    want = full[[int(c) in kept for c in full[:, 0]]]
    assert np.array_equal(a.pairs(inst.codes), want)
    # clauses added after a reduction take new ids; ids are never reused
    first = a.add(inst.offsets[:11], inst.lits[: int(inst.offsets[10])])
    assert first == inst.n_clauses and a.ids[-1] == inst.n_clauses + 9


@pytest.mark.parametrize("n_vars", [1, 2, 3])
def test_aggregate_tests_match_set_definitions(n_vars):
    """Section 4.2, both directions and both modes: over every group of two and three distinct
    assignments out of the 3^V, every clause of up to three literals passes the oracle's
    aggregate test exactly when the definitions, evaluated on the members' value sets, say so."""
    assert pin_aggregate_brute_force(n_vars) == []
