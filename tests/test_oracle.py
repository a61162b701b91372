"""The oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle
import synth
from pins import (pin_aggregate_theorem, pin_brute_force, pin_golden, pin_invariants, pin_monotone)

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
           4: "skips first literal", 5: "exists instead of for-all", 6: "trigger threshold off by one"}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_reject_mutant(mutant, tiny_instance):
    fails = []
    for name in GOLDEN:
        fails += pin_golden(name, mutant=mutant)
    fails += pin_brute_force(3, mutant=mutant)
    if mutant != 6:
        fails += pin_invariants(tiny_instance, mutant=mutant)
    assert fails, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"
