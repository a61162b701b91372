"""The seeded input generator: determinism and the recipe's shapes (CPU only)."""
import numpy as np

import synth


def test_deterministic(tiny_instance):
    again = synth.tiny()
    assert synth.content_hash(tiny_instance.offsets, tiny_instance.lits, tiny_instance.codes) == \
        synth.content_hash(again.offsets, again.lits, again.codes)
    assert np.array_equal(tiny_instance.planted, again.planted)


def test_tiny_shape(tiny_instance):
    I = tiny_instance
    sz = np.diff(I.offsets)
    assert I.n_clauses == 20000 and I.n_vars == 2000 and I.n_assign == 64
    assert sz.min() >= 2 and sz.max() <= 30 and 7.0 < sz.mean() < 8.2
    assert len(I.planted) == 200 and len(I.tautologies) == 50
    assert (I.codes[I.all_u] == 0).all()
    assert I.lits.max() < 2 * I.n_vars


def test_no_duplicate_literals(tiny_instance):
    I = tiny_instance
    for c in range(0, I.n_clauses, 7):
        cl = I.lits[I.offsets[c]:I.offsets[c + 1]]
        assert len(np.unique(cl)) == len(cl)


def test_lognormal_and_trail():
    I = synth.single(scale=0.01)
    sz = np.diff(I.offsets)
    assert 18 <= np.median(sz) <= 22 and sz.max() <= 500 and sz.min() >= 2
    frac = (I.codes != 0).mean(axis=1)
    assert frac.min() > 0.28 and frac.max() < 0.75  # 30-70 % assigned (+ planted forcing)


def test_planted_literals_false():
    I = synth.single(scale=0.005)
    for c, a in I.planted[:100]:
        for l in I.lits[I.offsets[c]:I.offsets[c + 1]]:
            assert I.codes[a, l >> 1] == (2 if l % 2 == 0 else 1)


def test_communities():
    I = synth.structured(scale=0.002)  # 2 communities of 10k vars, 20k clauses
    assert I.n_vars == 20000 and I.n_clauses == 20000
    sz = np.diff(I.offsets)
    assert 35 <= np.median(sz) <= 45 and sz.max() <= 1000
