"""The oracle for clause activity and deletion -- TEST INFRASTRUCTURE ONLY.

Section 3.6 says the GPU deletes clauses by activity, the way MiniSat does on the CPU, and
bumps a clause's activity whenever it triggers.  The paper gives no constants, so this
statement takes MiniSat's scheme with these readings:

* a clause's activity is an IEEE single-precision number; a clause starts at the current
  increment `inc` when it is added (MiniSat bumps a learnt clause once when it is created);
* after every test, each clause reported for at least one assignment of that test is bumped
  once: activity <- activity + inc (one addition per clause per test, in single precision);
* then inc <- inc * (1 / decay), with 1 / decay computed once in single precision; when inc
  exceeds 1e20 every activity and inc are multiplied by 1e-20 (single precision);
* reducing removes floor(f * n) of the n clauses with more than two literals, f the removed
  fraction: those whose key (activity, clause id) is smallest, where the activity's IEEE bit
  pattern orders keys (all activities are non-negative).  Clauses of one or two literals are
  always kept.  Kept clauses keep their ids and their relative order; ids are never reused.

Plain numpy in float32, in the order the steps are stated; shares no code with the library.
"""
from __future__ import annotations

import math

import numpy as np

RESCALE_LIMIT = np.float32(1e20)
RESCALE_BY = np.float32(1e-20)


class ActivityOracle:
    """A clause database with MiniSat-style activities, tracked step by step."""

    def __init__(self, decay: float):
        self.decay = np.float32(decay)
        self.inv_decay = np.float32(np.float32(1.0) / self.decay)
        self.inc = np.float32(1.0)
        self.offsets = np.zeros(1, np.uint64)
        self.lits = np.zeros(0, np.uint32)
        self.ids = np.zeros(0, np.uint32)
        self.act = np.zeros(0, np.float32)
        self.next_id = 0

    @property
    def n_clauses(self) -> int:
        return len(self.ids)

    def add(self, offsets, lits) -> int:
        """Append clauses (CSR, offsets[0] = 0); each starts at activity inc.  Returns the first id."""
        off = np.asarray(offsets, np.uint64)
        n = len(off) - 1
        first = self.next_id
        self.offsets = np.concatenate([self.offsets, self.offsets[-1] + off[1:]])
        self.lits = np.concatenate([self.lits, np.asarray(lits, np.uint32)])
        self.ids = np.concatenate([self.ids, np.arange(first, first + n, dtype=np.uint32)])
        self.act = np.concatenate([self.act, np.full(n, self.inc, np.float32)])
        self.next_id += n
        return first

    def after_test(self, reported_ids) -> None:
        """Bump every clause reported by one test (ids, any multiplicity), then decay."""
        hit = np.isin(self.ids, np.unique(np.asarray(reported_ids, np.uint32)))
        self.act[hit] = (self.act[hit] + self.inc).astype(np.float32)
        self.inc = np.float32(self.inc * self.inv_decay)
        if self.inc > RESCALE_LIMIT:
            self.act = (self.act * RESCALE_BY).astype(np.float32)
            self.inc = np.float32(self.inc * RESCALE_BY)

    def reduce(self, remove_fraction: float) -> int:
        """Remove floor(f * n) of the n long clauses with the smallest (activity, id) keys."""
        sizes = np.diff(self.offsets).astype(np.int64)
        long_ = np.nonzero(sizes > 2)[0]
        n_remove = int(math.floor(remove_fraction * len(long_)))
        keep = np.ones(self.n_clauses, bool)
        if n_remove > 0:
            bits = self.act[long_].view(np.uint32).astype(np.uint64)
            order = np.lexsort((self.ids[long_].astype(np.uint64), bits))  # activity first, then id
            keep[long_[order[:n_remove]]] = False
        self._compact(keep)
        return n_remove

    def _compact(self, keep: np.ndarray) -> None:
        sizes = np.diff(self.offsets).astype(np.int64)
        kept = np.nonzero(keep)[0]
        self.lits = self.lits[np.repeat(keep, sizes)]  # every literal of a kept clause, in order
        self.offsets = np.concatenate([[0], np.cumsum(sizes[kept])]).astype(np.uint64)
        self.ids = self.ids[kept]
        self.act = self.act[kept]

    def pairs(self, codes, mode: int = 0) -> np.ndarray:
        """(clause id, assignment) pairs of the resident clauses, sorted (the oracle's definitions)."""
        from . import pairs as oracle_pairs, sort_pairs
        p = oracle_pairs(self.offsets, self.lits, codes, mode)
        if len(p) == 0:
            return p
        p = p.copy()
        p[:, 0] = self.ids[p[:, 0]]
        return sort_pairs(p)
