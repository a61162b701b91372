"""One clause database over several GPUs, one process per GPU.

Every (clause, assignment) pair is decided by that clause alone (Section 3.5: GPU threads test
different clauses independently), so a database splits into clause ranges and the test needs
no exchange: each rank holds one range, tests it against the same assignment set, offsets its
clause ids to global ids, and the per-rank record sets -- disjoint by construction -- are
concatenated.  The only collective is the final gather of the records.

    ranges = clause_ranges(offsets, world)                 # the same on every rank
    lo, hi = ranges[rank]
    ctx.add_clauses(*local_csr(offsets, lits, lo, hi))     # ids 0 .. hi - lo - 1 on this rank
    ctx.run(codes)
    rec = globalize(ctx.fetch_reports(), lo)               # global clause ids
    all_rec = gather_records(rec, dist)                    # on rank 0: every rank's records

Host-side marshalling only: the test itself runs in the library's kernels on each rank.
"""
from __future__ import annotations

import numpy as np

from . import REPORT_DTYPE


def clause_ranges(offsets, world: int, per_clause: int = 0) -> list[tuple[int, int]]:
    """Split clauses [0, m) into `world` contiguous ranges of about equal cost, the cost of a
    clause being its literal count plus `per_clause`.  Cut k is the first clause whose
    cumulative cost reaches k / world of the total, so every range's cost is within one clause
    of the ideal share.  Ranges may be empty when there are fewer clauses than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    off = np.asarray(offsets, dtype=np.uint64)
    m = len(off) - 1
    cost = off.astype(np.float64) + per_clause * np.arange(m + 1, dtype=np.float64)  # cumulative cost before clause c
    total = cost[-1]
    cuts = [0]
    for k in range(1, world):
        c = int(np.searchsorted(cost, total * k / world, side="left"))
        cuts.append(min(max(c, cuts[-1]), m))
    cuts.append(m)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def local_csr(offsets, lits, lo: int, hi: int) -> tuple[np.ndarray, np.ndarray]:
    """The CSR of clauses [lo, hi), offsets rebased to 0 (clause lo becomes local id 0)."""
    off = np.asarray(offsets, dtype=np.uint64)
    b, e = int(off[lo]), int(off[hi])
    return (off[lo:hi + 1] - off[lo]).astype(np.uint64), np.ascontiguousarray(np.asarray(lits)[b:e], dtype=np.uint32)


def globalize(records: np.ndarray, lo: int) -> np.ndarray:
    """Records of a rank holding clauses [lo, hi) with their local ids -> global clause ids."""
    out = np.array(records, dtype=REPORT_DTYPE, copy=True)
    if lo and len(out):
        if int(out["clause_id"].max()) + lo >= 1 << 32:
            raise ValueError("global clause id does not fit in 32 bits")
        out["clause_id"] += np.uint32(lo)
    return out


def gather_records(records: np.ndarray, dist=None, dst: int = 0) -> np.ndarray | None:
    """Concatenate every rank's records on rank `dst` (None on the other ranks).  The ranks'
    sets are disjoint (each holds its own clauses), so no de-duplication or reduction is
    needed.  Without a process group the records are returned as they are."""
    rec = np.asarray(records, dtype=REPORT_DTYPE)
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return rec
    parts = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object(rec.tobytes(), parts, dst=dst)
    if dist.get_rank() != dst:
        return None
    return np.concatenate([np.frombuffer(p, dtype=REPORT_DTYPE) for p in parts])
