"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and validate records."""
import numpy as np

import paper_2012_03119_gb300 as gss


def gpu_records(inst, mode=gss.GSS_MODE_ALLF, report_capacity=None, max_assignments=None, codes=None,
                clauses_per_tile=0):
    codes = inst.codes if codes is None else codes
    N = codes.shape[0]
    cap = report_capacity or max(1024, inst.n_clauses * max(1, (N + 31) // 32))  # one record per (clause, word) at most
    with gss.Context(inst.n_vars, report_capacity=cap, max_assignments=max_assignments or max(N, 1),
                     mode=mode, clauses_per_tile=clauses_per_tile) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.set_assignments(codes)
        ctx.test()
        return ctx.fetch_reports()


def check_records(rec, m, N):
    """Every record is well formed and (clause, word) pairs are unique."""
    assert (rec["mask"] != 0).all()
    assert (rec["clause_id"] < m).all()
    W = (N + 31) // 32
    assert (rec["word"] < W).all()
    last = rec["word"] == W - 1
    if N % 32:
        assert (rec["mask"][last] >> np.uint32(N % 32) == 0).all(), "bit for a nonexistent assignment"
    key = rec["clause_id"].astype(np.uint64) << np.uint64(32) | rec["word"].astype(np.uint64)
    assert len(np.unique(key)) == len(key), "duplicate (clause, word) record"


def pair_keys(pairs):
    """(clause, assignment) pairs as sorted uint64 keys."""
    p = np.asarray(pairs).reshape(-1, 2)
    return np.sort((p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64))


def contains_all(pairs, wanted):
    """Every pair of `wanted` is among `pairs` (vectorised; no Python sets)."""
    k, w = pair_keys(pairs), pair_keys(wanted)
    if len(w) == 0:
        return True
    if len(k) == 0:
        return False
    i = np.minimum(np.searchsorted(k, w), len(k) - 1)
    return bool(np.all(k[i] == w))


def gpu_pairs(inst, **kw):
    rec = gpu_records(inst, **kw)
    codes = kw.get("codes", inst.codes)
    check_records(rec, inst.n_clauses, codes.shape[0])
    return gss.expand_reports(rec)
