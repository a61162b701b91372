"""Pins for the oracle: checks against what the paper and the mathematics fix,
independent of the oracle's own code.  Each pin returns a list of failure
messages (empty = pass) so that the same pins can be run against deliberately
wrong oracle builds (``mutant``) to show that they catch plausible mistakes.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CODE = {"U": 0, "T": 1, "F": 2}


# --------------------------------------------------------------- golden files
def parse_golden(name: str) -> list[dict]:
    """Parse a worked-example fixture into a list of checks."""
    names: dict[str, int] = {}
    checks: list[dict] = []
    cur_assign = None
    group: list[np.ndarray] = []
    for raw in open(os.path.join(GOLDEN, name)):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        kind = tok[0]
        if kind == "vars":
            names = {n: i for i, n in enumerate(tok[1:])}
        elif kind == "group":
            group = []
        elif kind == "assign":
            row = np.zeros(len(names), np.uint8)
            for t in tok[1:]:
                k, v = t.split("=")
                row[names[k]] = CODE[v]
            cur_assign = row
            group.append(row)
        elif kind in ("expect", "expect_each", "expect_group"):
            lits = []
            for t in tok[1].split("|"):
                neg = t.startswith("-")
                lits.append(2 * names[t.lstrip("-")] + (1 if neg else 0))
            exp = {}
            for t in tok[2:]:
                k, v = t.split("=")
                exp[k] = [int(x) for x in v.split(",")]
            checks.append(dict(kind=kind, lits=lits, expect=exp, assign=cur_assign,
                               group=[g.copy() for g in group], text=line))
        elif kind == "expect_aggregate":
            exp = {}
            for t in tok[1:]:
                k, v = t.split("=")
                exp[names[k]] = set(v)
            checks.append(dict(kind=kind, expect=exp, group=[g.copy() for g in group], text=line))
        else:
            raise ValueError(f"bad golden line: {line}")
    return checks


def _one_clause_db(lits):
    return np.array([0, len(lits)], np.uint64), np.array(lits, np.uint32)


def pin_golden(name: str, mutant: int = 0) -> list[str]:
    fails = []
    modes = {"allf": oracle.MODE_ALLF, "trigger": oracle.MODE_TRIGGER}
    for ch in parse_golden(name):
        if ch["kind"] == "expect":
            off, lt = _one_clause_db(ch["lits"])
            for key, want in ch["expect"].items():
                got = int(oracle.pair(off, lt, ch["assign"], 0, modes[key], mutant=mutant))
                if got != want[0]:
                    fails.append(f"{name}: {ch['text']}: {key} got {got}")
        elif ch["kind"] == "expect_each":
            off, lt = _one_clause_db(ch["lits"])
            for key, want in ch["expect"].items():
                got = [int(oracle.pair(off, lt, g, 0, modes[key], mutant=mutant)) for g in ch["group"]]
                if got != want:
                    fails.append(f"{name}: {ch['text']}: {key} got {got}")
        elif ch["kind"] == "expect_group":
            off, lt = _one_clause_db(ch["lits"])
            codes = np.stack(ch["group"])
            for key, want in ch["expect"].items():
                got = len(oracle.aggregate_pairs(off, lt, codes, group=len(codes), mode=modes[key], mutant=mutant)) > 0
                if int(got) != want[0]:
                    fails.append(f"{name}: {ch['text']}: aggregate {key} got {int(got)}")
        elif ch["kind"] == "expect_aggregate":
            codes = np.stack(ch["group"])
            agg = oracle.aggregate(codes, group=len(codes), mutant=mutant)[0]
            for v, want in ch["expect"].items():
                got = {c for bit, c in ((1, "T"), (2, "F"), (4, "U")) if agg[v] & bit}
                if got != want:
                    fails.append(f"{name}: {ch['text']}: var {v} aggregate {sorted(got)}")
    return fails


# --------------------------------------------------------------- brute force
def all_assignments(n_vars: int) -> np.ndarray:
    """Every one of the 3^V three-valued assignments, uint8 [3^V, V]."""
    return np.array(list(itertools.product([0, 1, 2], repeat=n_vars)), np.uint8).reshape(-1, n_vars)


def all_small_clauses(n_vars: int, max_size: int = 3):
    """Every clause of 1..max_size distinct literals over 2V literals (tautologies included)."""
    out = []
    for s in range(1, max_size + 1):
        out.extend(itertools.combinations(range(2 * n_vars), s))
    return out


def pin_brute_force(n_vars: int, mutant: int = 0, max_size: int = 3) -> list[str]:
    """Closed forms from the definitions: a clause whose literals are all on distinct
    variables is all-F exactly on the assignments that give each variable its
    falsifying value (F for l = v, T for l = not v): 3^(V-k) of them for k literals;
    it triggers exactly when at most one of its variables is U instead:
    (1 + k) * 3^(V-k) assignments.  A clause holding l and not l never does either."""
    fails = []
    A = all_assignments(n_vars)
    clauses = all_small_clauses(n_vars, max_size)
    off = np.zeros(len(clauses) + 1, np.uint64)
    off[1:] = np.cumsum([len(c) for c in clauses])
    lits = np.array([l for c in clauses for l in c], np.uint32)
    R = oracle.pairs(off, lits, A, oracle.MODE_ALLF, mutant=mutant, threads=2)
    T = oracle.pairs(off, lits, A, oracle.MODE_TRIGGER, mutant=mutant, threads=2)
    hits_allf = {c: set() for c in range(len(clauses))}
    for c, a in R:
        hits_allf[int(c)].add(int(a))
    hits_trig = {c: set() for c in range(len(clauses))}
    for c, a in T:
        hits_trig[int(c)].add(int(a))
    for ci, cl in enumerate(clauses):
        vs = [l >> 1 for l in cl]
        taut = len(set(vs)) < len(vs)
        k = len(cl)
        if taut:
            exp_allf, exp_trig = set(), set()
        else:
            need = np.array([2 if (l & 1) == 0 else 1 for l in cl], np.uint8)  # F for v, T for not v
            sub = A[:, vs]
            match = sub == need
            exp_allf = set(np.nonzero(match.all(axis=1))[0].tolist())
            undef = sub == 0
            exp_trig = set(np.nonzero((match | undef).all(axis=1) & (undef.sum(axis=1) <= 1))[0].tolist())
            if len(exp_allf) != 3 ** (n_vars - k) or len(exp_trig) != (1 + k) * 3 ** (n_vars - k):
                fails.append(f"closed form count mismatch for {cl}")  # guards the pin itself
        if hits_allf[ci] != exp_allf:
            fails.append(f"V={n_vars} clause {cl}: all-F set differs ({len(hits_allf[ci])} vs {len(exp_allf)})")
        if hits_trig[ci] != exp_trig:
            fails.append(f"V={n_vars} clause {cl}: trigger set differs ({len(hits_trig[ci])} vs {len(exp_trig)})")
    return fails


# --------------------------------------------------------------- invariants
def falsifying_partial(lits) -> dict[int, int] | None:
    """The unique partial assignment under which every literal is F (None for a tautology)."""
    need: dict[int, int] = {}
    for l in lits:
        v, val = int(l) >> 1, (2 if (int(l) & 1) == 0 else 1)
        if need.get(v, val) != val:
            return None
        need[v] = val
    return need


def recount_clause_major(offsets, lits, codes) -> np.ndarray:
    """R recomputed clause by clause from each clause's falsifying partial assignment
    (a different loop order and a different formulation from the oracle's)."""
    out = []
    for c in range(len(offsets) - 1):
        need = falsifying_partial(lits[int(offsets[c]):int(offsets[c + 1])])
        if need is None:
            continue
        vs = np.fromiter(need.keys(), np.int64)
        vals = np.fromiter(need.values(), np.uint8)
        hit = np.nonzero((codes[:, vs] == vals).all(axis=1))[0]
        out.extend((c, int(a)) for a in hit)
    return oracle.sort_pairs(np.array(out, np.uint32).reshape(-1, 2))


def pin_invariants(inst, mutant: int = 0) -> list[str]:
    fails = []
    R = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, mutant=mutant)
    # a clause holding l and not l is never all-F
    taut = [c for c in range(inst.n_clauses)
            if falsifying_partial(inst.lits[int(inst.offsets[c]):int(inst.offsets[c + 1])]) is None]
    if len(taut) < len(inst.tautologies):
        fails.append("generator tautologies not detected")
    if np.isin(R[:, 0], np.array(taut, np.uint32)).any():
        fails.append("a tautology was reported")
    # the all-U assignment reports nothing
    if len(inst.all_u) and np.isin(R[:, 1], inst.all_u).any():
        fails.append("the all-U assignment reported a hit")
    # every planted pair is found
    got = set(map(tuple, R.tolist()))
    missing = [tuple(p) for p in inst.planted.tolist() if tuple(p) not in got]
    if missing:
        fails.append(f"{len(missing)} planted pairs missing")
    # recount in clause-major order from falsifying partial assignments
    R2 = recount_clause_major(inst.offsets, inst.lits, inst.codes)
    if R.shape != R2.shape or not np.array_equal(R, R2):
        fails.append(f"clause-major recount differs: {len(R)} vs {len(R2)}")
    return fails


def pin_monotone(inst, mutant: int = 0, n_changes: int = 200, seed: int = 7) -> list[str]:
    """Setting a U variable to T or F keeps every hit and only adds hits of clauses
    that contain that variable."""
    fails = []
    rng = np.random.default_rng(seed)
    R = set(map(tuple, oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, mutant=mutant).tolist()))
    codes = inst.codes.copy()
    N, V = codes.shape
    us = np.argwhere(codes == 0)
    pick = us[rng.choice(len(us), size=min(n_changes, len(us)), replace=False)]
    changed = {}
    for a, v in pick:
        codes[a, v] = rng.integers(1, 3)
        changed.setdefault(int(a), set()).add(int(v))
    R2 = set(map(tuple, oracle.allf_pairs(inst.offsets, inst.lits, codes, mutant=mutant).tolist()))
    if not R <= R2:
        fails.append("a hit disappeared after setting U variables")
    for c, a in R2 - R:
        vs = {int(l) >> 1 for l in inst.lits[int(inst.offsets[c]):int(inst.offsets[c + 1])]}
        if not vs & changed.get(a, set()):
            fails.append(f"new hit ({c},{a}) does not involve a changed variable")
            break
    return fails


def pin_aggregate_theorem(inst, mode: int, group: int = 32, mutant: int = 0, max_clauses: int = 3000) -> list[str]:
    """Theorem of Section 4.2: a clause that passes on some assignment of a group passes on
    the group's aggregate (no false negatives of the group prefilter)."""
    fails = []
    m = min(inst.n_clauses, max_clauses)
    off = inst.offsets[: m + 1]
    lt = inst.lits[: int(off[-1])]
    indiv = oracle.pairs(off, lt, inst.codes, mode, mutant=mutant)
    aggp = set(map(tuple, oracle.aggregate_pairs(off, lt, inst.codes, group=group, mode=mode).tolist()))
    for c, a in indiv.tolist():
        if (c, a // group) not in aggp:
            fails.append(f"pair ({c},{a}) passes but its group aggregate does not")
            break
    return fails


def _member_values(group_rows: np.ndarray, lit: int) -> set[str]:
    """The values the members of a group give literal lit = 2v + s, read member by member
    (Section 3.1: the literal takes v's value when s = 0 and its negation when s = 1)."""
    v, neg = lit >> 1, lit & 1
    name = {0: "U", 1: "T", 2: "F"}
    flip = {"T": "F", "F": "T", "U": "U"}
    vals = {name[int(x)] for x in group_rows[:, v]}
    return {flip[x] for x in vals} if neg else vals


def aggregate_by_members(group_rows: np.ndarray, clause, mode: int) -> bool:
    """Section 4.2 on sets, without the oracle's bit encoding: G(l) is the set of values the
    members give l.  All-F (the all-F restriction of aggregateTrigger): F is in G(l) for every
    literal.  Trigger (the Definition of Section 4.2): F or U is in G(l) for every literal, and
    F is in G(l) for at least s - 1 of them."""
    sets = [_member_values(group_rows, l) for l in clause]
    if mode == oracle.MODE_ALLF:
        return all("F" in g for g in sets)
    return all(("F" in g) or ("U" in g) for g in sets) and sum("F" in g for g in sets) + 1 >= len(clause)


def pin_aggregate_brute_force(n_vars: int, sizes=(2, 3), mutant: int = 0, max_groups: int | None = None) -> list[str]:
    """Both directions of the aggregate tests: for every group of distinct assignments (of each
    size in `sizes`) out of the 3^V, and every clause of 1..3 distinct literals, the oracle's
    aggregate test is positive exactly when the set definition above says so."""
    fails = []
    A = all_assignments(n_vars)
    clauses = all_small_clauses(n_vars, 3)
    off = np.zeros(len(clauses) + 1, np.uint64)
    off[1:] = np.cumsum([len(c) for c in clauses])
    lits = np.array([l for c in clauses for l in c], np.uint32)
    for k in sizes:
        groups = list(itertools.combinations(range(len(A)), k))
        if max_groups is not None and len(groups) > max_groups:
            pick = np.random.default_rng(k).choice(len(groups), size=max_groups, replace=False)
            groups = [groups[i] for i in sorted(pick)]
        codes = np.concatenate([A[list(g)] for g in groups])  # group j = rows k*j .. k*j + k - 1
        for mode in (oracle.MODE_ALLF, oracle.MODE_TRIGGER):
            got = set(map(tuple, oracle.aggregate_pairs(off, lits, codes, group=k, mode=mode, mutant=mutant).tolist()))
            for j, g in enumerate(groups):
                rows = A[list(g)]
                for ci, cl in enumerate(clauses):
                    want = aggregate_by_members(rows, cl, mode)
                    if ((ci, j) in got) != want:
                        fails.append(f"V={n_vars} group {g} clause {cl} mode {mode}: aggregate test "
                                     f"{'positive' if not want else 'negative'}, set definition says {want}")
                        if len(fails) > 5:
                            return fails
    return fails
