"""The oracle -- TEST INFRASTRUCTURE ONLY.

Plain CPU statement of the clause x assignment tests, written from the paper's
definitions (Section 3.1 truth values and literal values; Section 3.3 "would
have been in conflict" and Definition "triggers"; Section 4.2 aggregates).  See
``gss_oracle.c``.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import this package; the product
path never does.  It shares no code with the CUDA library.

All results are returned as ``(clause, assignment)`` pairs, sorted by clause
then assignment (the set R of the all-F definition is unique; order is only
for comparison).
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gss_oracle.c")
_libs: dict[int, ctypes.CDLL] = {}

MODE_ALLF, MODE_TRIGGER = 0, 1
AGG_T, AGG_F, AGG_U = 1, 2, 4


def lib_path(mutant: int = 0) -> str:
    return os.path.join(_HERE, "libgss_oracle.so" if mutant == 0 else f"libgss_oracle_mutant{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (plain C, pthreads).  ``mutant`` > 0 builds a deliberately wrong
    variant used only to show that the pins reject it."""
    path = lib_path(mutant)
    with open(path + ".lock", "w") as lf:
        fcntl.flock(lf, fcntl.LOCK_EX)
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", f"-DORACLE_MUTANT={mutant}",
                                   "-o", tmp, _SRC, "-lpthread"])
            os.replace(tmp, path)
    return path


def _load(mutant: int = 0) -> ctypes.CDLL:
    if mutant in _libs:
        return _libs[mutant]
    lib = ctypes.CDLL(build(mutant))
    P = ctypes.c_void_p
    u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    lib.gss_oracle_pair.argtypes = [i32, P, P, u64, P]
    lib.gss_oracle_pair.restype = i32
    lib.gss_oracle_pairs.argtypes = [i32, u64, P, P, u32, P, u64, u64, i32,
                                     ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32)),
                                     ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))]
    lib.gss_oracle_pairs.restype = ctypes.c_int64
    lib.gss_oracle_free.argtypes = [P]
    lib.gss_oracle_free.restype = None
    lib.gss_oracle_aggregate.argtypes = [u32, u32, P, u32, P]
    lib.gss_oracle_aggregate.restype = None
    lib.gss_oracle_aggregate_test.argtypes = [i32, P, P, u64, P]
    lib.gss_oracle_aggregate_test.restype = i32
    _libs[mutant] = lib
    return lib


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def sort_pairs(pairs: np.ndarray) -> np.ndarray:
    """Canonical (clause, assignment) order."""
    pairs = np.asarray(pairs, dtype=np.uint32).reshape(-1, 2)
    if len(pairs) == 0:
        return pairs
    key = (pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1].astype(np.uint64)
    return pairs[np.argsort(key, kind="stable")]


def pairs(offsets, lits, codes, mode: int = MODE_ALLF, a_range: tuple[int, int] | None = None,
          threads: int | None = None, mutant: int = 0) -> np.ndarray:
    """All pairs (c, a) passing ``mode`` (all-F by default) for assignments in ``a_range``.
    Returns uint32 [R, 2] sorted by (c, a)."""
    off = _arr(offsets, np.uint64)
    lt = _arr(lits, np.uint32)
    cd = np.ascontiguousarray(codes, dtype=np.uint8)
    n_a, V = cd.shape
    lo, hi = (0, n_a) if a_range is None else a_range
    th = threads or max(1, os.cpu_count() or 1)
    lib = _load(mutant)
    pc = ctypes.POINTER(ctypes.c_uint32)()
    pa = ctypes.POINTER(ctypes.c_uint32)()
    n = lib.gss_oracle_pairs(mode, len(off) - 1, _p(off), _p(lt), V, _p(cd), lo, hi, th,
                             ctypes.byref(pc), ctypes.byref(pa))
    if n < 0:
        raise ValueError("bad assignment range")
    out = np.empty((n, 2), dtype=np.uint32)
    if n:
        out[:, 0] = np.ctypeslib.as_array(pc, shape=(n,))
        out[:, 1] = np.ctypeslib.as_array(pa, shape=(n,))
    lib.gss_oracle_free(ctypes.cast(pc, ctypes.c_void_p))
    lib.gss_oracle_free(ctypes.cast(pa, ctypes.c_void_p))
    return sort_pairs(out)


def allf_pairs(offsets, lits, codes, **kw) -> np.ndarray:
    """Set R of Section 3.3's "would have been in conflict": every literal of c is F under a."""
    return pairs(offsets, lits, codes, MODE_ALLF, **kw)


def trigger_pairs(offsets, lits, codes, **kw) -> np.ndarray:
    """Definition "triggers" (Section 3.3)."""
    return pairs(offsets, lits, codes, MODE_TRIGGER, **kw)


def pair(offsets, lits, codes_row, c: int, mode: int = MODE_ALLF, mutant: int = 0) -> bool:
    """Test one clause against one assignment row (V codes)."""
    off = _arr(offsets, np.uint64)
    lt = _arr(lits, np.uint32)
    row = np.ascontiguousarray(codes_row, dtype=np.uint8)
    return bool(_load(mutant).gss_oracle_pair(mode, _p(off), _p(lt), c, _p(row)))


def aggregate(codes, group: int = 32, mutant: int = 0) -> np.ndarray:
    """Section 4.2 aggregate assignments: uint8 [ceil(N/group), V], bits T=1, F=2, U=4."""
    cd = np.ascontiguousarray(codes, dtype=np.uint8)
    N, V = cd.shape
    G = (N + group - 1) // group
    out = np.empty((G, V), dtype=np.uint8)
    _load(mutant).gss_oracle_aggregate(V, N, _p(cd), group, _p(out))
    return out


def aggregate_pairs(offsets, lits, codes, group: int = 32, mode: int = MODE_ALLF, mutant: int = 0) -> np.ndarray:
    """(clause, group) pairs on which the aggregate test of Section 4.2 is positive, sorted."""
    off = _arr(offsets, np.uint64)
    lt = _arr(lits, np.uint32)
    agg = aggregate(codes, group, mutant=mutant)
    lib = _load(mutant)
    out = []
    for g in range(agg.shape[0]):
        row = np.ascontiguousarray(agg[g])
        for c in range(len(off) - 1):
            if lib.gss_oracle_aggregate_test(mode, _p(off), _p(lt), c, _p(row)):
                out.append((c, g))
    return sort_pairs(np.array(out, dtype=np.uint32).reshape(-1, 2))
