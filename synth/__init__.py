"""Seeded synthetic workloads for the clause x assignment all-F test.

A module of its own: it draws clause databases and three-valued assignments and
holds none of the tested method's arithmetic.  The oracle tests and the CUDA
path both consume its arrays; it imports neither of them.

Shapes follow the paper's workload statistics: learned clauses are often 20 or
more literals long (Section 5), a GPU run tests up to 1024 assignments in groups
of 32 sent by one solver thread (Section 4.3), successive assignments of one
thread share most values (Section 4.1, commonality table), and about 5 M
clauses sit on the GPU (Section 5).  Value codes: 0 = U, 1 = T, 2 = F, stored
row-major ``codes[a, v]``.  Literals: ``l = 2 v + s`` with ``s = 1`` negated.
"""
from __future__ import annotations

import ctypes
import fcntl
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gss_synth.c")
_LIB_PATH = os.path.join(_HERE, "libgss_synth.so")
_lib = None

CODE_U, CODE_T, CODE_F = 0, 1, 2
SEED_BASE = 0x65535300


def seed_for(config: int, instance: int = 0) -> int:
    """Seed of instance ``instance`` of workload ``config`` (1..5)."""
    return SEED_BASE + config * 1000 + instance


def build(force: bool = False) -> str:
    """Compile the generator (plain C, pthreads) next to its source."""
    lock = _LIB_PATH + ".lock"
    with open(lock, "w") as lf:
        fcntl.flock(lf, fcntl.LOCK_EX)
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lpthread"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    u64, u32, i32, f64 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
    lib.synth_sizes.argtypes = [u64, i32, f64, f64, u32, u32, u64, i32, P]
    lib.synth_sizes.restype = i32
    lib.synth_lits.argtypes = [u64, P, u32, f64, u32, u32, f64, u32, u64, i32, P]
    lib.synth_lits.restype = i32
    lib.synth_assign_indep.argtypes = [u32, u32, f64, u64, i32, P]
    lib.synth_assign_indep.restype = i32
    lib.synth_assign_trail.argtypes = [u32, u32, u32, f64, f64, f64, u64, i32, P]
    lib.synth_assign_trail.restype = i32
    lib.synth_plant.argtypes = [u64, P, P, u32, u32, P, P, u64, u64, P, P]
    lib.synth_plant.restype = ctypes.c_int64
    lib.synth_tautologies.argtypes = [u64, P, P, u64, u64, P]
    lib.synth_tautologies.restype = ctypes.c_int64
    lib.synth_hash.argtypes = [P, u64, i32]
    lib.synth_hash.restype = u64
    _lib = lib
    return lib


def _threads() -> int:
    return max(1, os.cpu_count() or 1)


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# ------------------------------------------------------------------ primitives
def clause_sizes(m: int, law: str, p1: float, p2: float, cap: int, n_vars: int, seed: int) -> np.ndarray:
    """Clause sizes: ``law='geom'``: 2 + Geom(p1) redrawn above cap; ``'lognormal'``:
    clamp(round(exp(ln p1 + p2 Z)), 2, cap).  Never more than 2*n_vars."""
    out = np.empty(m, dtype=np.uint32)
    law_id = {"geom": 0, "lognormal": 1}[law]
    _load().synth_sizes(m, law_id, p1, p2, cap, min(2 * n_vars, 2**32 - 1), seed, _threads(), _ptr(out))
    return out


def offsets_from_sizes(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, dtype=np.uint64)
    np.cumsum(sizes, dtype=np.uint64, out=off[1:])
    return off


def clause_lits(offsets: np.ndarray, n_vars: int, seed: int, zipf_s: float = 1.1, n_comm: int = 0,
                comm_size: int = 0, p_home: float = 0.0) -> np.ndarray:
    """Literals for every clause: Zipf(zipf_s) variables through a seeded permutation, fair-coin
    signs, exact duplicates redrawn; optional communities (see gss_synth.c)."""
    m = len(offsets) - 1
    lits = np.empty(int(offsets[-1]), dtype=np.uint32)
    max_size = int(np.max(np.diff(offsets))) if m else 1
    _load().synth_lits(m, _ptr(offsets), n_vars, zipf_s, n_comm, comm_size, p_home, max_size, seed,
                       _threads(), _ptr(lits))
    return lits


def assign_indep(n_vars: int, n_assign: int, p_set: float, seed: int) -> np.ndarray:
    codes = np.empty((n_assign, n_vars), dtype=np.uint8)
    _load().synth_assign_indep(n_vars, n_assign, p_set, seed, _threads(), _ptr(codes))
    return codes


def assign_trail(n_vars: int, n_assign: int, lo: float, hi: float, seed: int, group: int = 32,
                 flip_frac: float = 0.02) -> np.ndarray:
    codes = np.empty((n_assign, n_vars), dtype=np.uint8)
    _load().synth_assign_trail(n_vars, n_assign, group, lo, hi, flip_frac, seed, _threads(), _ptr(codes))
    return codes


def plant(offsets: np.ndarray, lits: np.ndarray, codes: np.ndarray, k: int, seed: int,
          exclude: np.ndarray | None = None) -> np.ndarray:
    """Force k distinct (clause, assignment) pairs to be all-F hits (modifies codes). Returns [k, 2]."""
    n_assign, n_vars = codes.shape
    out_c = np.empty(max(k, 1), dtype=np.uint32)
    out_a = np.empty(max(k, 1), dtype=np.uint32)
    ex = None if exclude is None else np.ascontiguousarray(exclude, dtype=np.uint8)
    got = _load().synth_plant(len(offsets) - 1, _ptr(offsets), _ptr(lits), n_vars, n_assign, _ptr(codes),
                              None if ex is None else _ptr(ex), k, seed, _ptr(out_c), _ptr(out_a))
    return np.stack([out_c[:got], out_a[:got]], axis=1)


def tautologies(offsets: np.ndarray, lits: np.ndarray, count: int, seed: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.uint32)
    got = _load().synth_tautologies(len(offsets) - 1, _ptr(offsets), _ptr(lits), count, seed, _ptr(out))
    return np.sort(out[:got])


def content_hash(*arrays: np.ndarray) -> str:
    h = 0
    for a in arrays:
        a = np.ascontiguousarray(a)
        h = (h * 0x100000001B3 ^ int(_load().synth_hash(_ptr(a.view(np.uint8).reshape(-1)), a.nbytes,
                                                         _threads()))) & (2**64 - 1)
    return f"{h:016x}"


# ------------------------------------------------------------------ instances
@dataclass
class Instance:
    """One clause database plus one assignment set."""
    name: str
    n_vars: int
    offsets: np.ndarray          # uint64 [m + 1], offsets[0] = 0
    lits: np.ndarray             # uint32 [L], l = 2 v + s
    codes: np.ndarray            # uint8 [N, V], 0 = U, 1 = T, 2 = F
    planted: np.ndarray          # uint32 [K, 2] (clause, assignment) pairs forced to be hits
    tautologies: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))
    all_u: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))
    params: dict = field(default_factory=dict)

    @property
    def n_clauses(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_assign(self) -> int:
        return self.codes.shape[0]

    @property
    def n_lits(self) -> int:
        return int(self.offsets[-1])


def tiny(seed: int | None = None, n_vars: int = 2000, n_clauses: int = 20000, n_assign: int = 64,
         n_planted: int = 200, n_taut: int = 50) -> Instance:
    """Plain test, tiny: 2,000 vars, 20,000 clauses of geometric size 2 + Geom(1/7) (mean 8,
    redrawn above 30), Zipf(1.1) vars, fair signs; 64 independent assignments, each variable
    set with probability 0.5 then T/F 1/2 each; 50 clauses made explicit tautologies, the
    last assignment replaced by all-U, 200 planted pairs."""
    s = seed_for(1) if seed is None else seed
    sizes = clause_sizes(n_clauses, "geom", 1.0 / 7.0, 0.0, 30, n_vars, s)
    off = offsets_from_sizes(sizes)
    lits = clause_lits(off, n_vars, s)
    taut = tautologies(off, lits, n_taut, s)
    codes = assign_indep(n_vars, n_assign, 0.5, s)
    all_u = np.array([n_assign - 1], dtype=np.uint32) if n_assign else np.zeros(0, np.uint32)
    codes[all_u] = CODE_U
    ex = np.zeros(n_assign, np.uint8)
    ex[all_u] = 1
    pl = plant(off, lits, codes, n_planted, s, exclude=ex)
    return Instance("tiny", n_vars, off, lits, codes, pl, taut, all_u,
                    dict(config=1, seed=s, sizes="geom(1/7)+2<=30", zipf=1.1, assign="indep p_set=0.5"))


def single(scale: float = 1.0, seed: int | None = None, n_assign: int = 1024) -> Instance:
    """Plain test, single instance: 1M vars, 4M clauses, lognormal sizes (median 20, sigma 1,
    clamped to [2, 500]), Zipf(1.1) vars; 1024 assignments as 32 trail-prefix groups with
    30-70 % assigned; 10k planted pairs.  ``scale`` shrinks V, m and K together."""
    s = seed_for(2) if seed is None else seed
    V = max(64, int(round(1_000_000 * scale)))
    m = max(1, int(round(4_000_000 * scale)))
    K = max(1, int(round(10_000 * scale)))
    sizes = clause_sizes(m, "lognormal", 20.0, 1.0, 500, V, s)
    off = offsets_from_sizes(sizes)
    lits = clause_lits(off, V, s)
    codes = assign_trail(V, n_assign, 0.30, 0.70, s)
    pl = plant(off, lits, codes, K, s)
    return Instance(f"single(scale={scale:g})", V, off, lits, codes, pl, params=dict(
        config=2, seed=s, scale=scale, sizes="lognormal(20,1)[2,500]", zipf=1.1,
        assign="trail groups of 32, f~U[0.30,0.70], 2% flips"))


def structured(scale: float = 1.0, seed: int | None = None, n_assign: int = 1024) -> Instance:
    """Large structured: 10M vars in 1,000 communities of 10k vars; 10M clauses with lognormal
    sizes (median 40, sigma 1, clamped to [2, 1000]); each clause has a home community drawn by
    Zipf(1.1) over communities, each literal comes from it (uniformly) with probability 0.8, else
    from the global Zipf(1.1); 1024 trail-prefix assignments (30-70 % assigned); 10k planted.
    ``scale`` shrinks V (community size fixed at 10k), m and K together."""
    s = seed_for(5) if seed is None else seed
    comm_size = 10_000
    n_comm = max(1, int(round(1000 * scale)))
    V = n_comm * comm_size
    m = max(1, int(round(10_000_000 * scale)))
    K = max(1, int(round(10_000 * scale)))
    sizes = clause_sizes(m, "lognormal", 40.0, 1.0, 1000, V, s)
    off = offsets_from_sizes(sizes)
    lits = clause_lits(off, V, s, n_comm=n_comm, comm_size=comm_size, p_home=0.8)
    codes = assign_trail(V, n_assign, 0.30, 0.70, s)
    pl = plant(off, lits, codes, K, s)
    return Instance(f"structured(scale={scale:g})", V, off, lits, codes, pl, params=dict(
        config=5, seed=s, scale=scale, sizes="lognormal(40,1)[2,1000]", communities=f"{n_comm}x{comm_size}",
        p_home=0.8, zipf=1.1, assign="trail groups of 32, f~U[0.30,0.70], 2% flips"))


def wide(scale: float = 1.0, seed: int | None = None, n_assign: int = 8192, group: int = 1024) -> Instance:
    """Wide assignment set: the single-instance database (1M vars, 4M clauses, lognormal sizes
    median 20, sigma 1, clamped to [2, 500], Zipf(1.1) vars) against n_assign assignments in
    trail-prefix groups of ``group`` (one simulated solver thread's successive snapshots each,
    30-70 % assigned, the last 10 % of each prefix re-decided); 10k planted pairs."""
    s = seed_for(6) if seed is None else seed
    V = max(64, int(round(1_000_000 * scale)))
    m = max(1, int(round(4_000_000 * scale)))
    K = max(1, int(round(10_000 * scale)))
    sizes = clause_sizes(m, "lognormal", 20.0, 1.0, 500, V, s)
    off = offsets_from_sizes(sizes)
    lits = clause_lits(off, V, s)
    codes = assign_trail(V, n_assign, 0.30, 0.70, s, group=group, flip_frac=0.1)
    pl = plant(off, lits, codes, K, s)
    return Instance(f"wide(scale={scale:g}, N={n_assign})", V, off, lits, codes, pl, params=dict(
        config=6, seed=s, scale=scale, sizes="lognormal(20,1)[2,500]", zipf=1.1,
        assign=f"trail groups of {group}, f~U[0.30,0.70], 10% flips"))


def batch_specs(n_inst: int = 64, seed: int | None = None, scale: float = 1.0) -> list[dict]:
    """Batching workload: per instance m log-uniform in [10k, 2M], V log-uniform in [5k, 500k],
    N = 128 * U{1..8}; geometric sizes as in the tiny workload, trail assignments, 100 planted.
    ``scale`` multiplies m and V (for test-sized batches)."""
    s = seed_for(3) if seed is None else seed
    rng = np.random.Generator(np.random.Philox(key=s))
    out = []
    for i in range(n_inst):
        m = int(round(math.exp(rng.uniform(math.log(10_000), math.log(2_000_000))) * scale))
        V = int(round(math.exp(rng.uniform(math.log(5_000), math.log(500_000))) * scale))
        N = 128 * int(rng.integers(1, 9))
        out.append(dict(index=i, n_clauses=max(1, m), n_vars=max(16, V), n_assign=N, seed=s * 131 + i,
                        n_planted=100))
    return out


def batch_instance(spec: dict) -> Instance:
    s = spec["seed"]
    V, m, N = spec["n_vars"], spec["n_clauses"], spec["n_assign"]
    sizes = clause_sizes(m, "geom", 1.0 / 7.0, 0.0, 30, V, s)
    off = offsets_from_sizes(sizes)
    lits = clause_lits(off, V, s)
    codes = assign_trail(V, N, 0.30, 0.70, s)
    pl = plant(off, lits, codes, spec["n_planted"], s)
    return Instance(f"batch[{spec['index']}]", V, off, lits, codes, pl, params=dict(config=3, **spec))


@dataclass
class ServeWorkload:
    """A growing clause database and the request snapshots that query it."""
    n_vars: int
    offsets: np.ndarray   # uint64 [m_final + 1]: the initial clauses then every batch, in arrival order
    lits: np.ndarray      # uint32
    n_initial: int        # clauses resident before the first request
    batch: int            # clauses per later batch
    n_batches: int
    params: dict = field(default_factory=dict)

    def batch_range(self, i: int) -> tuple[int, int]:
        """Clause ids [lo, hi) of batch i (batch -1 is the initial database)."""
        if i < 0:
            return 0, self.n_initial
        lo = self.n_initial + i * self.batch
        return lo, lo + self.batch

    def csr(self, lo: int, hi: int) -> tuple[np.ndarray, np.ndarray]:
        """Clauses [lo, hi) as a CSR of their own (offsets rebased to 0)."""
        b, e = int(self.offsets[lo]), int(self.offsets[hi])
        return (self.offsets[lo:hi + 1] - np.uint64(b)).astype(np.uint64), self.lits[b:e]


def serve_workload(scale: float = 1.0, seed: int | None = None, n_batches: int = 80) -> ServeWorkload:
    """Serving workload: 1M vars; 2M clauses resident at the start, then n_batches batches of
    50k (6M at the end); clause sizes 2 + Geom(1/7) redrawn above 30 (mean 8) as in the tiny
    workload, Zipf(1.1) vars, fair signs.  ``scale`` shrinks V and every clause count."""
    s = seed_for(4) if seed is None else seed
    V = max(64, int(round(1_000_000 * scale)))
    m0 = max(1, int(round(2_000_000 * scale)))
    b = max(1, int(round(50_000 * scale)))
    m = m0 + n_batches * b
    sizes = clause_sizes(m, "geom", 1.0 / 7.0, 0.0, 30, V, s)
    off = offsets_from_sizes(sizes)
    lits = clause_lits(off, V, s)
    return ServeWorkload(V, off, lits, m0, b, n_batches, dict(
        config=4, seed=s, scale=scale, sizes="geom(1/7)+2<=30", zipf=1.1, initial=m0, batch=b, n_batches=n_batches))


def serve_snapshots(n_vars: int, n: int, seed: int, lo: float = 0.40, hi: float = 0.60) -> np.ndarray:
    """n request snapshots, uint8 [n, 32, V]: snapshot i is one trail-prefix group of 32
    assignments (its own variable order and polarity, f ~ U[lo, hi) assigned, the last 2 % of
    each prefix re-decided), standing in for one solver thread's parent assignments."""
    return assign_trail(n_vars, 32 * n, lo, hi, seed).reshape(n, 32, n_vars)
