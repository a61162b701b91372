"""The N > 1 paths on CPU, with gloo ranks and no GPU:
- bench.py's weak scaling: two ranks, each with its own clause database and the shared
  assignment set, timing reduced with a max over ranks (no data exchange);
- one database split over ranks by clause ranges (paper_2012_03119_gb300.shard): global ids and
  the gathered records equal the single-rank result."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst, workload = bench.make_instance("single", rank, scale=0.001)
    fake_elapsed = 1.0 + 0.5 * rank  # rank 1 is the slowest
    elapsed = bench.max_over_ranks(fake_elapsed, dist, device="cpu")
    value = bench.whole_job_rate(inst.n_clauses * inst.n_assign, world, 10, elapsed)
    out = {"rank": rank, "elapsed": elapsed, "value": value, "db": synth.content_hash(inst.offsets, inst.lits),
           "codes": synth.content_hash(inst.codes), "m": inst.n_clauses, "N": inst.n_assign,
           "seed": inst.params["seed"], "workload": workload}
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(out, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # every rank sees the slowest rank's time, and reports the whole job's units
    assert res[0]["elapsed"] == res[1]["elapsed"] == 1.5
    units = res[0]["m"] * res[0]["N"] * world * 10
    assert np.isclose(res[0]["value"], units / 1.5 / 1e9) and res[0]["value"] == res[1]["value"]
    # weak scaling: each rank its own database, the same assignment set
    assert res[0]["db"] != res[1]["db"] and res[0]["seed"] != res[1]["seed"]
    assert res[0]["codes"] == res[1]["codes"]
    assert res[0]["m"] == res[1]["m"] and res[0]["N"] == res[1]["N"]


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None) == 2.5
    assert bench.whole_job_rate(10**9, 4, 2, 8.0) == 1.0


def _pairs_to_records(pairs):
    """(clause, assignment) pairs -> records {clause, word, mask}, one per (clause, word)."""
    import paper_2012_03119_gb300 as gss
    p = np.asarray(pairs, np.uint64).reshape(-1, 2)
    key = (p[:, 0] << np.uint64(32)) | (p[:, 1] // np.uint64(32))
    uk, inv = np.unique(key, return_inverse=True)
    mask = np.zeros(len(uk), np.uint32)
    np.bitwise_or.at(mask, inv, (np.uint32(1) << (p[:, 1] % 32).astype(np.uint32)))
    rec = np.empty(len(uk), gss.REPORT_DTYPE)
    rec["clause_id"] = (uk >> np.uint64(32)).astype(np.uint32)
    rec["word"] = (uk & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    rec["mask"] = mask
    return rec


def _shard_rank_main(rank: int, world: int, port: int, out_dir: str):
    """One rank of a split database: its clause range, its local test (the oracle stands in for
    the GPU here, in the test only), global ids, and the gather on rank 0."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import oracle
    import synth
    from paper_2012_03119_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = synth.single(scale=0.002)  # 2k vars, 8k clauses, 1024 assignments
    ranges = shard.clause_ranges(inst.offsets, world)
    lo, hi = ranges[rank]
    off, lits = shard.local_csr(inst.offsets, inst.lits, lo, hi)
    local = _pairs_to_records(oracle.allf_pairs(off, lits, inst.codes))
    got = shard.gather_records(shard.globalize(local, lo), dist)
    if rank == 0:
        import paper_2012_03119_gb300 as gss
        pairs = gss.expand_reports(got)
        np.save(os.path.join(out_dir, "gathered.npy"), pairs)
        with open(os.path.join(out_dir, "ranges.json"), "w") as f:
            json.dump(ranges, f)
    else:
        assert got is None
    dist.barrier()
    dist.destroy_process_group()


def test_split_database_gathers_the_single_rank_result(tmp_path):
    """Two gloo ranks split one database by literal-balanced clause ranges; the gathered
    records, with global ids, equal the whole database's oracle result."""
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_shard_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    inst = synth.single(scale=0.002)
    want = oracle.allf_pairs(inst.offsets, inst.lits, inst.codes)
    got = np.load(tmp_path / "gathered.npy")
    assert len(want) > 0 and np.array_equal(got, want)
    ranges = json.load(open(tmp_path / "ranges.json"))
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == inst.n_clauses


def test_clause_ranges_balance_literals():
    sys.path.insert(0, ROOT)
    from paper_2012_03119_gb300 import shard
    rng = np.random.default_rng(3)
    sizes = rng.integers(1, 60, size=5000)
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(sizes)
    for world in (1, 2, 3, 7, 8):
        r = shard.clause_ranges(off, world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == len(sizes)
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
        share = [int(off[h]) - int(off[l]) for l, h in r]
        assert max(share) - min(share) <= 2 * sizes.max()  # each cut is within one clause of its target
    # fewer clauses than ranks: some ranges are empty, all clauses are covered once
    r = shard.clause_ranges(off[:4], 8)
    assert sum(h - l for l, h in r) == 3
    # local CSR and global ids
    lo, hi = 10, 20
    o, lits = shard.local_csr(off, np.arange(int(off[-1]), dtype=np.uint32), lo, hi)
    assert o[0] == 0 and len(o) == 11 and lits[0] == off[lo] and len(lits) == int(off[hi] - off[lo])
    import paper_2012_03119_gb300 as gss
    rec = np.zeros(3, gss.REPORT_DTYPE)
    rec["clause_id"] = [0, 1, 9]
    assert list(shard.globalize(rec, lo)["clause_id"]) == [10, 11, 19]
    assert list(rec["clause_id"]) == [0, 1, 9]
