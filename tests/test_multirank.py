"""The N > 1 path of bench.py, on CPU: two gloo ranks, each with its own clause database and
the shared assignment set, timing reduced with a max over ranks (weak scaling, no data
exchange).  Runs without a GPU."""
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
