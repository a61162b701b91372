"""Benchmark: clause x assignment all-F tests on one GB300 (or N, one process each).

Workload (default): plain test, single instance -- 1M variables, 4M clauses with
lognormal sizes (median 20, sigma 1, clamped to [2, 500]) over Zipf(1.1) variables,
1024 trail-prefix-correlated assignments in 32 groups (30-70 % assigned), 10k planted
hits; seeded synthetic data.  One step = one GPU run of the method over a resident
clause database: pack the step's assignment set (codes already in HBM) into planes,
test every clause against every assignment, compact the hits into report records and
read back their count.  value = clauses x assignments tested per second (G/s).

e2e: the same step through the public API from pinned HOST memory: the codes go
host->device inside the timed region and the records come back device->host.  The
context keeps two plane sets, so step k + 1's codes cross the host link while step k's
test runs and its records travel back (gss_fetch_reports_async); the line also carries
the host link's copy rate, measured in the same run, and the fraction of the bound it
sets that e2e reaches.

--impl reference runs the oracle (plain C on the host cores) on a bounded sample of
the same workload, the reference arm of this comparison.

Other workloads: --config structured | tiny | batch | serve, and --config wide: the same
database against 8192 assignments (--n-assign, up to 32768) in trail groups of 1024,
tested with two aggregate levels and compared with the same set in 4096-assignment chunks.

Under torchrun each rank holds its own 4M-clause database (seed + rank) and tests the
same assignment set: per-GPU work is fixed (weak scaling); ranks never exchange data
except the timing barrier and the max-over-ranks reduction.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "clause×assignment tests/s (G/s) + HBM roofline fraction; served p50/p99 latency"
UNIT = "G tests/s"
WORKLOAD = ("plain test, single instance: 1M vars, 4M clauses, lognormal sizes (median 20, cap 500), "
            "Zipf(1.1) vars; 1024 assignments as 32 trail-prefix groups, 30-70% assigned; 10k planted hits")


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_sha(name: str) -> str:
    src = open(os.path.join(ROOT, "paper_2012_03119_gb300", "csrc", name), "rb").read()
    return hashlib.sha256(src).hexdigest()[:16]


def profiled_traffic(kernel_file: str, summary: str) -> float | None:
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current source."""
    p = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m_sha = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != kernel_source_sha(kernel_file):
        return None
    return float(m_b.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the benchmark runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 100):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        # raw samples: BENCH_CLOCKS_DIR if set (to keep them), else the system's temporary directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"gss_bench_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", str(self.interval_ms)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_instance(config: str, rank: int, scale: float, n_assign: int = 8192):
    import synth
    if config == "single":
        inst = synth.single(scale=scale, seed=synth.seed_for(2, rank))
        if rank:  # every rank tests the same assignment set against its own clauses
            inst.codes = synth.single(scale=scale, seed=synth.seed_for(2, 0)).codes
        return inst, WORKLOAD if scale == 1.0 else f"{WORKLOAD} (scaled x{scale:g})"
    if config == "structured":
        return synth.structured(scale=scale, seed=synth.seed_for(5, rank)), (
            "large structured: 10M vars in 1,000 communities, 10M clauses, lognormal sizes (median 40, cap 1000), "
            f"1024 trail assignments (scaled x{scale:g})")
    if config == "tiny":
        return synth.tiny(), "plain test, tiny: 2,000 vars, 20,000 clauses, 64 assignments"
    if config == "wide":
        inst = synth.wide(scale=scale, seed=synth.seed_for(6, rank), n_assign=n_assign)
        if rank:
            inst.codes = synth.wide(scale=scale, seed=synth.seed_for(6, 0), n_assign=n_assign).codes
        return inst, (f"wide set: 1M vars, 4M clauses (lognormal sizes median 20), {n_assign} trail assignments in "
                      f"groups of 1024; two aggregate levels" + ("" if scale == 1.0 else f" (scaled x{scale:g})"))
    raise SystemExit(f"unknown config {config}")


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest x over all ranks: a job's time is its slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput in G units/s: every rank processes units_per_rank per step (weak scaling)."""
    return units_per_rank * world * steps / seconds / 1e9


def algorithmic_bytes(inst, n_records: int) -> dict:
    """Bytes the method must move per launch.
    test: 4(m+1) + 4L + 2*V*W*4 + 12*R (offsets, every literal once, each plane row once, records);
    pack: N*V + 2*V*W*4 (codes in, planes out)."""
    m, L, V, N = inst.n_clauses, inst.n_lits, inst.n_vars, inst.n_assign
    W = (N + 31) // 32
    return {"test": 4 * (m + 1) + 4 * L + 2 * V * W * 4 + 12 * n_records, "pack": N * V + 2 * V * W * 4}


def narrow_split(gss, ctx, stream, d_codes, pitch, N, m, wide_pairs, steps):
    """The same N assignments as sets of at most 4096 (no level-2 filter), through the same
    context: the records must be the wide test's, and the time is what the wide path saves."""
    import torch
    n_max = gss.GSS_MAX_NARROW_ASSIGNMENTS
    chunks = [(a, min(N, a + n_max)) for a in range(0, N, n_max)]

    def run(collect):
        got = []
        for a, b in chunks:
            gss.gss_set_assignments_device(ctx.ptr, d_codes.data_ptr() + a * pitch, pitch, b - a)
            ctx.test()
            if collect:
                p = gss.expand_reports(ctx.fetch_reports())
                p[:, 1] += a
                got.append(p)
            else:
                ctx.report_count()
        return got

    got = np.concatenate(run(True))
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    same = bool(np.array_equal(got, wide_pairs))
    for _ in range(2):
        run(False)
    k = max(3, min(steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        run(False)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / k
    return {"chunks": len(chunks), "ms_per_step": t * 1e3, "tests_per_s_G": m * N / t / 1e9,
            "identical_pairs": same}


def cpu_baseline(inst, max_seconds: float = 15.0) -> dict:
    """The oracle, as it stands, on the host cores over a bounded sample of assignments."""
    import oracle
    threads = os.cpu_count() or 1
    n = 32
    t0 = time.perf_counter()
    oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, a_range=(0, n), threads=threads)
    dt = time.perf_counter() - t0
    n2 = int(min(inst.n_assign, max(n, n * max_seconds / max(dt, 1e-3) * 0.8)) // 32 * 32) or 32
    if n2 > n:
        t0 = time.perf_counter()
        oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, a_range=(0, n2), threads=threads)
        dt = time.perf_counter() - t0
        n = n2
    out = {"value": inst.n_clauses * n / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"all {inst.n_clauses} clauses x assignments [0, {n}) ({n / inst.n_assign:.3g} of the set), "
                     f"{dt:.2f} s wall on {threads} threads"}
    # the same oracle on one thread, over the first 32 assignments (a few seconds)
    n1 = min(32, inst.n_assign)
    t0 = time.perf_counter()
    oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, a_range=(0, n1), threads=1)
    dt1 = time.perf_counter() - t0
    out["single_thread"] = {"value": inst.n_clauses * n1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                            "sample": f"all {inst.n_clauses} clauses x assignments [0, {n1}), {dt1:.2f} s"}
    return out


def run_reference(args, inst, workload):
    """Reference arm: the oracle on the host cores, one bounded sample per step."""
    import oracle
    threads = os.cpu_count() or 1
    n = max(32, min(inst.n_assign, args.ref_assignments))
    if args.warmup > 0:
        oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, a_range=(0, 32), threads=threads)
    times = []
    for k in range(args.steps):
        lo = (k * n) % inst.n_assign
        hi = min(inst.n_assign, lo + n)
        t0 = time.perf_counter()
        oracle.allf_pairs(inst.offsets, inst.lits, inst.codes, a_range=(lo, hi), threads=threads)
        times.append((time.perf_counter() - t0, hi - lo))
    tot_t = sum(t for t, _ in times)
    tot_u = sum(inst.n_clauses * a for _, a in times)
    value = tot_u / tot_t / 1e9
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload, "sample_per_step": f"all clauses x {n} assignments"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"all {inst.n_clauses} clauses x {n} assignments per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


BATCH_WORKLOAD = ("batching: 64 uneven instances, 10k-2M clauses and 5k-500k vars each (log-uniform), geometric "
                  "sizes 2 + Geom(1/7) <= 30, 128-1024 trail assignments each; one graph per run")


def run_batch(args):
    """Batching workload: one graph (per-instance packing + one work-stealing test launch) against
    64 separate single-instance pack + test launches on the same GPU, same records."""
    import torch
    import paper_2012_03119_gb300 as gss
    import synth
    torch.cuda.set_device(0)
    specs = synth.batch_specs(64, scale=args.scale)
    insts = [synth.batch_instance(sp) for sp in specs]
    units = sum(I.n_clauses * I.n_assign for I in insts)
    stream = torch.cuda.Stream()
    d_codes = [torch.from_numpy(I.codes).cuda() for I in insts]
    caps = [I.n_clauses * ((I.n_assign + 31) // 32) // 4 + 65536 for I in insts]
    b = gss.Batch(stream=stream)
    for I, d, cap in zip(insts, d_codes, caps):
        i = b.add_instance(I.n_vars, I.offsets, I.lits, max_assignments=I.n_assign, report_capacity=cap)
        b.set_assignments(i, d)
    ctxs = []
    for I, cap in zip(insts, caps):
        c = gss.Context(I.n_vars, stream=stream, report_capacity=cap, max_assignments=I.n_assign)
        c.add_clauses(I.offsets, I.lits)
        ctxs.append(c)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.test()  # first run: capture + autotune
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    def separate():
        for I, c, d in zip(insts, ctxs, d_codes):
            gss.gss_set_assignments_device(c.ptr, d.data_ptr(), I.n_vars, I.n_assign)
            c.test()

    for _ in range(max(3, args.warmup)):
        b.test()
        separate()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    for _ in range(args.steps):
        b.test()
    ev[1].record(stream)
    for _ in range(args.steps):
        separate()
    ev[2].record(stream)
    torch.cuda.synchronize()
    t_batch = ev[0].elapsed_time(ev[1]) / 1e3 / args.steps
    t_sep = ev[1].elapsed_time(ev[2]) / 1e3 / args.steps
    same = True
    for i, c in enumerate(ctxs):  # identical records, batched and separate
        same &= bool(np.array_equal(gss.expand_reports(b.fetch_reports(i)), gss.expand_reports(c.fetch_reports())))
    info = b.info()
    out = {"metric": METRIC, "value": units / t_batch / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": BATCH_WORKLOAD + (f" (scaled x{args.scale:g})" if args.scale != 1.0 else ""),
                      "instances": len(insts), "clauses": int(sum(I.n_clauses for I in insts)),
                      "pair_tests_per_step": units, "codes_resident": True},
           "separate": {"value": units / t_sep / 1e9, "ms_per_step": t_sep * 1e3,
                        "launches_per_step": 2 * len(insts)},
           "speedup_vs_separate": t_sep / t_batch, "identical_records": same, "autotune": info,
           "first_run_s": setup_s, "gpu_launches": (len(insts) + 2) * args.steps}
    b.close()
    for c in ctxs:
        c.close()
    return out


SERVE_WORKLOAD = ("serving: 1M vars, resident DB grows 2M -> 6M clauses (80 batches of 50k, one per 50 ms), "
                  "geometric sizes 2 + Geom(1/7) <= 30, Zipf(1.1) vars; 32 simulated solver threads submit "
                  "32-assignment trail snapshots (40-60% assigned), Poisson arrivals 2k req/s in total")


def run_serve(args):
    """Serving workload: an open-loop phase (Poisson arrivals while the database grows) for
    latency and achieved tests/s, then a closed-loop phase on the final database comparing the
    server's saturated throughput with one pack + test launch per request through a context."""
    import threading
    import torch
    import paper_2012_03119_gb300 as gss
    import synth
    torch.cuda.set_device(0)
    w = synth.serve_workload(scale=args.scale)
    V, final = w.n_vars, len(w.offsets) - 1
    n_pool = 32  # distinct snapshots, cycled by the clients (pinned, as a solver's own buffers would be)
    pool_t = torch.empty((n_pool, 32, V), dtype=torch.uint8, pin_memory=True)
    pool = pool_t.numpy()
    pool[:] = synth.serve_snapshots(V, n_pool, seed=synth.seed_for(4, 1))
    cap = 1 << 23
    srv = gss.Server(V, max_clauses=final + 1, max_lits=int(w.offsets[-1]) + 1, slots=64, lanes=3,
                     lane_report_capacity=cap, tests_in_flight=args.serve_tests_in_flight)
    srv.add_clauses(*w.csr(0, w.n_initial))
    for i in range(max(3, args.warmup)):
        srv.wait(srv.submit(pool[i], wait_us=10_000_000))

    n_threads, rate = args.serve_threads, args.serve_rate
    period = 0.05
    lock = threading.Lock()
    done = []  # (watermark, n_assign, records, latency_us, batch_words, admit_us, queue_us, run_us)
    drops = [0]
    errors = []
    t_start = time.perf_counter() + 0.05
    t_end = t_start + w.n_batches * period

    def keep(r):
        rec, info = r
        with lock:
            done.append((info["watermark"], info["n_assign"], len(rec), info["latency_us"], info["batch_words"],
                         info["admit_us"], info["queue_us"], info["run_us"]))

    def client(t):
        try:
            rng = np.random.default_rng(1000 + t)
            nxt = t_start + rng.exponential(n_threads / rate)
            pending, j = [], 0
            while nxt < t_end:
                dt = nxt - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                rid = srv.submit(pool[(7 * t + j) % n_pool], wait_us=0)  # not sent when the GPU is full
                j += 1
                if rid is None:
                    with lock:
                        drops[0] += 1
                else:
                    pending.append(rid)
                still = []
                for q in pending:
                    r = srv.wait(q, wait_us=0)
                    if r is None:
                        still.append(q)
                    else:
                        keep(r)
                pending = still
                nxt += rng.exponential(n_threads / rate)
            for q in pending:
                keep(srv.wait(q))
        except Exception as e:
            errors.append(e)

    def ingest():
        try:
            for b in range(w.n_batches):
                dt = t_start + b * period - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                srv.add_clauses(*w.csr(*w.batch_range(b)))
        except Exception as e:
            errors.append(e)

    clocks = ClockSampler(0, args.serve_clock_ms)
    clocks.start()
    s0 = srv.stats()
    ths = [threading.Thread(target=ingest)] + [threading.Thread(target=client, args=(t,)) for t in range(n_threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    t_open = time.perf_counter() - t_start
    s1 = srv.stats()
    if errors:
        raise errors[0]
    lat = np.array([d[3] for d in done])
    parts = {k: np.array([d[i] for d in done]) for k, i in (("admit", 5), ("queue", 6), ("run", 7))}
    tests_open = sum(d[0] * d[1] for d in done)

    # closed loop on the final database: every client keeps one request in flight
    n_sat = args.serve_sat_requests
    sat_recs = {}

    def sat_client(t):
        try:
            for j in range(t, n_sat, n_threads):
                rec, info = srv.wait(srv.submit(pool[j % n_pool], wait_us=10_000_000))
                if j < n_pool:
                    with lock:
                        sat_recs[j] = rec
        except Exception as e:
            errors.append(e)

    s2 = srv.stats()
    t0 = time.perf_counter()
    ths = [threading.Thread(target=sat_client, args=(t,)) for t in range(n_threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    t_sat = time.perf_counter() - t0
    s3 = srv.stats()
    if errors:
        raise errors[0]
    srv.close()

    # one pack + test launch per request (host codes, as the server receives them)
    ctx = gss.Context(V, max_assignments=32, report_capacity=cap)
    ctx.add_clauses(w.offsets, w.lits)
    n_one = min(n_sat, 4 * n_pool)
    for j in range(3):
        ctx.set_assignments(pool[j])
        ctx.test()
        ctx.fetch_reports()
    torch.cuda.synchronize()
    one_recs = {}
    t0 = time.perf_counter()
    for j in range(n_one):
        ctx.set_assignments(pool[j % n_pool])
        ctx.test()
        rec = ctx.fetch_reports()
        if j in sat_recs:
            one_recs[j] = rec
    t_one = time.perf_counter() - t0
    same = len(one_recs) == len(sat_recs) > 0 and all(
        np.array_equal(gss.expand_reports(one_recs[j]), gss.expand_reports(sat_recs[j])) for j in sat_recs)
    ctx.close()
    clk = clocks.stop()

    sat_tests = float(final) * 32 * n_sat
    out = {"metric": METRIC, "value": tests_open / t_open / 1e9, "unit": UNIT, "n_gpus": 1,
           "steps": len(done), "warmup": max(3, args.warmup), "ms_per_step": t_open * 1e3 / max(1, len(done)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": SERVE_WORKLOAD + (f" (scaled x{args.scale:g})" if args.scale != 1.0 else ""),
                      "threads": n_threads, "rate_req_s": rate, "snapshot_pool": n_pool, "slots": s1["slots"],
                      "lanes": 3, "tests_in_flight": args.serve_tests_in_flight, "final_clauses": final},
           "open_loop": {"seconds": t_open, "requests": len(done), "dropped": drops[0],
                         "launches": s1["launches"] - s0["launches"],
                         "mean_batch_words": (s1["words_launched"] - s0["words_launched"]) /
                         max(1, s1["launches"] - s0["launches"]),
                         "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                        "max": float(lat.max()), "mean": float(lat.mean())},
                         "latency_parts_us": {k: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99))}
                                              for k, a in parts.items()},
                         "records": int(sum(d[2] for d in done)), "req_per_s": len(done) / t_open},
           "saturated": {"requests": n_sat, "seconds": t_sat, "req_per_s": n_sat / t_sat,
                         "G_tests_s": sat_tests / t_sat / 1e9,
                         "mean_batch_words": (s3["words_launched"] - s2["words_launched"]) /
                         max(1, s3["launches"] - s2["launches"])},
           "one_launch_per_request": {"requests": n_one, "req_per_s": n_one / t_one,
                                      "G_tests_s": float(final) * 32 * n_one / t_one / 1e9},
           "speedup_vs_one_launch_per_request": (n_sat / t_sat) / (n_one / t_one),
           "identical_records": same, "clocks": clk,
           "gpu_launches": 3 * (s3["launches"] - s0["launches"])}
    return out


def child_summary(argv: list[str], summarise) -> dict:
    """Run bench.py with argv in a child process and summarise its JSON line."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), *argv], capture_output=True, text=True, timeout=900)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"error": f"bench.py {' '.join(argv)} exited {r.returncode}: {r.stderr[-500:]}"}
    return summarise(json.loads(lines[-1]))


def batch_summary(b: dict) -> dict:
    """The batching line's figures that the default line carries."""
    return {"workload": b["config"]["workload"], "value": b["value"], "unit": b["unit"],
            "ms_per_step": b["ms_per_step"], "pair_tests_per_step": b["config"]["pair_tests_per_step"],
            "separate": b["separate"], "speedup_vs_separate": b["speedup_vs_separate"],
            "identical_records": b["identical_records"], "autotune": b["autotune"], "steps": b["steps"]}


def serve_summary(v: dict) -> dict:
    """The serving line's figures that the default line carries."""
    ol = v["open_loop"]
    return {"workload": v["config"]["workload"], "value": v["value"], "unit": v["unit"],
            "latency_us": ol["latency_us"], "latency_parts_us": ol["latency_parts_us"],
            "requests": ol["requests"], "dropped": ol["dropped"],
            "mean_batch_words": ol["mean_batch_words"], "saturated": v["saturated"],
            "one_launch_per_request": v["one_launch_per_request"],
            "speedup_vs_one_launch_per_request": v["speedup_vs_one_launch_per_request"],
            "identical_records": v["identical_records"], "clocks": v["clocks"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gss", choices=["gss", "reference"])
    ap.add_argument("--config", default="single", choices=["single", "structured", "tiny", "wide", "batch", "serve"])
    ap.add_argument("--n-assign", type=int, default=8192, help="assignments of the wide workload (<= 32768)")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--ref-assignments", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="single workload only: skip the batching and serving runs the default line carries")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="requests/s over all simulated solver threads")
    ap.add_argument("--serve-threads", type=int, default=32)
    ap.add_argument("--serve-sat-requests", type=int, default=1024)
    ap.add_argument("--serve-tests-in-flight", type=int, default=1)
    ap.add_argument("--serve-clock-ms", type=int, default=100,
                    help="nvidia-smi sampling interval during the serving run")
    ap.add_argument("--mode", default="allf", choices=["allf", "trigger"],
                    help="what a pair reports: all literals F (default) or Definition 'triggers'")
    ap.add_argument("--overlap", action="store_true",
                    help="run step k+1's packing beside step k's test (default: queued behind it)")
    ap.add_argument("--layout", default="frequency", choices=["frequency", "identity"],
                    help="internal variable numbering of the clause database")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.config == "batch" and args.impl != "reference":
        if rank == 0:
            print(json.dumps(run_batch(args)), flush=True)
        return
    if args.config == "serve" and args.impl != "reference":
        if rank == 0:
            print(json.dumps(run_serve(args)), flush=True)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        inst, workload = make_instance(args.config, 0, args.scale, args.n_assign)
        print(json.dumps(run_reference(args, inst, workload)), flush=True)
        return

    # the batching and serving workloads on the same GPU, so that one run records every form;
    # each in a process of its own and before this process opens its own CUDA context, as when
    # run alone (measured: a serving run in a process that had run the other workloads, or
    # beside an idle context of this one, showed p99 latencies of 3-35 ms against 1.1 ms alone)
    extras = None
    if world == 1 and args.config == "single" and args.scale == 1.0 and args.mode == "allf" and not args.no_extras:
        steps = str(min(args.steps, 20))
        extras = (child_summary(["--config", "batch", "--steps", steps, "--warmup", "3"], batch_summary),
                  child_summary(["--config", "serve"], serve_summary))

    import torch
    import paper_2012_03119_gb300 as gss

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    warmup = max(3, args.warmup)
    inst, workload = make_instance(args.config, rank, args.scale, args.n_assign)
    stream = torch.cuda.Stream()
    N, V, m = inst.n_assign, inst.n_vars, inst.n_clauses
    cap = max(1 << 22, 8 * len(inst.planted) + (16 if args.mode == "trigger" else 4) * m * ((N + 1023) // 1024))
    layout = gss.GSS_LAYOUT_FREQUENCY if args.layout == "frequency" else gss.GSS_LAYOUT_IDENTITY
    mode = gss.GSS_MODE_TRIGGER if args.mode == "trigger" else gss.GSS_MODE_ALLF
    # two plane sets: the next set can be copied and packed while the last one is tested
    pack_stream = torch.cuda.Stream()
    ctx = gss.Context(V, device=local, stream=stream, report_capacity=cap, max_assignments=max(N, 32), layout=layout,
                      mode=mode, pipeline=2, pack_stream=pack_stream)

    # a-1: ingest the database (once; the database stays resident like the paper's GPU clause store)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.add_clauses(inst.offsets, inst.lits)
    torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t0

    d_codes = torch.from_numpy(inst.codes).to(f"cuda:{local}")
    torch.cuda.synchronize()
    pitch = V

    def step():
        gss.gss_set_assignments_device(ctx.ptr, d_codes.data_ptr(), pitch, N)
        ctx.test()

    # correctness guard outside timing: every planted pair is reported
    step()
    rec = ctx.fetch_reports()
    pairs = gss.expand_reports(rec)
    key = set((pairs[:, 0].astype(np.int64) << 32 | pairs[:, 1]).tolist())
    planted_ok = all(((int(c) << 32) | int(a)) in key for c, a in inst.planted.tolist())
    n_records = len(rec)
    st = gss.gss_get_stats(ctx.ptr)  # the aggregate test's selectivity (Section 4.2) on this workload
    aggregate = {"candidate_pairs": st["candidate_pairs"], "group_pairs": st["group_pairs"],
                 "negative_ratio": 1.0 - st["candidate_pairs"] / max(1, st["group_pairs"]),
                 "paper_negative_ratio": 0.999422}
    if N > gss.GSS_MAX_NARROW_ASSIGNMENTS:  # the level-2 (1024-assignment) filter in front of it
        sg = m * ((N + 1023) // 1024)
        aggregate.update({"super_pairs": st["super_pairs"], "super_group_pairs": sg,
                          "super_negative_ratio": 1.0 - st["super_pairs"] / max(1, sg)})

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for _ in range(warmup):
        step()
        ctx.report_count()

    def timed_steps(n_steps: int):
        """n_steps steps: pack step k's set, test it, read its record count back to the host.
        Packing and testing take turns (each kernel fills the GPU; running them side by side
        measured slower): step k + 1's packing (into the other plane set) is queued on the pack
        stream behind step k's test before the host waits for step k's count, so the GPU does
        not sit idle while the count travels to the host and the next launch is made.  With
        --overlap, step k + 1's packing does not wait for step k's test and runs beside it.
        Each kernel is bracketed by CUDA events on the stream it runs on (after its wait for
        the other stream)."""
        evp = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_steps)]
        evt = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_steps)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def pack(k):
            evp[k][0].record(pack_stream)
            gss.gss_set_assignments_device(ctx.ptr, d_codes.data_ptr(), pitch, N)
            evp[k][1].record(pack_stream)

        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(stream)
        pack_stream.wait_event(start)
        pack(0)
        for k in range(n_steps):
            stream.wait_event(evp[k][1])
            evt[k][0].record(stream)
            ctx.test()
            evt[k][1].record(stream)
            if k + 1 < n_steps:
                if not args.overlap:
                    pack_stream.wait_event(evt[k][1])  # in turn with step k's test
                pack(k + 1)
            ctx.report_count()  # step k's result (record count) read back to the host
        end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        el = start.elapsed_time(end) / 1e3
        tp = float(np.mean([e[0].elapsed_time(e[1]) for e in evp])) / 1e3
        tt = float(np.mean([e[0].elapsed_time(e[1]) for e in evt])) / 1e3
        return el, tp, tt

    elapsed, t_pack, t_test = timed_steps(args.steps)
    elapsed = max_over_ranks(elapsed, dist)

    split = None
    if N > gss.GSS_MAX_NARROW_ASSIGNMENTS:
        split = narrow_split(gss, ctx, stream, d_codes, pitch, N, m, pairs, args.steps)

    # e2e through the public API from pinned host memory
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 20))
    h_codes = torch.empty((N, V), dtype=torch.uint8).pin_memory()
    h_codes.numpy()[:] = inst.codes
    h_rec = torch.empty((cap * 12,), dtype=torch.uint8).pin_memory().numpy().view(gss.REPORT_DTYPE)
    for _ in range(2):
        ctx.set_assignments(h_codes.numpy())
        ctx.test()
        ctx.fetch_reports(h_rec)
    def host_link_seconds(reps: int = 3) -> list[float]:
        """One step's codes, pinned host -> device, as one copy: the host link's rate, measured
        just before and just after the e2e loop (the best of both bounds e2e)."""
        out = []
        for _ in range(reps):
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                l0.record(stream)
                d_codes.copy_(h_codes, non_blocking=True)
                l1.record(stream)
            l1.synchronize()
            out.append(l0.elapsed_time(l1) / 1e3)
        return out

    link_s = host_link_seconds()
    def e2e_loop() -> float:
        """e2e_steps steps through the API; their wall time (max over ranks)."""
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # every step copies its codes in and its records out; with two plane sets the codes of
        # step k + 1 cross the host link (queued behind step k's copy) while step k is packed
        # and tested and its records travel back
        ctx.set_assignments_async(h_codes.numpy())
        for k in range(e2e_steps):
            ctx.test()
            ctx.fetch_reports_async(h_rec)
            if k + 1 < e2e_steps:
                ctx.set_assignments_async(h_codes.numpy())
            ctx.fetch_wait()
        ctx.copy_wait()
        return max_over_ranks(time.perf_counter() - t0, dist)

    # the host is shared with other jobs: the loop runs three times and the median counts
    e2e_samples = [e2e_loop() for _ in range(3)]
    e2e_s = float(np.median(e2e_samples))
    link_s += host_link_seconds()
    link_gbs = N * V / min(link_s) / 1e9
    clk = clocks.stop()

    value = whole_job_rate(m * N, world, args.steps, elapsed)
    pk = peaks()
    B = algorithmic_bytes(inst, n_records)
    # ncu summaries taken on this exact workload (traffic is null for any other)
    summary = None
    if args.scale == 1.0 and args.mode == "allf" and args.layout == "frequency":
        if args.config == "single":
            summary = {"pack": "k_pack__single_V1M_N1024.md", "test": "k_test__single_V1M_N1024.md"}
        elif args.config == "wide" and N == 8192:
            summary = {"pack": "k_pack__wide_V1M_N8192.md", "test": "k_test__wide_V1M_N8192.md"}
        elif args.config == "structured":
            summary = {"pack": "k_pack__structured_V10M_N1024.md", "test": "k_test__structured_V10M_N1024.md"}
    roof = {
        "pack": {"bound": "hbm", "achieved": B["pack"] / t_pack / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": B["pack"] / t_pack / 1e9 / pk["hbm_gbs"], "time_us": t_pack * 1e6, "bytes": B["pack"],
                 "traffic": profiled_traffic("k_pack.cu", summary["pack"]) if summary else None,
                 "kernel": "k_pack",
                 "peak_source": f"{pk['source']} hbm_gbs"},
        "test": {"bound": "hbm", "achieved": B["test"] / t_test / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": B["test"] / t_test / 1e9 / pk["hbm_gbs"], "time_us": t_test * 1e6, "bytes": B["test"],
                 "traffic": profiled_traffic("k_test.cu", summary["test"]) if summary else None,
                 "kernel": "k_test",
                 "peak_source": f"{pk['source']} hbm_gbs"},
    }
    for k, t in (("pack", t_pack), ("test", t_test)):
        # the fraction on the bytes DRAM really moved (ncu), beside the one on algorithmic bytes:
        # an early-exit test reads far fewer literals than the algorithmic count assumes
        tr = roof[k]["traffic"]
        roof[k]["frac_traffic"] = tr / t / 1e9 / pk["hbm_gbs"] if tr else None
    dominant = "pack" if t_pack >= t_test else "test"
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload, "n_vars": V, "n_clauses": m, "n_lits": inst.n_lits, "n_assign": N,
                   "seed": inst.params.get("seed"),
                   "l2": f"inputs larger than L2 ({N * V / 1e9:.3g} GB codes + {8 * V * ((N + 31) // 32) / 1e9:.3g} GB "
                         "planes streamed per step)" if N * V > 129e6 else "inputs smaller than L2",
                   "parallelism": f"weak x{world}: one clause database per GPU, shared assignment set",
                   "layout": args.layout, "mode": args.mode},
        "e2e": {"value": whole_job_rate(m * N, world, e2e_steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": N * V,
                "d2h_bytes_per_step": 12 * n_records + 48,
                # the bound the host link sets: one step's codes at the measured copy rate
                "host_link_GBps": link_gbs, "link_cap_value": m * N * world / (N * V / (link_gbs * 1e9)) / 1e9,
                "frac_of_link_cap": whole_job_rate(m * N, world, e2e_steps, e2e_s) /
                (m * N * world / (N * V / (link_gbs * 1e9)) / 1e9),
                "samples": [whole_job_rate(m * N, world, e2e_steps, t) for t in e2e_samples],
                "steps_per_sample": e2e_steps},
        "roofline": {k: v for k, v in roof[dominant].items()},
        "roofline_all": roof,
        "kernel_only": {"test_tests_per_s_G": m * N / t_test / 1e9, "pack_us": t_pack * 1e6,
                        "test_us": t_test * 1e6},
        "ingest": {"seconds": ingest_s, "clauses": m, "lits": inst.n_lits,
                   "GB_per_s": (8 * (m + 1) + 4 * inst.n_lits) / ingest_s / 1e9},
        "gpu_launches": (3 if N > gss.GSS_MAX_NARROW_ASSIGNMENTS else 2) * args.steps,  # pack (+ level 2) + test
        "records": n_records, "pairs": int(len(pairs)), "planted_found": planted_ok,
        "aggregate_test": aggregate,
        "clocks": clk,
    }
    if split:
        out["narrow_split"] = split
    ctx.close()
    del d_codes, h_codes
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(inst)
    if extras:
        out["batch"], out["serve"] = extras
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
