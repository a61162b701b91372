"""Serving (gss_server_*): continuous batching of 32-assignment requests against a growing
resident database.  Every request must equal the oracle on the database prefix given by its
watermark, and the same request must give the same records alone and in a mix of concurrent
requests while clauses stream in."""
import threading
from concurrent.futures import ThreadPoolExecutor
import time

import numpy as np
import pytest

import oracle
import synth
import paper_2012_03119_gb300 as gss

pytestmark = pytest.mark.gpu


def submit_together(srv, codes_list):
    """Submit every request at the same moment, one thread each: requests that arrive while a
    launch runs join the next one.  Returns the request ids in order."""
    bar = threading.Barrier(len(codes_list))

    def submit(c):
        bar.wait()
        return srv.submit(c, wait_us=10_000_000)

    with ThreadPoolExecutor(len(codes_list)) as ex:
        return list(ex.map(submit, codes_list))


@pytest.fixture(scope="module")
def work():
    # 10k vars, 20k clauses at the start, then 20 batches of 500 (30k at the end)
    return synth.serve_workload(scale=0.01, seed=0x5E17E, n_batches=20)


@pytest.fixture(scope="module")
def snaps(work):
    return synth.serve_snapshots(work.n_vars, 24, seed=0x5A9)


def make_server(work, **kw):
    args = dict(max_clauses=len(work.offsets) + 1024, max_lits=int(work.offsets[-1]) + 65536, slots=16, lanes=2,
                lane_report_capacity=1 << 20)
    args.update(kw)
    return gss.Server(work.n_vars, **args)


def prefix_oracle(work, wm, codes, mode=oracle.MODE_ALLF):
    off = work.offsets[: wm + 1]
    return oracle.pairs(off, work.lits[: int(off[-1])], codes, mode)


def run_alone(srv, codes, wm=None):
    rid = srv.submit(codes, watermark=wm, wait_us=10_000_000)
    rec, info = srv.wait(rid)
    return gss.expand_reports(rec), info


def test_serve_alone_mixed_and_oracle(work, snaps):
    srv = make_server(work, lanes=2)
    with srv:
        srv.add_clauses(*work.csr(0, work.n_initial))
        probes = [(i, work.n_initial - 3000 * i) for i in range(4)]
        alone = {}
        for i, wm in probes:
            pairs, info = run_alone(srv, snaps[i], wm)
            assert info["watermark"] == wm and info["batch_words"] == 1
            np.testing.assert_array_equal(pairs, prefix_oracle(work, wm, snaps[i]))
            assert len(pairs) > 0
            alone[i] = pairs

        results, errors = [], []
        lock = threading.Lock()

        def ingest():
            try:
                for b in range(work.n_batches):
                    srv.add_clauses(*work.csr(*work.batch_range(b)))
                    time.sleep(0.002)
            except Exception as e:  # reported by the main thread
                errors.append(e)

        def client(t):
            try:
                ids = []
                for j in range(5):
                    k = (t * 5 + j) % len(snaps)
                    rid = srv.submit(snaps[k], wait_us=10_000_000)
                    ids.append((k, rid))
                for k, rid in ids:
                    rec, info = srv.wait(rid)
                    with lock:
                        results.append((k, rec, info))
            except Exception as e:
                errors.append(e)

        threads = [threading.Thread(target=ingest)] + [threading.Thread(target=client, args=(t,)) for t in range(8)]
        for th in threads:
            th.start()
        mixed = {}
        for i, wm in probes:  # the same probes again, inside the mix
            mixed[i], info = run_alone(srv, snaps[i], wm)
            assert info["watermark"] == wm
        for th in threads:
            th.join()
        assert not errors, errors
        st = srv.stats()
        # continuous batching: requests that arrive while a launch runs join the next one.  The
        # mix above usually shows it; if its timing did not, bursts of back-to-back submissions do
        final = len(work.offsets) - 1
        for attempt in range(20):
            if st["launches"] < st["words_launched"]:
                break
            ids = list(enumerate(submit_together(srv, snaps[:8])))
            for k, rid in ids:
                rec, info = srv.wait(rid)
                np.testing.assert_array_equal(gss.expand_reports(rec), prefix_oracle(work, info["watermark"], snaps[k]))
            st = srv.stats()

    for i, _ in probes:
        np.testing.assert_array_equal(mixed[i], alone[i])
    assert len(results) == 40
    final = len(work.offsets) - 1
    for k, rec, info in results:
        wm = info["watermark"]
        assert work.n_initial <= wm <= final
        assert (rec["word"] == 0).all()
        np.testing.assert_array_equal(gss.expand_reports(rec), prefix_oracle(work, wm, snaps[k]))
    assert st["committed_clauses"] == final
    assert st["completed"] == st["submitted"] == st["words_launched"] and st["submitted"] % 8 == 0
    assert st["submitted"] >= 48 and st["dropped"] == 0
    assert st["launches"] < st["words_launched"], "no launch carried more than one request"
    assert st["p99_us"] >= st["p50_us"] > 0


def test_serve_partial_requests_trigger(work, snaps):
    """Requests with fewer than 32 assignments: the U rows that pad the plane word must not
    report, even where a unit clause triggers on an all-U assignment (Definition "triggers")."""
    off0, lits0 = work.csr(0, work.n_initial)
    rng = np.random.default_rng(7)
    units = rng.integers(0, 2 * work.n_vars, size=300).astype(np.uint32)
    off = np.concatenate([off0, off0[-1] + np.arange(1, len(units) + 1, dtype=np.uint64)])
    lits = np.concatenate([lits0, units])
    for mode, ofn in ((gss.GSS_MODE_TRIGGER, oracle.trigger_pairs), (gss.GSS_MODE_ALLF, oracle.allf_pairs)):
        with make_server(work, mode=mode) as srv:
            srv.add_clauses(off, lits)
            for n in (1, 5, 31, 32):
                codes = np.ascontiguousarray(snaps[n % len(snaps), :n])
                pairs, info = run_alone(srv, codes)
                assert info["n_assign"] == n
                np.testing.assert_array_equal(pairs, ofn(off, lits, codes))
                if mode == gss.GSS_MODE_TRIGGER:
                    assert len(pairs) > 0


def test_serve_admission_busy(work, snaps):
    """One slot, four submitters that do not wait: some submissions are refused
    (GSS_E_BUSY, the request is not sent), every admitted one completes, none is lost."""
    with make_server(work, slots=1, lanes=1) as srv:
        assert srv.stats()["slots"] == 1
        srv.add_clauses(*work.csr(0, work.n_initial))
        admitted = []

        def client(t):
            for j in range(30):
                rid = srv.submit(snaps[(t + j) % len(snaps)], wait_us=0, keep=False)
                admitted.append(rid is not None)

        threads = [threading.Thread(target=client, args=(t,)) for t in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        deadline = time.time() + 30
        while True:
            st = srv.stats()
            if st["completed"] + st["dropped"] == st["submitted"] or time.time() > deadline:
                break
            time.sleep(0.01)
        assert st["submitted"] == 120
        assert st["dropped"] == admitted.count(False) > 0
        assert st["completed"] == admitted.count(True) > 0
        # a submitter that waits for a slot is always admitted
        pairs, _ = run_alone(srv, snaps[0])
        np.testing.assert_array_equal(pairs, prefix_oracle(work, work.n_initial, snaps[0]))


def test_serve_slot_memory_budget(work):
    slot = 32 * ((work.n_vars + 15) // 16 * 16)
    with make_server(work, slots=64, slot_memory_bytes=3 * slot + 17) as srv:
        assert srv.stats()["slots"] == 3
    with pytest.raises(gss.GssError) as ei:
        make_server(work, slot_memory_bytes=slot - 1)
    assert ei.value.code == gss.GSS_E_NOMEM


def test_serve_errors(work, snaps):
    with make_server(work, max_clauses=1000, max_lits=100_000) as srv:
        off, lits = work.csr(0, 900)
        srv.add_clauses(off, lits)
        with pytest.raises(gss.GssError) as ei:  # past the reserved capacity
            srv.add_clauses(*work.csr(900, 1200))
        assert ei.value.code == gss.GSS_E_NOMEM
        assert srv.stats()["committed_clauses"] == 900
        with pytest.raises(ValueError):
            srv.submit(np.zeros((2, work.n_vars + 1), np.uint8))
        with pytest.raises(gss.GssError) as ei:
            srv.submit(np.zeros((33, work.n_vars), np.uint8))
        assert ei.value.code == gss.GSS_E_INVAL
        # an invalid code spoils its own request only
        bad = snaps[1].copy()
        bad[3, 17] = 3
        rb = srv.submit(bad, wait_us=10_000_000)
        rg = srv.submit(snaps[2], wait_us=10_000_000)
        with pytest.raises(gss.GssError) as ei:
            srv.wait(rb)
        assert ei.value.code == gss.GSS_E_INVAL
        rec, info = srv.wait(rg)
        np.testing.assert_array_equal(gss.expand_reports(rec), prefix_oracle(work, 900, snaps[2]))
        with pytest.raises(gss.GssError):  # already taken
            srv.wait(rg)
        # all-U request: nothing is all-F
        rec, info = srv.wait(srv.submit(np.zeros((32, work.n_vars), np.uint8), wait_us=10_000_000))
        assert len(rec) == 0 and info["watermark"] == 900


def test_serve_empty_database(work, snaps):
    with make_server(work) as srv:
        rec, info = srv.wait(srv.submit(snaps[0], wait_us=10_000_000))
        assert len(rec) == 0 and info["watermark"] == 0
        srv.add_clauses(*work.csr(0, 5000))
        pairs, info = run_alone(srv, snaps[0])
        assert info["watermark"] == 5000
        np.testing.assert_array_equal(pairs, prefix_oracle(work, 5000, snaps[0]))


def test_serve_identity_layout(work, snaps):
    with make_server(work, layout=gss.GSS_LAYOUT_IDENTITY) as srv:
        srv.add_clauses(*work.csr(0, work.n_initial))
        pairs, _ = run_alone(srv, snaps[3])
        np.testing.assert_array_equal(pairs, prefix_oracle(work, work.n_initial, snaps[3]))


def test_serve_result_deadline(work, snaps):
    """A client that never collects its kept results (a solver thread that died): they are
    dropped after result_ttl_us and counted; a waiting client is never cut off."""
    with make_server(work, result_ttl_us=200_000) as srv:
        srv.add_clauses(*work.csr(0, work.n_initial))
        lost = srv.submit(snaps[0], wait_us=10_000_000)
        rec, _ = srv.wait(srv.submit(snaps[1], wait_us=10_000_000))  # taken in time
        deadline = time.time() + 10
        while srv.stats()["expired"] == 0 and time.time() < deadline:
            time.sleep(0.05)
        assert srv.stats()["expired"] == 1
        with pytest.raises(gss.GssError) as ei:
            srv.wait(lost)
        assert ei.value.code == gss.GSS_E_INVAL
        # a result taken within the deadline is unaffected
        rec, info = srv.wait(srv.submit(snaps[2], wait_us=10_000_000), wait_us=5_000_000)
        np.testing.assert_array_equal(gss.expand_reports(rec), prefix_oracle(work, work.n_initial, snaps[2]))


def test_serve_padding_never_counts_against_capacity(work):
    """Trigger mode, unit clauses, requests of fewer than 32 assignments launched together: the
    U rows that pad each request's plane word would make every unit clause trigger.  Their
    records must never be made, so a launch capacity that only those records would exceed does
    not fail any request, and each result equals the oracle alone and in the mix."""
    V = work.n_vars
    n_units = 256
    rng = np.random.default_rng(11)
    vs = rng.choice(V, size=n_units, replace=False)
    lits = (2 * vs + rng.integers(0, 2, size=n_units)).astype(np.uint32)
    off = np.arange(n_units + 1, dtype=np.uint64)
    # every real assignment makes every unit literal T, except literal i in request i: one real record each
    base = np.zeros(V, np.uint8)
    base[vs] = np.where(lits & 1, 2, 1)  # v = T for literal v, v = F for literal not v
    reqs = []
    for i, n in enumerate((1, 3, 7, 12, 20, 31, 2, 5)):
        codes = np.tile(base, (n, 1))
        codes[n - 1, vs[i]] = 0  # literal i becomes U in the last row: the unit clause triggers there
        reqs.append(codes)
    want = [oracle.trigger_pairs(off, lits, c) for c in reqs]
    assert all(len(w) == 1 for w in want)
    with make_server(work, mode=gss.GSS_MODE_TRIGGER, lanes=1, lane_report_capacity=16) as srv:
        srv.add_clauses(off, lits)
        alone = [run_alone(srv, c)[0] for c in reqs]
        batched = False
        for attempt in range(20):  # submitted at once from several threads: they join launches together
            ids = submit_together(srv, reqs)
            mixed = [srv.wait(rid) for rid in ids]
            for (rec, info), w in zip(mixed, want):
                np.testing.assert_array_equal(gss.expand_reports(rec), w)
            batched |= max(info["batch_words"] for _, info in mixed) > 1
            if batched:
                break
        st = srv.stats()
    for a, w in zip(alone, want):
        np.testing.assert_array_equal(a, w)
    assert st["completed"] == st["submitted"] and st["reports"] == st["completed"]
    assert batched, "no launch carried more than one request"


@pytest.mark.parametrize("mode", [gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER])
def test_serve_activity_and_reduce(work, snaps, mode):
    """Section 3.6 on the server's resident database: each launch bumps the clauses it reports,
    and a reduction removes the lowest-activity long clauses between launches.  Requests before
    and after the reduction, and after more clauses arrive, equal the activity oracle's pairs
    on its database; activities and ids match bit for bit; a watermark below the newest ids
    keeps out the clauses added after it."""
    from oracle.activity import ActivityOracle
    ao = ActivityOracle(0.8)
    ofn = oracle.trigger_pairs if mode == gss.GSS_MODE_TRIGGER else oracle.allf_pairs
    with make_server(work, mode=mode, lanes=2, tests_in_flight=1) as srv:
        srv.set_activity(0.8)
        off0, lits0 = work.csr(0, work.n_initial)
        assert srv.add_clauses(off0, lits0) == ao.add(off0, lits0) == 0

        def request(k, watermark=None):
            rec, info = srv.wait(srv.submit(snaps[k], watermark=watermark, wait_us=10_000_000))
            got = gss.expand_reports(rec)
            want = ao.pairs(snaps[k], mode)
            if watermark is not None:
                want = want[want[:, 0] < watermark]
            np.testing.assert_array_equal(got, want)
            ao.after_test(want[:, 0])  # one launch per request: one test for the bumps
            return info

        for k in range(4):
            request(k)
        n = srv.reduce(0.5)
        assert n == ao.reduce(0.5) > 0
        np.testing.assert_array_equal(srv.clause_ids(), ao.ids)
        np.testing.assert_array_equal(srv.activity().view(np.uint32), ao.act.view(np.uint32))
        for k in range(4, 7):
            request(k)
        off1, lits1 = work.csr(*work.batch_range(0))  # new clauses take new ids, never reused ones
        first = srv.add_clauses(off1, lits1)
        assert first == ao.add(off1, lits1) == work.n_initial
        for k in range(7, 10):
            request(k)
        info = request(10, watermark=first)  # only the clauses committed before the new batch
        assert info["watermark"] == first
        np.testing.assert_array_equal(srv.clause_ids(), ao.ids)
        np.testing.assert_array_equal(srv.activity().view(np.uint32), ao.act.view(np.uint32))
        st = srv.stats()
        assert st["reductions"] == 1 and st["clauses_removed"] == n
        assert st["committed_clauses"] == ao.n_clauses and st["next_clause_id"] == ao.next_id


def test_serve_reduce_while_requests_run(work, snaps):
    """A reduction issued while clients submit: it waits for running launches, holds new ones,
    and every request's records equal the oracle on the database before or after it."""
    from oracle.activity import ActivityOracle
    ao = ActivityOracle(1.0)
    with make_server(work, lanes=3, tests_in_flight=1) as srv:
        srv.set_activity(1.0)
        off0, lits0 = work.csr(0, work.n_initial)
        srv.add_clauses(off0, lits0)
        ao.add(off0, lits0)
        before = [ao.pairs(s) for s in snaps[:8]]
        results, errors = [], []

        def client():
            try:
                ids = [(k, srv.submit(snaps[k], wait_us=10_000_000)) for k in range(8) for _ in range(3)]
                results.extend((k, srv.wait(rid)[0]) for k, rid in ids)
            except Exception as e:  # reported below
                errors.append(e)

        th = threading.Thread(target=client)
        th.start()
        time.sleep(0.001)
        removed = srv.reduce(0.3)
        th.join()
        assert not errors, errors
        assert removed > 0
        kept = set(srv.clause_ids().tolist())
        for k, rec in results:
            got = gss.expand_reports(rec)
            after = before[k][np.isin(before[k][:, 0], np.array(sorted(kept), np.uint32))]
            assert np.array_equal(got, before[k]) or np.array_equal(got, after)
        assert srv.stats()["completed"] == 24


def test_serve_activity_needs_one_test_in_flight(work):
    with make_server(work, lanes=2, tests_in_flight=2) as srv:
        with pytest.raises(gss.GssError) as ei:
            srv.set_activity(0.9)
        assert ei.value.code == gss.GSS_E_STATE
        with pytest.raises(gss.GssError) as ei:
            srv.reduce(0.5)
        assert ei.value.code == gss.GSS_E_STATE
