"""Two plane sets (pipeline = 2): the packing of the next assignment set runs on its own
stream while the last set's test runs.  Records must be those of each set alone, whatever
the interleaving of set / test / fetch calls."""
import numpy as np
import pytest

import oracle
import paper_2012_03119_gb300 as gss
import synth

pytestmark = pytest.mark.gpu


def sets_for(inst, k, seed0=100):
    out = [inst.codes]
    for i in range(1, k):
        out.append(synth.assign_trail(inst.n_vars, inst.n_assign, 0.3, 0.7, seed0 + i))
    return out


@pytest.mark.parametrize("mode", [gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER])
def test_interleaved_sets_equal_each_set_alone(mode):
    import torch
    inst = synth.single(scale=0.01)  # 10k vars, 40k clauses, 1024 trail assignments
    sets = sets_for(inst, 5)
    want = [oracle.pairs(inst.offsets, inst.lits, c, mode) for c in sets]
    d_sets = [torch.from_numpy(c).cuda() for c in sets]
    cap = inst.n_clauses * 32 + 1024
    with gss.Context(inst.n_vars, max_assignments=1024, report_capacity=cap, mode=mode, pipeline=2) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        torch.cuda.synchronize()
        # set k + 1 is given (packed on the second stream) before set k's records are read
        ctx.set_assignments(d_sets[0])
        for k in range(len(sets)):
            ctx.test()
            if k + 1 < len(sets):
                ctx.set_assignments(d_sets[k + 1] if k % 2 else sets[k + 1])  # device and host sets alternate
            got = gss.expand_reports(ctx.fetch_reports())
            np.testing.assert_array_equal(got, want[k])
        # and again in the plain order
        for k in range(len(sets)):
            np.testing.assert_array_equal(gss.expand_reports(ctx.run(sets[k])), want[k])


def test_second_set_without_test_drops_the_last_results():
    """Two sets in a row after a test: the second reuses the tested plane set, so the last
    test's results are gone (GSS_E_STATE), and the next test reads the newest set."""
    inst = synth.single(scale=0.005)
    a, b, c = sets_for(inst, 3)
    with gss.Context(inst.n_vars, max_assignments=1024, report_capacity=1 << 22, pipeline=2) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.set_assignments(a)
        ctx.test()
        ctx.set_assignments(b)
        np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_reports()),
                                      oracle.allf_pairs(inst.offsets, inst.lits, a))
        ctx.set_assignments(c)
        ctx.test()
        np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_reports()),
                                      oracle.allf_pairs(inst.offsets, inst.lits, c))
        ctx.set_assignments(a)
        ctx.set_assignments(b)
        with pytest.raises(gss.GssError) as ei:
            ctx.fetch_reports()
        assert ei.value.code == gss.GSS_E_STATE
        ctx.test()
        np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_reports()),
                                      oracle.allf_pairs(inst.offsets, inst.lits, b))


def test_pipelined_wide_sets_and_stats():
    """Sets above 4096 assignments (second aggregate level) through two plane sets, and the
    statistics of the last test while the next set is being packed."""
    V, N = 600, 5000
    off = synth.offsets_from_sizes(synth.clause_sizes(3000, "geom", 1 / 7, 0, 30, V, 5))
    lits = synth.clause_lits(off, V, 5)
    s1 = synth.assign_trail(V, N, 0.3, 0.7, 5, group=1024, flip_frac=0.1)
    s2 = synth.assign_trail(V, N - 333, 0.3, 0.7, 6, group=1024, flip_frac=0.1)
    with gss.Context(V, max_assignments=N, report_capacity=1 << 20, pipeline=2) as ctx:
        ctx.add_clauses(off, lits)
        ctx.set_assignments(s1)
        ctx.test()
        ctx.set_assignments(s2)
        got1 = gss.expand_reports(ctx.fetch_reports())
        st = ctx.stats()
        assert st["group_pairs"] == 3000 * ((N + 31) // 32)
        want_groups = oracle.aggregate_pairs(off, lits, s1, group=32)
        assert st["candidate_pairs"] == len(want_groups)
        ctx.test()
        got2 = gss.expand_reports(ctx.fetch_reports())
    np.testing.assert_array_equal(got1, oracle.allf_pairs(off, lits, s1))
    np.testing.assert_array_equal(got2, oracle.allf_pairs(off, lits, s2))


def test_pipeline_config_checks():
    with pytest.raises(gss.GssError) as ei:
        gss.Context(100, pipeline=3)
    assert ei.value.code == gss.GSS_E_INVAL


def test_async_fetch():
    """gss_fetch_reports_async writes the records into the caller's buffer on the stream, so
    the next set can be given before they are waited for; the results equal gss_fetch_reports,
    overflow reports the full count, and a buffer the GPU cannot write is refused."""
    import torch
    inst = synth.single(scale=0.005)
    a, b = sets_for(inst, 2)
    want_a = oracle.allf_pairs(inst.offsets, inst.lits, a)
    want_b = oracle.allf_pairs(inst.offsets, inst.lits, b)
    cap = 1 << 20
    pinned = torch.empty(cap * 12, dtype=torch.uint8).pin_memory().numpy().view(gss.REPORT_DTYPE)
    with gss.Context(inst.n_vars, max_assignments=1024, report_capacity=cap, pipeline=2) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        with pytest.raises(gss.GssError) as ei:
            ctx.fetch_wait()
        assert ei.value.code == gss.GSS_E_STATE
        ctx.set_assignments(a)
        ctx.test()
        ctx.fetch_reports_async(pinned)
        ctx.set_assignments(b)  # set b's copy and packing while set a's records travel
        np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_wait()), want_a)
        ctx.test()
        ctx.fetch_reports_async(pinned)
        np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_wait()), want_b)
        n_all = ctx.report_count()
        ctx.fetch_reports_async(pinned[:5])  # too small: the first 5 records, the full count
        with pytest.raises(gss.GssError) as ei:
            ctx.fetch_wait()
        assert ei.value.code == gss.GSS_E_OVERFLOW and n_all > 5
        part = gss.expand_reports(pinned[:5])
        assert set(map(tuple, part.tolist())) <= set(map(tuple, want_b.tolist()))
        # pageable memory: written where the device can reach it, refused where it cannot
        pageable = np.zeros(cap, gss.REPORT_DTYPE)
        try:
            ctx.fetch_reports_async(pageable)
        except gss.GssError as e:
            assert e.code == gss.GSS_E_INVAL
        else:
            np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_wait()), want_b)


def test_host_sets_alternate_staging_buffers():
    """Host sets through two plane sets: each set is copied into its own staging buffer on a
    copy stream, while the last set is packed and tested.  The caller's buffer is free once
    gss_set_assignments returns (it is overwritten with invalid codes at once), sets of
    different sizes follow each other, and every test equals the oracle on its own set."""
    inst = synth.single(scale=0.005)
    sizes = [1024, 700, 1024, 33, 512, 1024]
    sets = [c[:n] for c, n in zip(sets_for(inst, len(sizes)), sizes)]
    want = [oracle.allf_pairs(inst.offsets, inst.lits, c) for c in sets]
    buf = np.empty((1024, inst.n_vars), np.uint8)
    with gss.Context(inst.n_vars, max_assignments=1024, report_capacity=1 << 22, pipeline=2) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)

        def give(k):
            n = len(sets[k])
            buf[:n] = sets[k]
            ctx.set_assignments(buf[:n])
            buf[:] = 3  # invalid codes: a copy still reading the buffer would see them

        give(0)
        for k in range(len(sets)):
            ctx.test()
            if k + 1 < len(sets):
                give(k + 1)
            np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_reports()), want[k])


@pytest.mark.parametrize("pipeline", [1, 2])
def test_async_host_sets(pipeline):
    """gss_set_assignments_async returns once the copy is queued (with two plane sets, set k+1's
    copy queues behind set k's while set k is tested); every test equals the oracle on its set,
    and after gss_copy_wait the caller's buffers are free: overwriting them changes nothing."""
    import torch
    inst = synth.single(scale=0.005)
    sets = sets_for(inst, 4)
    want = [oracle.allf_pairs(inst.offsets, inst.lits, c) for c in sets]
    bufs = []
    for c in sets:
        b = torch.empty(c.shape, dtype=torch.uint8).pin_memory().numpy()
        b[:] = c
        bufs.append(b)
    with gss.Context(inst.n_vars, max_assignments=1024, report_capacity=1 << 22, pipeline=pipeline) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        ctx.set_assignments_async(bufs[0])
        for k in range(len(sets)):
            ctx.test()
            if k + 1 < len(sets) and pipeline == 2:
                ctx.set_assignments_async(bufs[k + 1])
            np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_reports()), want[k])
            if k + 1 < len(sets) and pipeline == 1:
                ctx.set_assignments_async(bufs[k + 1])
        ctx.copy_wait()
        for b in bufs:
            b[:] = 3  # invalid codes, written after the wait: no queued copy reads them
        ctx.test()
        np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_reports()), want[-1])
    with pytest.raises(ValueError):
        with gss.Context(inst.n_vars, max_assignments=1024) as ctx:
            ctx.set_assignments_async(torch.from_numpy(sets[0]).cuda())


def test_device_sets_ordered_on_the_pack_stream():
    """Device values in a layout the packer cannot read in place (a pitch that is not a multiple
    of 16) are staged by a copy on pack_stream: values written by work the caller queued on
    pack_stream, with no host synchronisation, are the ones packed."""
    import torch
    inst = synth.single(scale=0.005)  # 5000 vars
    sets = sets_for(inst, 3)
    want = [oracle.allf_pairs(inst.offsets, inst.lits, c) for c in sets]
    N, V = sets[0].shape
    pitch = V + 3
    ps = torch.cuda.Stream()
    pinned = [torch.from_numpy(c).pin_memory() for c in sets]
    bufs = [torch.zeros((N, pitch), dtype=torch.uint8, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    with gss.Context(V, max_assignments=1024, report_capacity=1 << 22, pipeline=2, pack_stream=ps) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        for k in range(len(sets)):
            d = bufs[k % 2]
            with torch.cuda.stream(ps):
                d[:, :V].copy_(pinned[k], non_blocking=True)  # written on pack_stream
            gss.gss_set_assignments_device(ctx.ptr, d.data_ptr(), pitch, N)
            ctx.test()
            np.testing.assert_array_equal(gss.expand_reports(ctx.fetch_reports()), want[k])
