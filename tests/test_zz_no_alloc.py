"""gss_test_noalloc: the clause test for callers that cannot allocate device memory.

Some callers own no allocator at the moment they test: their GPU memory belongs to another
runtime's pool reserved up front, or they run in a loop where a cudaMalloc, which may
synchronise the whole device, is not acceptable.  This entry point works in one fixed array
compiled into the library.  It must give the oracle's records, call after call, from that
array; it must leave the device's free memory unchanged; and it must report an overflow
with the full count.  Collected last (file name) so that a run stopping at the first failure
has already run every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle
import paper_2012_03119_gb300 as gss
import synth

pytestmark = pytest.mark.gpu


class Buffers:
    """Device copies of an instance and output space, made before the calls under test."""

    def __init__(self, inst, cap=None):
        import torch
        self.inst = inst
        V, N = inst.n_vars, inst.n_assign
        self.off = torch.from_numpy(inst.offsets.view(np.int64)).cuda()
        self.lits = torch.from_numpy(inst.lits.view(np.int32)).cuda()
        self.pitch = (V + 15) // 16 * 16
        self.codes = torch.zeros((N, self.pitch), dtype=torch.uint8, device="cuda")
        self.codes[:, :V] = torch.from_numpy(inst.codes).cuda()
        self.cap = inst.n_clauses * ((N + 31) // 32) + 1024 if cap is None else cap
        self.out = torch.zeros(max(1, self.cap) * 3, dtype=torch.int32, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()

    def call(self, mode, cap=None):
        cap = self.cap if cap is None else cap
        gss.gss_test_noalloc(self.off.data_ptr(), self.inst.n_clauses, self.lits.data_ptr(), self.inst.n_vars,
                             self.codes.data_ptr(), self.pitch, self.inst.n_assign, mode, self.out.data_ptr(), cap,
                             self.count.data_ptr())

    def pairs(self):
        n = int(self.count.item())
        rec = self.out[: 3 * n].cpu().numpy().view(np.uint32).view(gss.REPORT_DTYPE)
        return gss.expand_reports(rec)


def oracle_pairs(inst, mode):
    return oracle.pairs(inst.offsets, inst.lits, inst.codes, mode)


def context_pairs(inst, mode):
    with gss.Context(inst.n_vars, mode=mode, max_assignments=max(inst.n_assign, 32),
                     report_capacity=inst.n_clauses * ((inst.n_assign + 31) // 32) + 1024) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        return gss.expand_reports(ctx.run(inst.codes))


@pytest.mark.parametrize("mode", [gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER])
def test_two_calls_match_oracle_and_context(mode):
    """Two calls in a row on different problems: each equals the oracle and the context API
    (stale contents of the shared array from the first call must not leak into the second)."""
    first = synth.single(scale=0.01)                        # 10k vars, 40k clauses, N = 1024
    second = synth.single(scale=0.005, seed=12345, n_assign=700)  # different sizes, ragged last word
    for inst in (first, second):
        b = Buffers(inst)
        b.call(mode)
        got = b.pairs()
        np.testing.assert_array_equal(got, oracle_pairs(inst, mode))
        np.testing.assert_array_equal(got, context_pairs(inst, mode))


def test_allocates_nothing():
    """A warmed-up call leaves the device's free memory and torch's pool unchanged."""
    import torch
    inst = synth.single(scale=0.005)
    b = Buffers(inst)
    b.call(gss.GSS_MODE_ALLF)  # warm-up: loads the library's kernels and looks up the array's address
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(3):
        b.call(gss.GSS_MODE_ALLF)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    np.testing.assert_array_equal(b.pairs(), oracle_pairs(inst, oracle.MODE_ALLF))


def test_overflow_reports_the_full_count():
    """A capacity below the record count: GSS_E_OVERFLOW, the full count in *d_count and the
    records that fit written; the next call with room gives the whole set again."""
    inst = synth.single(scale=0.005)
    b = Buffers(inst)
    b.call(gss.GSS_MODE_ALLF)
    full = int(b.count.item())
    assert full > 20
    with pytest.raises(gss.GssError) as ei:
        b.call(gss.GSS_MODE_ALLF, cap=17)
    assert ei.value.code == gss.GSS_E_OVERFLOW
    assert int(b.count.item()) == full
    want = set(map(tuple, oracle_pairs(inst, oracle.MODE_ALLF).tolist()))
    part = b.out[: 3 * 17].cpu().numpy().view(np.uint32).view(gss.REPORT_DTYPE)
    assert set(map(tuple, gss.expand_reports(part).tolist())) <= want
    b.call(gss.GSS_MODE_ALLF)
    np.testing.assert_array_equal(b.pairs(), oracle_pairs(inst, oracle.MODE_ALLF))


def test_rejects_problems_beyond_the_scratch_size():
    import torch
    V = 1_000_000  # planes alone need about 270 MB at N = 1024
    off = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    lits = torch.tensor([0], dtype=torch.int32, device="cuda")
    codes = torch.zeros((1024, 16), dtype=torch.uint8, device="cuda")  # never read: rejected before any work
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(gss.GssError) as ei:
        gss.gss_test_noalloc(off.data_ptr(), 1, lits.data_ptr(), V, codes.data_ptr(), 1_000_000, 1024,
                             gss.GSS_MODE_ALLF, 0, 0, count.data_ptr())
    assert ei.value.code == gss.GSS_E_INVAL and "GSS_NOALLOC_SCRATCH_BYTES" in str(ei.value)
