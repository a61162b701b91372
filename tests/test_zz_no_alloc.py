"""gss_test_noalloc: the clause test for callers that cannot allocate device memory.

It must give the same records as the context API, call after call, from its fixed
working array.  Collected last (file name) so that a run stopping at the first failure
has already run every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import paper_2012_03119_gb300 as gss
import synth

pytestmark = pytest.mark.gpu


def context_pairs(inst, mode):
    with gss.Context(inst.n_vars, mode=mode, max_assignments=max(inst.n_assign, 32),
                     report_capacity=inst.n_clauses * ((inst.n_assign + 31) // 32) + 1024) as ctx:
        ctx.add_clauses(inst.offsets, inst.lits)
        return gss.expand_reports(ctx.run(inst.codes))


def noalloc_pairs(inst, mode):
    import torch
    off = torch.from_numpy(inst.offsets.view(np.int64)).cuda()
    lits = torch.from_numpy(inst.lits.view(np.int32)).cuda()
    V, N = inst.n_vars, inst.n_assign
    pitch = (V + 15) // 16 * 16
    codes = torch.zeros((N, pitch), dtype=torch.uint8, device="cuda")
    codes[:, :V] = torch.from_numpy(inst.codes).cuda()
    cap = inst.n_clauses * ((N + 31) // 32) + 1024
    out = torch.empty(cap * 3, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    gss.gss_test_noalloc(off.data_ptr(), inst.n_clauses, lits.data_ptr(), V, codes.data_ptr(), pitch, N, mode,
                         out.data_ptr(), cap, count.data_ptr())
    n = int(count.item())
    rec = out[: 3 * n].cpu().numpy().view(np.uint32).view(gss.REPORT_DTYPE)
    return gss.expand_reports(rec)


@pytest.mark.parametrize("mode", [gss.GSS_MODE_ALLF, gss.GSS_MODE_TRIGGER])
def test_two_calls_match_context(mode):
    first = synth.single(scale=0.01)                        # 10k vars, 40k clauses, N = 1024
    second = synth.single(scale=0.005, seed=12345, n_assign=700)  # different sizes: stale scratch must not leak
    for inst in (first, second):
        assert np.array_equal(noalloc_pairs(inst, mode), context_pairs(inst, mode))


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
