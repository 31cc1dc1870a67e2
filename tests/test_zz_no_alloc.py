"""GPU test of hd_convolve_batched_noalloc, the allocation-free batched call.

It serves callers that cannot allocate device memory while they convolve (a
service that reserves its GPU memory at start-up, code inside another
runtime's memory manager, a hot loop that must not synchronize the device on
an allocation).  It runs the split path over the library's fixed work buffer
instead of the plan's own.  The test calls it through the C ABI twice in a
row: the kernels and the per-instance work are those of hd_convolve_batched
(only the chunking of the batch differs), so each result must equal
hd_convolve_batched's bit for bit; rows on both sides of a chunk boundary are
also compared with the FP64 oracle within the FP32 tolerance of the other
parity tests (rel-L2 <= 1e-5).  It also checks the size limit, the plans the
call refuses and a plan created without its own work buffer.  It is self-contained, so it runs alone
in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import inputs
from oracle import cdirect

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
NOALLOC_BYTES = 32 << 20       # HD_NOALLOC_SCRATCH_BYTES in include/hd.h


def _rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def _call(b, plan, count, fs, h, stride):
    import torch
    fa = (ctypes.c_void_p * len(fs))(*[x.data_ptr() for x in fs])
    ha = (ctypes.c_void_p * 1)(h.data_ptr())
    return b.lib.hd_convolve_batched_noalloc(ctypes.c_void_p(plan.handle), count, fa, ha, stride,
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_batched_on_two_calls(hd):
    import torch
    from paper_2303_17510_gb300 import _binding as b

    L, M, count = 9000, 18010, 70
    cand = [c for c in hd.enumerate_candidates(L=L, M=M) if c["S"] > 4096][0]
    per_instance = 2 * cand["n"] * cand["S"] * 8
    chunk = NOALLOC_BYTES // per_instance
    assert count > chunk                                 # the batch needs more than one chunk
    host = [inputs.uniform_complex((count, L), 900 + a, dtype=np.complex64) for a in range(2)]
    f = [torch.from_numpy(x).cuda() for x in host]
    rows = sorted({0, chunk - 1, chunk, count - 1})      # first, last, both sides of a chunk boundary
    want_rows = cdirect.conv1d_batch([x[rows].astype(np.complex128) for x in host], L, "complex")
    with hd.Plan(L, M, candidate=cand) as plan:
        ref = torch.empty_like(f[0])
        plan.convolve_batched(f, ref, count, L)
        torch.cuda.synchronize()
        want = ref.cpu().numpy()
        for call in range(2):
            out = torch.full_like(f[0], float("nan"))
            rc = _call(b, plan, count, f, out, L)
            assert rc == 0, b.STATUS.get(rc, rc)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.array_equal(got, want), call
            for k, r in enumerate(rows):
                assert _rel_l2(got[r].astype(np.complex128), want_rows[k]) <= F32_TOL, (call, r)


def test_noalloc_plan_without_work_buffer(hd):
    """A plan created with HD_PLAN_NO_WORK_BUFFER allocates no work buffer of
    its own; only the allocation-free call runs it, with the same result."""
    import torch
    from paper_2303_17510_gb300 import _binding as b

    L, M, count = 20000, 39999, 5
    cand = [c for c in hd.enumerate_candidates(L=L, M=M) if c["S"] > 4096][0]
    host = [inputs.uniform_complex((count, L), 950 + a, dtype=np.complex64) for a in range(2)]
    f = [torch.from_numpy(x).cuda() for x in host]
    with hd.Plan(L, M, candidate=cand) as plan:
        ref = torch.empty_like(f[0])
        plan.convolve_batched(f, ref, count, L)
        torch.cuda.synchronize()
    with hd.Plan(L, M, candidate=cand, flags=hd.PLAN_NO_WORK_BUFFER) as plan:
        assert plan.params()["scratch_bytes"] == 0
        out = torch.full_like(f[0], float("nan"))
        with pytest.raises(hd.HdError) as e:
            plan.convolve_batched(f, out, count, L)
        assert e.value.name == "HD_ERR_UNSUPPORTED"
        assert b.STATUS[_call(b, plan, count, f, out, L)] == "HD_OK"
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    with pytest.raises(hd.HdError) as e:                       # unknown flag bits
        hd.Plan(L, M, flags=2)
    assert e.value.name == "HD_ERR_INVALID"


def test_noalloc_rejects_oversize_and_other_plans(hd):
    import torch
    from paper_2303_17510_gb300 import _binding as b

    # one instance needs A n S * 8 bytes = 2 * 33 * 65536 * 8 > 32 MiB
    L, M = 60000, 33 * 65536
    cand = [c for c in hd.enumerate_candidates(L=L, M=M) if c["S"] == 65536][0]
    assert 2 * cand["n"] * cand["S"] * 8 > NOALLOC_BYTES
    x = torch.zeros(L, dtype=torch.complex64, device="cuda")
    with hd.Plan(L, M, candidate=cand) as plan:
        assert b.STATUS[_call(b, plan, 1, [x, x], x, L)] == "HD_ERR_SCRATCH_LIMIT"
    y = torch.zeros(1024, dtype=torch.complex64, device="cuda")
    with hd.Plan(1024, 2047) as plan:                        # fused path: no work buffer
        assert b.STATUS[_call(b, plan, 1, [y, y], y, 1024)] == "HD_ERR_UNSUPPORTED"
    with hd.RaggedPlan([dict(L=9000, M=17999, A=2, kind="complex")]) as plan:
        assert b.STATUS[_call(b, plan, 1, [y, y], y, 1024)] == "HD_ERR_INVALID"


def test_noalloc_residue_blocks_lift_the_size_limit(hd):
    """An instance whose work buffer for all residues exceeds the fixed buffer
    (A n S values) runs when its plan processes the residues in blocks of D
    (A D S values per instance): same result as hd_convolve_batched on the same
    plan, bit for bit, and the FP32 bound against the oracle on sampled points."""
    import torch
    from paper_2303_17510_gb300 import _binding as b

    L, M = 60000, 33 * 65536
    cand = [c for c in hd.enumerate_candidates(L=L, M=M) if c["S"] == 65536][0]
    assert 2 * cand["n"] * cand["S"] * 8 > NOALLOC_BYTES
    host = [inputs.uniform_complex((1, L), 990 + a, dtype=np.complex64) for a in range(2)]
    f = [torch.from_numpy(x[0]).cuda() for x in host]
    with hd.Plan(L, M, m=cand["m"], p=cand["p"], q=cand["q"], D=16) as plan:
        assert 2 * 16 * cand["S"] * 8 <= NOALLOC_BYTES
        ref = torch.empty_like(f[0])
        plan.convolve_batched(f, ref, 1, L)
        out = torch.full_like(f[0], float("nan"))
        assert b.STATUS[_call(b, plan, 1, f, out, L)] == "HD_OK"
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    idx = np.unique(np.linspace(0, L - 1, 48).astype(np.int64))
    want = cdirect.conv1d_points([x[0].astype(np.complex128) for x in host], L, idx, "complex")
    assert _rel_l2(out.cpu().numpy()[idx].astype(np.complex128), want) <= F32_TOL
