"""GPU parity of the split path (residue transforms larger than one CTA,
computed as size-S1 DFTs along the block index and size-S2 row FFTs through a
work buffer, Section 6.1) against the FP64 direct oracle."""
import numpy as np
import pytest

import inputs
from oracle import cdirect, params
from tests.gpu_util import rel_l2_rows, run_conv
from tests.test_conv1d_gpu import check, make_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def split_cands(hd, **kw):
    lim = 4096 if kw.get("dtype", "f32") == "f32" else 2048
    return [c for c in hd.enumerate_candidates(**kw) if c["S"] > lim]


@pytest.mark.parametrize("kind,L,A", [("complex", 9000, 2), ("centered", 20000, 2), ("hermitian", 30001, 2),
                                      ("complex", 6000, 3), ("centered", 9999, 3)])
def test_split_f32_matches_oracle(hd, kind, L, A):
    M = params.dealias_bound(kind, L) + 11
    fs = make_inputs(kind, L, A, 2, 300 + L)
    mult = "product" if A == 2 else "sum_pairs3"
    ref = cdirect.conv1d_batch(fs, L, kind, mult)
    cands = split_cands(hd, L=L, M=M, A=A, kind=kind)
    assert cands, "no split candidate"
    for c in cands:
        with hd.Plan(L, M, A=A, kind=kind, candidate=c) as plan:
            assert plan.params()["scratch_bytes"] > 0
            got = run_conv(hd, plan, fs)
            e = rel_l2_rows(got, ref)
            assert e <= 1e-5, (c, e)


def test_split_f64_explicit_is_exact_on_integers(hd):
    L, M = 4096, 8191
    fs = make_inputs("complex", L, 2, 3, 17, integer=True)
    ref = cdirect.conv1d_batch(fs, L, "complex")
    with hd.Plan(L, M, m=8192, p=1, q=1, dtype="f64") as plan:
        assert plan.params()["scratch_bytes"] > 0
        got = run_conv(hd, plan, fs)
        check(got, ref, "f64", True, "explicit f64 S=8192")


def test_split_chunking_and_inplace(hd):
    """More instances than one scratch chunk, and h = f_0 in place."""
    import torch
    L, M = 20000, 39999
    count = 70
    fs = make_inputs("complex", L, 2, count, 5)
    ref_idx = [0, 33, 69]
    ref = cdirect.conv1d_batch([f[ref_idx] for f in fs], L, "complex")
    c = split_cands(hd, L=L, M=M)[0]
    with hd.Plan(L, M, candidate=c) as plan:
        per_instance = 2 * c["n"] * c["S"] * 8          # work buffer: A n S complex64 values
        assert plan.params()["scratch_bytes"] // per_instance < count   # several chunks
        d = [torch.from_numpy(f.astype(np.complex64)).cuda() for f in fs]
        plan.convolve_batched(d, d[0], count, L)
        torch.cuda.synchronize()
        got = d[0].cpu().numpy()[ref_idx]
        assert rel_l2_rows(got, ref) <= 1e-5


@pytest.mark.parametrize("kind,L,A", [("complex", 9000, 2), ("centered", 20000, 2), ("hermitian", 30001, 2),
                                      ("complex", 6000, 3)])
def test_split_residue_blocks(hd, kind, L, A):
    """D residues per pass on the split path (Section 6.5): the residues run in
    blocks of D whose contributions are added into the output, so the work
    buffer holds A D S values per instance instead of A n S.  Every block size
    gives the oracle's result; writing over an input is refused."""
    import torch
    M = 2 * params.dealias_bound(kind, L) + 11          # more residues than the tightest padding
    mult = "product" if A == 2 else "sum_pairs3"
    fs = make_inputs(kind, L, A, 3, 900 + L)
    ref = cdirect.conv1d_batch(fs, L, kind, mult)
    c = max(split_cands(hd, L=L, M=M, A=A, kind=kind), key=lambda c: c["n"])
    assert c["n"] >= 3, c
    with hd.Plan(L, M, A=A, kind=kind, candidate=c) as plan:
        one = plan.params()["scratch_bytes"]
    for D in (2, c["n"] - 1):
        with hd.Plan(L, M, A=A, kind=kind, m=c["m"], p=c["p"], q=c["q"], D=D) as plan:
            ax = plan.axis_params(0)
            assert (ax["S"], ax["n"], ax["D"]) == (c["S"], c["n"], D)
            per_block = A * D * c["S"] * 8
            assert plan.params()["scratch_bytes"] % per_block == 0
            assert plan.params()["scratch_bytes"] // per_block >= one // (A * c["n"] * c["S"] * 8)
            got = run_conv(hd, plan, fs)
            assert rel_l2_rows(got, ref) <= 1e-5, (kind, D)
            d = [torch.from_numpy(f.astype(np.complex64)).cuda() for f in fs]
            with pytest.raises(hd.HdError) as e:
                plan.convolve_batched(d, d[0], 3, fs[0].shape[1])
            assert e.value.name == "HD_ERR_INVALID"


@pytest.mark.parametrize("mult,kind,L", [("basdevant2", "complex", 9000), ("basdevant2", "hermitian", 20001),
                                         ("basdevant3", "centered", 9999), ("mhd3", "complex", 6000),
                                         ("mhd3", "hermitian", 12001)])
def test_split_multi_output(hd, mult, kind, L):
    """B > 1 outputs on the split path: the rows form the B output spectra (two
    together, or one at a time for five and eight) and write output b over part
    b of the work buffer, which holds max(A, B) parts per residue; every output
    of every candidate against the FP64 oracle, FP32 rel-L2 <= 1e-5 per output
    and instance, and one FP64 case exact after rint on integer inputs."""
    import torch
    A, B = {"basdevant2": (2, 2), "basdevant3": (3, 5), "mhd3": (6, 8)}[mult]
    M = params.dealias_bound(kind, L, mult) + 11
    fs = make_inputs(kind, L, A, 2, 950 + L)
    ref = cdirect.conv1d_batch(fs, L, kind, mult)
    cands = split_cands(hd, L=L, M=M, A=A, B=B, kind=kind)
    assert cands, "no split candidate"
    for c in cands[:3]:
        with hd.Plan(L, M, A=A, B=B, kind=kind, candidate=c) as plan:
            assert plan.params()["scratch_bytes"] % (max(A, B) * c["S"] * 8) == 0
            d = [torch.from_numpy(f.astype(np.complex64)).cuda() for f in fs]
            outs = [torch.zeros_like(d[0]) for _ in range(B)]
            plan.convolve_batched(d, outs, 2, fs[0].shape[1])
            torch.cuda.synchronize()
            for b in range(B):
                e = rel_l2_rows(outs[b].cpu().numpy(), ref[b])
                assert e <= 1e-5, (c, b, e)
    if mult == "basdevant2" and kind == "complex":
        fi = make_inputs(kind, 4096, A, 2, 960, integer=True)
        refi = cdirect.conv1d_batch(fi, 4096, kind, mult)
        with hd.Plan(4096, 8191, A=A, B=B, m=8192, p=1, q=1, dtype="f64") as plan:
            d = [torch.from_numpy(f).cuda() for f in fi]
            outs = [torch.zeros_like(d[0]) for _ in range(B)]
            plan.convolve_batched(d, outs, 2, 4096)
            torch.cuda.synchronize()
            for b in range(B):
                g = outs[b].cpu().numpy()
                assert np.array_equal(np.rint(g.real) + 1j * np.rint(g.imag), refi[b]), b
