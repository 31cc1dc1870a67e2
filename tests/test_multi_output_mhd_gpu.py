"""GPU parity of the eight-output mult (HD_MULT_MHD3, A = 6, B = 8: from the
Elsasser components z+ = u + b and z- = u - b of a 3D incompressible MHD flow,
the traceless part of the flux tensor z-_i z+_j) against the FP64 oracle,
through the C ABI: the fused 1D kernels of every kind and dtype (residue sums
of the eight outputs in shared memory, six forward spectra in registers),
in-place outputs, 3D Hermitian plans, and the cases the path rejects.  FP64 on
integer-valued inputs rounds exactly to the oracle; FP32 rel-L2 <= 1e-5 per
output and instance.
"""
import numpy as np
import pytest

import inputs
from oracle import direct, explicit, params
from tests.gpu_util import rel_l2, rel_l2_rows, to_dev

pytestmark = pytest.mark.gpu

MULT = "mhd3"
A, B = 6, 8


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def make_inputs(kind, L, count, seed, integer=False):
    if kind == "hermitian":
        return [inputs.hermitian_1d(count, L, seed + a, integer=integer) for a in range(A)]
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    return [gen((count, L), seed + a) for a in range(A)]


def run(plan, fs, in_place=False):
    """All B outputs of a batched convolution, shape (B, count, n); in place:
    outputs 0..A-1 over the inputs, the others in their own buffers."""
    import torch
    d = [to_dev(f, plan.dtype) for f in fs]
    outs = [d[b] if (in_place and b < A) else torch.zeros_like(d[0]) for b in range(B)]
    plan.convolve_batched(d, outs, d[0].shape[0], d[0].shape[1])
    torch.cuda.synchronize()
    return np.stack([o.cpu().numpy() for o in outs])


def check(got, ref, dtype, integer, ctx):
    assert got.shape == ref.shape, ctx
    if dtype == "f64" and integer:
        r = np.rint(got.real) + 1j * np.rint(got.imag)
        assert np.array_equal(r, ref), ctx
        assert np.max(np.abs(got - r)) < 1e-6, ctx
    else:
        for b in range(B):
            e = rel_l2_rows(got[b], ref[b])
            assert e <= (1e-5 if dtype == "f32" else 1e-12), (ctx, b, e)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_mhd3_1d_every_candidate(hd, kind, dtype):
    integer = dtype == "f64"
    ran = 0
    for L in (1, 5, 31, 100, 257):
        fs = make_inputs(kind, L, 3, 800 + L, integer)
        ref = direct.conv1d_batch(fs, kind, MULT)
        for M in (params.dealias_bound(kind, L, MULT), 2 * L + 3):
            for c in hd.enumerate_candidates(L=L, M=M, A=A, B=B, kind=kind, dtype=dtype):
                assert c["D"] <= 1 or kind == "hermitian"         # no cluster form with eight outputs
                with hd.Plan(L, M, A=A, B=B, kind=kind, dtype=dtype, candidate=c) as plan:
                    got = run(plan, fs)
                check(got, ref, dtype, integer, (kind, dtype, L, M, c))
                ran += 1
            with hd.Plan(L, M, A=A, B=B, kind=kind, dtype=dtype) as plan:   # automatic parameters
                check(run(plan, fs), ref, dtype, integer, (kind, dtype, L, M))
    assert ran >= 10


@pytest.mark.parametrize("kind", ["complex", "hermitian"])
def test_mhd3_in_place(hd, kind):
    """h[b] = f[b] for b < A: the inputs are staged before any output is written."""
    L = 500
    fs = make_inputs(kind, L, 4, 830)
    ref = direct.conv1d_batch(fs, kind, MULT)
    with hd.Plan(L, params.dealias_bound(kind, L, MULT), A=A, B=B, kind=kind) as plan:
        got = run(plan, fs, in_place=True)
    check(got, ref, "f32", False, kind)


def run_nd(plan, fs, dtype):
    import torch
    d = [to_dev(f, dtype) for f in fs]
    outs = [torch.zeros_like(d[0]) for _ in range(B)]
    plan.convolve(d, outs)
    torch.cuda.synchronize()
    return np.stack([o.cpu().numpy() for o in outs])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("L", [8, 11])
def test_mhd3_3d(hd, dtype, L):
    """3D incompressible MHD: Elsasser spectra (centered x, y, Hermitian z)
    in, the spectra of the eight flux-tensor products out, against the N-D
    definition."""
    fs = [inputs.hermitian_3d(L, 840 + a, dtype=np.complex128) for a in range(A)]
    kinds = ("centered", "centered", "hermitian")
    ref = direct.convnd(fs, kinds, MULT)
    Ms = [params.dealias_bound(k, L, MULT) for k in kinds]
    with hd.Plan([L, L, L], Ms, A=A, B=B, kind="hermitian", dtype=dtype) as plan:
        got = run_nd(plan, fs, dtype)
    for b in range(B):
        assert rel_l2(got[b], ref[b]) <= (1e-5 if dtype == "f32" else 1e-12), (dtype, L, b)


def test_mhd3_3d_whole_field(hd):
    """A 64^3 Elsasser field (M = 96 per axis, the 2/3 rule): every output over
    the whole stored field against the FP64 explicit zero-padded FFT
    convolution of the expanded Hermitian arrays on 96^3, and sampled points
    against the exact direct sums."""
    L = 64
    fs = [inputs.hermitian_3d(L, 850 + a, dtype=np.complex64) for a in range(A)]
    kinds = ("centered", "centered", "hermitian")
    with hd.Plan([L, L, L], [96, 96, 96], A=A, B=B, kind="hermitian") as plan:
        got = run_nd(plan, fs, "f32")
    f64 = [f.astype(np.complex128) for f in fs]
    full = explicit.convnd_explicit(f64, kinds, [96, 96, 96], MULT)
    for b in range(B):
        assert rel_l2(got[b], full[b]) <= 1e-5, b
    g = np.random.default_rng(8)
    pts = np.stack([g.integers(0, L, 24), g.integers(0, L, 24), g.integers(0, L // 2, 24)], 1)
    want = direct.convnd_points(f64, kinds, pts, MULT)
    for b in range(B):
        assert np.allclose(full[b][tuple(pts.T)], want[b], rtol=1e-10, atol=1e-10 * np.max(np.abs(want[b])))
        assert rel_l2(got[b][tuple(pts.T)], want[b]) <= 1e-5, b


def test_mhd3_rejections(hd):
    """(A, B) must match the mult; ragged batches take one output."""
    with pytest.raises(hd.HdError) as e:
        hd.Plan(100, 199, A=3, B=8, mult="mhd3")
    assert e.value.name == "HD_ERR_INVALID"
    with pytest.raises(hd.HdError) as e:
        hd.RaggedPlan([dict(L=100, M=199, A=6, kind="complex", mult="mhd3")])
