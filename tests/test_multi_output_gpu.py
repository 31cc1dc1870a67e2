"""GPU parity of the two-output mult (HD_MULT_BASDEVANT2, A = B = 2: from
u, v the products u v and u^2 - v^2, the nonlinear terms of 2D
incompressible Navier-Stokes in Basdevant's form) against the FP64 oracle,
through the C ABI: the fused 1D kernels of every kind and dtype (plain and
persistent bulk-copy variants), in-place outputs, 2D and 3D plans, the
autotuner, and the cases the path rejects.

Tolerances as for the single-output mults: FP64 on integer-valued inputs
rounds exactly to the oracle, FP32 rel-L2 <= 1e-5 per output.
"""
import numpy as np
import pytest

import inputs
from oracle import direct, params
from tests.gpu_util import rel_l2, rel_l2_rows, to_dev

pytestmark = pytest.mark.gpu

MULT = "basdevant2"


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def make_inputs(kind, L, count, seed, integer=False):
    if kind == "hermitian":
        return [inputs.hermitian_1d(count, L, seed + a, integer=integer) for a in range(2)]
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    return [gen((count, L), seed + a) for a in range(2)]


def run_b2(plan, fs, in_place=False):
    """Both outputs of a batched convolution, shape (2, count, n)."""
    import torch
    d = [to_dev(f, plan.dtype) for f in fs]
    outs = d if in_place else [torch.zeros_like(d[0]) for _ in range(2)]
    plan.convolve_batched(d, outs, d[0].shape[0], d[0].shape[1])
    torch.cuda.synchronize()
    return np.stack([o.cpu().numpy() for o in outs])


def check(got, ref, dtype, integer, ctx):
    assert got.shape == ref.shape, ctx
    if dtype == "f64" and integer:
        r = np.rint(got.real) + 1j * np.rint(got.imag)
        assert np.array_equal(r, ref), ctx
    else:
        for b in range(ref.shape[0]):
            e = rel_l2_rows(got[b], ref[b])
            assert e <= (1e-5 if dtype == "f32" else 1e-12), (ctx, b, e)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_basdevant2_1d_matches_oracle(hd, kind, dtype):
    integer = dtype == "f64"
    for L in (1, 2, 5, 31, 64, 255, 257, 1000):
        fs = make_inputs(kind, L, 3, 500 + L, integer)
        ref = direct.conv1d_batch(fs, kind, MULT)
        for M in (params.dealias_bound(kind, L, MULT), 2 * L + 3):
            with hd.Plan(L, M, A=2, B=2, kind=kind, dtype=dtype) as plan:
                got = run_b2(plan, fs)
            check(got, ref, dtype, integer, (kind, dtype, L, M))


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_basdevant2_every_candidate(hd, kind):
    """Every legal (m, p, q) and compiled kernel variant the enumeration offers."""
    L = 300
    M = params.dealias_bound(kind, L, MULT)
    fs = make_inputs(kind, L, 4, 610)
    ref = direct.conv1d_batch(fs, kind, MULT)
    cands = hd.enumerate_candidates(L=L, M=M, A=2, B=2, kind=kind)
    assert len(cands) >= 4
    for c in cands:
        with hd.Plan(L, M, A=2, B=2, kind=kind, candidate=c) as plan:
            got = run_b2(plan, fs)
        check(got, ref, "f32", False, (kind, c))


@pytest.mark.parametrize("kind,L,M", [("complex", 4096, 8191), ("centered", 4096, 6144), ("hermitian", 8192, 12288)])
def test_basdevant2_persistent_kernels(hd, kind, L, M):
    """Transforms of 256 threads or more run the persistent bulk-copy kernel
    on 16-byte aligned rows; a batch larger than the grid makes every CTA
    loop (sampled outputs against the oracle's direct sums)."""
    count = 640
    fs = make_inputs(kind, L, count, 620)
    cands = [c for c in hd.enumerate_candidates(L=L, M=M, A=2, B=2, kind=kind) if c["S"] // c["E"] >= 256]
    assert cands
    g = np.random.default_rng(5)
    rows = [0, 1, count // 2, count - 1]
    n = fs[0].shape[1]
    idx = np.unique(np.concatenate([[0, n - 1], g.integers(0, n, 24)]))
    for c in cands:
        with hd.Plan(L, M, A=2, B=2, kind=kind, candidate=c) as plan:
            got = run_b2(plan, fs)
        for i in rows:
            want = direct.conv1d_points([f[i] for f in fs], kind, idx, MULT)
            for b in range(2):
                assert rel_l2(got[b, i, idx], want[b]) <= 1e-5, (kind, c, i, b)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_basdevant2_in_place(hd, kind):
    """h[b] = f[b]: both inputs are staged before any output is written."""
    L = 777
    fs = make_inputs(kind, L, 5, 630)
    ref = direct.conv1d_batch(fs, kind, MULT)
    with hd.Plan(L, params.dealias_bound(kind, L, MULT), A=2, B=2, kind=kind) as plan:
        got = run_b2(plan, fs, in_place=True)
    check(got, ref, "f32", False, kind)


def run_nd_b2(plan, fs, dtype):
    import torch
    d = [to_dev(f, dtype) for f in fs]
    outs = [torch.zeros_like(d[0]) for _ in range(2)]
    plan.convolve(d, outs)
    torch.cuda.synchronize()
    return np.stack([o.cpu().numpy() for o in outs])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("L", [12, 33])
def test_basdevant2_2d_navier_stokes(hd, dtype, L):
    """2D incompressible flow: velocity spectra (centered x, Hermitian y) in,
    the spectra of u v and u^2 - v^2 out, against the N-D definition."""
    fs = [inputs.hermitian_2d(L, 640 + a, dtype=np.complex128) for a in range(2)]
    kinds = ("centered", "hermitian")
    ref = direct.convnd(fs, kinds, MULT)
    Ms = [params.dealias_bound(k, L, MULT) for k in kinds]
    with hd.Plan([L, L], Ms, A=2, B=2, kind="hermitian", dtype=dtype) as plan:
        got = run_nd_b2(plan, fs, dtype)
    for b in range(2):
        assert rel_l2(got[b], ref[b]) <= (1e-5 if dtype == "f32" else 1e-12), (dtype, L, b)


def test_basdevant2_2d_large_sampled(hd):
    """A 512^2 velocity field (M = 3L/2 per axis) on sampled output points."""
    L = 512
    fs = [inputs.hermitian_2d(L, 650 + a, dtype=np.complex64) for a in range(2)]
    kinds = ("centered", "hermitian")
    with hd.Plan([L, L], [3 * L // 2, 3 * L // 2], A=2, B=2, kind="hermitian") as plan:
        got = run_nd_b2(plan, fs, "f32")
    g = np.random.default_rng(6)
    pts = np.stack([g.integers(0, L, 40), g.integers(0, L // 2, 40)], 1)
    pts[0] = [L // 2, 0]
    want = direct.convnd_points([f.astype(np.complex128) for f in fs], kinds, pts, MULT)
    for b in range(2):
        assert rel_l2(got[b][tuple(pts.T)], want[b]) <= 1e-5, b


@pytest.mark.parametrize("kind", ["complex", "hermitian"])
def test_basdevant2_3d_and_outer_blocks(hd, kind):
    """3D recursion with two outputs, and the outermost residues one block at
    a time (a middle axis runs all of its residues in one block: its outputs
    overwrite its inputs, so fewer per block is refused)."""
    L = 10
    if kind == "hermitian":
        fs = [inputs.hermitian_3d(L, 660 + a, dtype=np.complex128) for a in range(2)]
        kinds = ("centered", "centered", "hermitian")
    else:
        fs = [inputs.uniform_complex((L, L, L), 660 + a) for a in range(2)]
        kinds = ("complex", "complex", "complex")
    ref = direct.convnd(fs, kinds, MULT)
    Ms = [params.dealias_bound(k, L, MULT) for k in kinds]
    for D in (0, 1):
        with hd.Plan([L, L, L], Ms, A=2, B=2, kind=kind, D=[D, 0, 0]) as plan:
            got = run_nd_b2(plan, fs, "f32")
        for b in range(2):
            assert rel_l2(got[b], ref[b]) <= 1e-5, (kind, D, b)
    with pytest.raises(hd.HdError) as e:
        hd.Plan([L, L, L], Ms, A=2, B=2, kind=kind, D=[0, 1, 0])
    assert e.value.name == "HD_ERR_UNSUPPORTED"


def test_basdevant2_autotune_and_cache(hd):
    """The tuner times the two-output candidates; a plan with m = 0 then takes
    the cached choice."""
    L, M = 2048, 3072
    hd.tune_cache_clear()
    best, allc = hd.autotune(256, reps=2, L=L, M=M, A=2, B=2, kind="centered")
    assert best["ms"] > 0 and len(allc) >= 3
    fs = make_inputs("centered", L, 6, 670)
    ref = direct.conv1d_batch(fs, "centered", MULT)
    with hd.Plan(L, M, A=2, B=2, kind="centered") as plan:
        pr = plan.params()
        got = run_b2(plan, fs)
    assert (pr["m"], pr["p"], pr["q"]) == (best["m"], best["p"], best["q"])
    check(got, ref, "f32", False, "tuned")
    hd.tune_cache_clear()
