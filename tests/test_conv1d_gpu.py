"""GPU parity of the fused 1D kernels against the FP64 oracle (through the C ABI).

Tolerances: FP64 on integer-valued inputs must round (rint) to the exact
oracle result; FP64 on real-valued inputs rel-L2 <= 1e-12; FP32 rel-L2 <=
1e-5 (the FP32 contract: FFT rounding grows like eps * log2 S, eps = 6e-8,
and the residue sum is compensated from 8 residues on).  Norms are taken
per instance of a batch and the largest must meet the bound.
"""
import numpy as np
import pytest

import inputs
from oracle import cdirect, direct, params, residue
from tests.gpu_util import rel_l2, rel_l2_rows, run_conv, to_dev

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
F64_TOL = 1e-12


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def make_inputs(kind, L, A, count, seed, integer=False):
    if kind == "hermitian":
        return [inputs.hermitian_1d(count, L, seed + a, integer=integer) for a in range(A)]
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    return [gen((count, L), seed + a) for a in range(A)]


def check(got, ref, dtype, integer, ctx):
    if dtype == "f64" and integer:
        r = np.rint(got.real) + 1j * np.rint(got.imag)
        assert np.array_equal(r, ref), ctx
        assert np.max(np.abs(got - r)) < 1e-6, ctx
    else:
        tol = F32_TOL if dtype == "f32" else F64_TOL
        e = rel_l2_rows(got, ref)
        assert e <= tol, (ctx, e)


def candidate_ms(M):
    ms, m = [], 1
    while m <= 2 * M:
        ms.append(m)
        m *= 2
    return ms


SMALL_L = [1, 2, 3, 5, 8, 13, 31, 64, 100, 255, 256, 257, 1000, 1024]


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("mult", ["product", "sum_pairs3"])
def test_every_supported_m(hd, kind, dtype, mult):
    A = 2 if mult == "product" else 3
    integer = dtype == "f64"
    ran = 0
    for L in SMALL_L:
        fs = make_inputs(kind, L, A, 3, 100 + L, integer=integer)
        ref = direct.conv1d_batch(fs, kind, mult)
        lo = params.dealias_bound(kind, L, mult)
        for M in sorted({lo, lo + 1, 3 * L + 1}):
            for m in candidate_ms(M):
                try:
                    plan = hd.Plan(L, M, A=A, m=m, kind=kind, dtype=dtype)
                except hd.HdError as e:
                    assert e.name == "HD_ERR_UNSUPPORTED", (L, M, m, e)
                    continue
                got = run_conv(hd, plan, fs)
                check(got, ref, dtype, integer, (kind, dtype, mult, L, M, m, plan.params()))
                plan.close()
                ran += 1
    assert ran > 50


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_auto_parameters(hd, kind, dtype):
    for L in (7, 300, 1024, 3000, 4096):
        M = params.dealias_bound(kind, L) + 3
        fs = make_inputs(kind, L, 2, 2, 7 + L)
        ref = direct.conv1d_batch(fs, kind)
        with hd.Plan(L, M, kind=kind, dtype=dtype) as plan:
            got = run_conv(hd, plan, fs)
            p = plan.params()
            check(got, ref, dtype, False, (kind, dtype, L, p))
            pp, qq, nn = params.derive(kind, L, M, p["m"]) if not (p["p"] == 1 and p["q"] == 1) else (1, 1, 1)
            assert p["q"] * p["m"] >= M and p["p"] * p["m"] >= (L if kind == "complex" else (L + 1) // 2)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_forward_residue_intermediates(hd, kind, dtype):
    """Each residue contribution equals the naive length-qm DFT at k = q l + r
    (Eq. forStan), k = q l + u n + v (Section 6.1) or the centered/Hermitian
    analogues (Eq. centDFT, Eq. forCentIn)."""
    import torch
    L = 37
    f = make_inputs(kind, L, 1, 1, 5)[0][0]
    M = params.dealias_bound(kind, L) + 2
    tol = 2e-6 if dtype == "f32" else 1e-12
    ran = 0
    for m in (4, 8, 16, 32, 64, 128):
        try:
            plan = hd.Plan(L, M, m=m, kind=kind, dtype=dtype)
        except hd.HdError as e:
            assert e.name == "HD_ERR_UNSUPPORTED"
            continue
        pr = plan.params()
        defs = residue.residue_forward(kind, f, L, M, pr["m"], pr["p"], pr["q"])
        fd = to_dev(f, dtype)
        for r, want in enumerate(defs):
            out = torch.zeros(len(want), dtype=fd.dtype, device=fd.device)
            plan.forward_residue(fd, r, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            scale = np.max(np.abs(want)) + 1e-30
            assert np.max(np.abs(got - want)) / scale <= tol, (kind, dtype, m, r)
            ran += 1
        plan.close()
    assert ran > 5


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batched_stride_and_inplace(hd, dtype):
    import torch
    L, M, count, stride = 500, 999, 37, 512
    fs = make_inputs("complex", L, 2, count, 3)
    ref = direct.conv1d_batch(fs, "complex")
    npdt = np.complex64 if dtype == "f32" else np.complex128
    buf = [np.zeros((count, stride), dtype=npdt) for _ in range(2)]
    for a in range(2):
        buf[a][:, :L] = fs[a]
    with hd.Plan(L, M, m=256, kind="complex", dtype=dtype) as plan:
        d = [torch.from_numpy(b).cuda() for b in buf]
        out = torch.full_like(d[0], 7.0)
        plan.convolve_batched(d, out, count, stride)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        check(got[:, :L], ref, dtype, False, "strided")
        assert np.all(got[:, L:] == 7.0)                    # gaps untouched
        plan.convolve_batched(d, d[0], count, stride)       # in place: h = f_0
        torch.cuda.synchronize()
        check(d[0].cpu().numpy()[:, :L], ref, dtype, False, "in place")


def test_edge_cases_and_errors(hd):
    import torch
    # L = 1: the product of two scalars
    f = make_inputs("complex", 1, 2, 1, 9)
    with hd.Plan(1, 1) as plan:
        got = run_conv(hd, plan, f)
        assert rel_l2(got, f[0] * f[1]) < 1e-6
    # count = 0 is a no-op
    with hd.Plan(16, 31) as plan:
        x = torch.zeros(16, dtype=torch.complex64, device="cuda")
        plan.convolve_batched([x, x], x, 0, 16)
    # M below the dealiasing bound
    with pytest.raises(hd.HdError) as e:
        hd.Plan(100, 198)
    assert e.value.name == "HD_ERR_ALIASED"
    with pytest.raises(hd.HdError) as e:
        hd.Plan(100, 149, kind="centered")
    assert e.value.name == "HD_ERR_ALIASED"
    # inconsistent explicit parameters
    for kw in (dict(m=64, p=1, q=4), dict(m=64, p=2, q=3), dict(m=16, p=8, q=12)):
        with pytest.raises(hd.HdError) as e:
            hd.Plan(100, 199, **kw)
        assert e.value.name == "HD_ERR_INVALID", kw
    # batch stride smaller than an instance
    with hd.Plan(16, 31) as plan:
        x = torch.zeros(64, dtype=torch.complex64, device="cuda")
        with pytest.raises(hd.HdError):
            plan.convolve_batched([x, x], x, 2, 8)
    # residue index out of range
    with hd.Plan(16, 31, m=16) as plan:
        x = torch.zeros(64, dtype=torch.complex64, device="cuda")
        with pytest.raises(hd.HdError):
            plan.forward_residue(x, 5, x)


def test_explicit_plan_equals_hybrid(hd):
    """p = q = 1 with m >= M is explicit zero padding (Section 2.1); both
    paddings give the oracle result."""
    L, M = 1000, 1999
    fs = make_inputs("complex", L, 2, 4, 21, integer=True)
    ref = direct.conv1d_batch(fs, "complex")
    for kw in (dict(m=2048, p=1, q=1), dict(m=1024), dict(m=512), dict(m=128, p=8)):
        with hd.Plan(L, M, m=kw["m"], p=kw.get("p", 0), q=kw.get("q", 0), dtype="f64") as plan:
            got = run_conv(hd, plan, fs)
            check(got, ref, "f64", True, kw)


def test_determinism(hd):
    L, M = 4096, 8191
    fs = make_inputs("complex", L, 2, 64, 31)
    with hd.Plan(L, M, m=2048) as plan:
        a = run_conv(hd, plan, fs)
        b = run_conv(hd, plan, fs)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("comp", ["0", "1"])
@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_plain_and_compensated_residue_sums(hd, monkeypatch, kind, comp):
    """Both accumulations of the residue contributions (HD_COMP forces the
    TwoSum or the plain sum; by default TwoSum is used from 8 residues on)
    meet the FP32 bound, with few and with many residues."""
    monkeypatch.setenv("HD_COMP", comp)
    L = 1000
    fs = make_inputs(kind, L, 2, 3, 31)
    ref = direct.conv1d_batch(fs, kind)
    M = params.dealias_bound(kind, L) + 7
    for m in (16, 64, 512):
        try:
            plan = hd.Plan(L, M, m=m, kind=kind)
        except hd.HdError as e:
            assert e.name == "HD_ERR_UNSUPPORTED"
            continue
        with plan:
            check(run_conv(hd, plan, fs), ref, "f32", False, (kind, comp, m, plan.params()))


def test_persistent_bulk_copy_variant_matches_plain_kernel(hd):
    """The persistent kernel (next batch element staged by bulk copies) and the
    plain kernel run the same residue body: their outputs agree to FP32
    rounding and both meet the FP32 bound.  A row that starts off a 16-byte
    boundary (odd element offset) falls back to the plain kernel, whose output
    it reproduces bit for bit."""
    import os
    import subprocess
    import sys
    import torch
    L, M, count = 4096, 8191, 300
    fs = make_inputs("complex", L, 2, count, 21)
    best, cands = hd.autotune(count, reps=1, L=L, M=M)
    pipe = [c for c in cands if c["minb"] == 1 and c["S"] <= 4096]
    assert pipe, cands
    ref = cdirect.conv1d_batch([f[[0, 150, 299]] for f in fs], L, "complex")
    outs = []
    for c in pipe[:2]:
        with hd.Plan(L, M, candidate=c) as plan:
            got = run_conv(hd, plan, fs)
        check(got[[0, 150, 299]], ref, "f32", False, ("pipe", c))
        outs.append(got)
    # the same candidates with the persistent variant switched off, in a fresh process
    code = (
        "import sys, json, numpy as np, torch; sys.path.insert(0, '.');"
        "import inputs, paper_2303_17510_gb300 as hd;"
        f"L, M, count = {L}, {M}, {count};"
        "fs = [inputs.uniform_complex((count, L), 21 + a) for a in range(2)];"
        f"cands = {pipe[:2]!r};"
        "res = [];\n"
        "for c in cands:\n"
        "    p = hd.Plan(L, M, candidate=c); d = [torch.from_numpy(f.astype(np.complex64)).cuda() for f in fs]\n"
        "    o = torch.zeros_like(d[0]); p.convolve_batched(d, o, count, L); torch.cuda.synchronize()\n"
        "    np.save(f'/tmp/hd_plain_{len(res)}.npy', o.cpu().numpy()); res.append(1); p.close()\n"
    )
    env = dict(os.environ, HD_PIPE="0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code], cwd=root, env=env, check=True, timeout=300)
    plains = [np.load(f"/tmp/hd_plain_{i}.npy") for i in range(len(outs))]
    for i, got in enumerate(outs):
        assert rel_l2_rows(got, plains[i]) <= 1e-6, i
    # a misaligned row start (one complex64 past a 16-byte boundary) takes the plain kernel
    buf = [np.zeros((count * L + 1,), dtype=np.complex64) for _ in range(2)]
    for a in range(2):
        buf[a][1:] = fs[a].astype(np.complex64).ravel()
    with hd.Plan(L, M, candidate=pipe[0]) as plan:
        d = [torch.from_numpy(b).cuda() for b in buf]
        out = torch.zeros(count * L + 1, dtype=torch.complex64, device="cuda")
        plan.convolve_batched([x[1:] for x in d], out[1:], count, L)
        torch.cuda.synchronize()
        got = out[1:].cpu().numpy().reshape(count, L)
    assert np.array_equal(got, plains[0])
    assert hd.device_status() == "HD_OK"     # no bounded wait of the persistent kernels ran out


@pytest.mark.parametrize("kind", ["complex", "centered"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_cluster_residue_groups(hd, kind, dtype):
    """D > 1 residues per pass (Section 6.5): one convolution on a cluster of
    D x A CTAs, residue groups reduced through distributed shared memory.
    Every enumerated cluster candidate, both mults; FP64 on integer inputs is
    exact after rint, FP32 within the bound; the sums are deterministic."""
    ran = 0
    for mult, A in (("product", 2), ("sum_pairs3", 3)):
        for L in (5, 100, 1000, 1024, 3000):
            fs = make_inputs(kind, L, A, 3, 500 + L, integer=(dtype == "f64"))
            ref = direct.conv1d_batch(fs, kind, mult)
            M = params.dealias_bound(kind, L, mult) + 1
            for c in hd.enumerate_candidates(L=L, M=M, A=A, kind=kind, dtype=dtype):
                if c["D"] <= 1:
                    continue
                assert c["D"] <= c["n"] and c["D"] * A <= 8
                with hd.Plan(L, M, A=A, kind=kind, dtype=dtype, candidate=c) as plan:
                    got = run_conv(hd, plan, fs)
                    check(got, ref, dtype, dtype == "f64", (kind, dtype, mult, L, c))
                    assert np.array_equal(run_conv(hd, plan, fs), got)
                ran += 1
    assert ran >= 8


def test_cluster_explicit_D_and_refusals(hd):
    """Plans asking for D residue groups directly: the single FP64 convolution
    of L = 1024, M = 2047 with m = 512 (n = 4 residues) at D = 2 and 4; D
    beyond the residue count or the cluster size is refused."""
    L, M = 1024, 2047
    fs = make_inputs("complex", L, 2, 1, 77, integer=True)
    ref = direct.conv1d_batch(fs, "complex")
    for D in (2, 4):
        with hd.Plan(L, M, m=512, D=D, dtype="f64") as plan:
            assert plan.axis_params(0)["D"] == D and plan.axis_params(0)["n"] == 4
            check(run_conv(hd, plan, [f[0] for f in fs]), ref[0], "f64", True, D)
    for kw in (dict(m=512, D=8), dict(m=1024, D=4), dict(m=512, D=4, A=3)):
        A = kw.pop("A", 2)
        with pytest.raises(hd.HdError) as e:
            hd.Plan(L, 3 * L if A == 3 else M, A=A, dtype="f64", **kw)
        assert e.value.name == "HD_ERR_UNSUPPORTED", kw
