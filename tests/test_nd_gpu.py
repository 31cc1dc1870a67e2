"""GPU parity of multidimensional convolutions (Section 5 decomposition:
outer-axis residue transforms, inner sub-convolutions, inverse outer
transforms) against the FP64 direct N-D oracle."""
import itertools

import numpy as np
import pytest

import inputs
from oracle import direct, params
from tests.gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def run_nd(hd, plan, fs, dtype):
    import torch
    d = [to_dev(f, dtype) for f in fs]
    out = torch.zeros_like(d[0])
    plan.convolve(d, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def axis_kinds(kind, nd):
    outer = "complex" if kind == "complex" else "centered"
    return tuple([outer] * (nd - 1) + [kind])


def bounds(kind, shape_L, mult="product"):
    ks = axis_kinds(kind, len(shape_L))
    return [params.dealias_bound(k, L, mult) for k, L in zip(ks, shape_L)]


def make_nd(kind, Ls, A, seed, integer=False):
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    return [gen(tuple(Ls), seed + a) for a in range(A)]


@pytest.mark.parametrize("kind", ["complex", "centered"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("Ls", [(5, 7), (16, 12), (31, 33), (6, 5, 7)])
def test_nd_small_matches_oracle(hd, kind, dtype, Ls):
    fs = make_nd(kind, Ls, 2, 10 + sum(Ls), integer=(dtype == "f64"))
    ref = direct.convnd(fs, axis_kinds(kind, len(Ls)))
    Ms = [b + 1 for b in bounds(kind, Ls)]
    with hd.Plan(list(Ls), Ms, kind=kind, dtype=dtype) as plan:
        got = run_nd(hd, plan, fs, dtype)
    if dtype == "f64":
        assert np.array_equal(np.rint(got.real) + 1j * np.rint(got.imag), ref)
    else:
        assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_nd_hermitian_small(hd, dtype):
    L = 12
    fs = [inputs.hermitian_3d(L, 40 + a, dtype=np.complex128) for a in range(2)]
    ref = direct.convnd(fs, ("centered", "centered", "hermitian"))
    Ms = [b + 2 for b in bounds("hermitian", (L, L, L))]
    with hd.Plan([L, L, L], Ms, kind="hermitian", dtype=dtype) as plan:
        got = run_nd(hd, plan, fs, dtype)
    assert rel_l2(got, ref) <= (1e-5 if dtype == "f32" else 1e-12)


def test_nd_sum_pairs3_and_explicit_parameters(hd):
    Ls = (20, 24)
    fs = make_nd("complex", Ls, 3, 77)
    ref = direct.convnd(fs, ("complex", "complex"), "sum_pairs3")
    Ms = bounds("complex", Ls, "sum_pairs3")
    # every legal m of the outer axis, with residues one at a time (D = 1) or all at once
    for mx in (4, 8, 16, 32, 64):
        for D in (0, 1):
            try:
                plan = hd.Plan(list(Ls), Ms, A=3, m=[mx, 0], D=[D, 0])
            except hd.HdError as e:
                assert e.name == "HD_ERR_UNSUPPORTED"
                continue
            with plan:
                got = run_nd(hd, plan, fs, "f32")
                assert rel_l2(got, ref) <= 1e-5, (mx, D, plan.axis_params(0))


def test_2d_full_size_sampled(hd):
    """2048 x 2048 complex, M = 4095 per axis, spectrum (1+|k|)^-1 (the 2D workload)."""
    L = 2048
    fs = [inputs.spectral_2d(L, L, 3 + a, dtype=np.complex64) for a in range(2)]
    with hd.Plan([L, L], [2 * L - 1, 2 * L - 1]) as plan:
        got = run_nd(hd, plan, fs, "f32")
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, L, 48), rng.integers(0, L, 48)], axis=1)
    pts = np.concatenate([pts, [[0, 0], [L - 1, L - 1], [0, L - 1], [L - 1, 0]]])
    want = direct.convnd_points([f.astype(np.complex128) for f in fs], ("complex", "complex"), pts)
    assert rel_l2(got[tuple(pts.T)], want) <= 1e-5


def test_3d_hermitian_full_size_sampled(hd):
    """256^3 centered Hermitian (128 stored on the last axis), M = 384 per axis."""
    L = 256
    fs = [inputs.hermitian_3d(L, 5 + a, dtype=np.complex64) for a in range(2)]
    with hd.Plan([L, L, L], [384, 384, 384], kind="hermitian") as plan:
        got = run_nd(hd, plan, fs, "f32")
    rng = np.random.default_rng(1)
    H = L // 2
    pts = np.stack([rng.integers(0, L, 24), rng.integers(0, L, 24), rng.integers(0, H, 24)], axis=1)
    pts = np.concatenate([pts, [[L // 2, L // 2, 0], [0, 0, 0], [L - 1, L - 1, H - 1]]])
    want = direct.convnd_points([f.astype(np.complex128) for f in fs], ("centered", "centered", "hermitian"), pts)
    assert rel_l2(got[tuple(pts.T)], want) <= 1e-5
