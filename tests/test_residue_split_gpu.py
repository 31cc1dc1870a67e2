"""GPU parity of hd_convolve_residues: partial sums over residue ranges.

Residues are independent and their backward transforms add into the output
(Section 2.2), so the partial sum over residues r_begin <= r < r_end of the
outermost axis is the inverse padded DFT of the product spectrum restricted to
the frequencies k = r mod n on that axis.  Each partial is checked against that
restricted FP64 explicit FFT convolution (oracle/explicit.py, pinned on the CPU
against the step-by-step oracle and the direct sum), and the partials of a
partition against the whole convolution (hd_convolve_batched) and the oracle.
Paths: the fused kernel (plain and persistent), Hermitian residue pairs that
start at an odd residue, the cluster variant, the split path, 2D plans; FP32
rel-L2 <= 1e-5 per instance, FP64 integer inputs exact after rint of the sum.
"""
import numpy as np
import pytest

import inputs
from oracle import cdirect, direct, explicit, params
from tests.gpu_util import rel_l2, rel_l2_rows, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def _inputs(kind, L, count, seed, integer=False):
    if kind == "hermitian":
        return [inputs.hermitian_1d(count, L, seed + a, integer=integer) for a in range(2)]
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    return [gen((count, L), seed + a) for a in range(2)]


def _partial_dev(plan, d, r0, r1, count, stride):
    import torch
    out = torch.full_like(d[0], complex(7.0, -3.0))      # stale values must be overwritten
    plan.convolve_residues(d, out, r0, r1, count, stride)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _restricted(kind, fs_rows, N, n, r0, r1):
    return np.stack([explicit.convnd_explicit([f[i] for f in fs_rows], [kind], [N], residues=(n, r0, r1))
                     for i in range(fs_rows[0].shape[0])])


def _ranges(n):
    out = {(0, n), (0, 1), (n - 1, n), (n // 2, n)}
    out |= {(r, min(n, r + 2)) for r in range(1, n, 2)}
    return sorted(out)


CASES = [   # (kind, L, M, m, count): p = 1, 2, > 2; counts that take the persistent kernel
    ("complex", 1000, 1999, 1024, 5), ("complex", 1000, 1999, 256, 5), ("complex", 4096, 8191, 4096, 300),
    ("centered", 300, 450, 128, 5), ("centered", 4096, 6144, 2048, 300), ("centered", 777, 1200, 64, 3),
    ("hermitian", 257, 385, 64, 5), ("hermitian", 1000, 1500, 128, 4), ("hermitian", 301, 460, 32, 3),
]


@pytest.mark.parametrize("kind,L,M,m,count", CASES)
def test_partials_match_restricted_oracle_f32(hd, kind, L, M, m, count):
    import torch
    fs = _inputs(kind, L, count, 900 + L)
    Ls = fs[0].shape[1]
    rows = [0, count - 1] if count > 2 else list(range(count))
    with hd.Plan(L, M, m=m, kind=kind) as plan:
        ax = plan.axis_params(0)
        n, N = ax["n"], ax["q"] * ax["m"]
        d = [to_dev(f, "f32") for f in fs]
        whole = torch.zeros_like(d[0])
        plan.convolve_batched(d, whole, count, Ls)
        full = _partial_dev(plan, d, 0, n, count, Ls)
        assert np.array_equal(full, whole.cpu().numpy())             # the whole range is the convolution
        for r0, r1 in _ranges(n):
            got = _partial_dev(plan, d, r0, r1, count, Ls)
            want = _restricted(kind, [f[rows] for f in fs], N, n, r0, r1)
            e = rel_l2_rows(got[rows], want)
            assert e <= 1e-5, (r0, r1, e)
        # a partition of [0, n) sums to the oracle's convolution
        cuts = sorted({0, n, n // 3, (2 * n) // 3})
        total = sum(_partial_dev(plan, d, a, b, count, Ls).astype(np.complex128) for a, b in zip(cuts[:-1], cuts[1:]))
        ref = cdirect.conv1d_batch([f[rows] for f in fs], L, kind)
        assert rel_l2_rows(total[rows], ref) <= 1e-5
        # empty range: zeros
        assert not np.any(_partial_dev(plan, d, 1, 1, count, Ls))


@pytest.mark.parametrize("kind,m", [("complex", 512), ("complex", 128), ("centered", 64), ("hermitian", 64)])
def test_partition_f64_integer_exact(hd, kind, m):
    L = 1000
    M = params.dealias_bound(kind, L) + 5
    fs = _inputs(kind, L, 3, 40, integer=True)
    ref = direct.conv1d_batch(fs, kind)
    with hd.Plan(L, M, m=m, kind=kind, dtype="f64") as plan:
        n = plan.residues
        assert n >= 2
        d = [to_dev(f, "f64") for f in fs]
        Ls = fs[0].shape[1]
        for cuts in ([0, 1, n], [0, n // 2, n // 2 + 1, n], list(range(n + 1))):
            total = sum(_partial_dev(plan, d, a, b, 3, Ls) for a, b in zip(cuts[:-1], cuts[1:]))
            assert np.array_equal(np.rint(total.real) + 1j * np.rint(total.imag), ref), cuts


def test_cluster_variant_partials(hd):
    """The cluster variant (D residue groups on one cluster) over residue ranges."""
    L, M = 1024, 2047
    fs = _inputs("complex", L, 1, 77, integer=True)
    ref = direct.conv1d_batch(fs, "complex")
    for D in (2, 4):
        with hd.Plan(L, M, m=512, D=D, dtype="f64") as plan:
            n = plan.residues
            assert n == 4 and plan.axis_params(0)["D"] == D
            N = plan.axis_params(0)["q"] * 512
            d = [to_dev(f[0], "f64") for f in fs]
            parts = []
            for a, b in ((0, 1), (1, n - 2), (n - 2, n)):
                got = _partial_dev(plan, d, a, b, 1, L)
                want = explicit.convnd_explicit([f[0] for f in fs], ["complex"], [N], residues=(n, a, b))
                assert rel_l2(got, want) <= 1e-12, (D, a, b)
                parts.append(got)
            tot = sum(parts)
            assert np.array_equal(np.rint(tot.real) + 1j * np.rint(tot.imag), ref[0])


@pytest.mark.parametrize("kind,L", [("complex", 9000), ("centered", 20000)])
def test_split_path_partials(hd, kind, L):
    M = params.dealias_bound(kind, L) + 11
    fs = _inputs(kind, L, 2, 300 + L)
    cands = [c for c in hd.enumerate_candidates(L=L, M=M, kind=kind) if c["S"] > 4096]
    assert cands
    c = cands[0]
    with hd.Plan(L, M, kind=kind, candidate=c) as plan:
        n = plan.residues
        N = c["q"] * c["m"]
        d = [to_dev(f, "f32") for f in fs]
        ref = cdirect.conv1d_batch(fs, L, kind)
        cuts = sorted({0, n // 2, n})
        tot = 0
        for a, b in zip(cuts[:-1], cuts[1:]):
            got = _partial_dev(plan, d, a, b, 2, L)
            want = _restricted(kind, fs, N, n, a, b)
            assert rel_l2_rows(got, want) <= 1e-5, (a, b)
            tot = tot + got.astype(np.complex128)
        assert rel_l2_rows(tot, ref) <= 1e-5


def test_2d_partials_along_outer_axis(hd):
    Ls = (31, 33)
    Ms = [params.dealias_bound("complex", L) + 1 for L in Ls]
    fs = [inputs.uniform_complex(Ls, 12 + a) for a in range(2)]
    ref = direct.convnd(fs, ("complex", "complex"))
    with hd.Plan(list(Ls), Ms) as plan:
        ax0, ax1 = plan.axis_params(0), plan.axis_params(1)
        n = ax0["n"]
        Ns = [ax0["q"] * ax0["m"], ax1["q"] * ax1["m"]]
        d = [to_dev(f.reshape(-1), "f32") for f in fs]
        tot = 0
        for a, b in zip([0, n // 2], [n // 2, n]):
            got = _partial_dev(plan, d, a, b, 1, 0).reshape(Ls)
            want = explicit.convnd_explicit(fs, ["complex", "complex"], Ns, residues=(n, a, b))
            assert rel_l2(got, want) <= 1e-5, (a, b)
            tot = tot + got.astype(np.complex128)
        assert rel_l2(tot, ref) <= 1e-5


def test_refusals(hd):
    import torch
    L, M = 100, 199
    with hd.Plan(L, M, m=32) as plan:
        n = plan.residues
        d = [to_dev(inputs.uniform_complex(L, s), "f32") for s in (1, 2)]
        out = torch.zeros_like(d[0])
        for a, b in ((-1, 1), (2, 1), (0, n + 1)):
            with pytest.raises(hd.HdError) as e:
                plan.convolve_residues(d, out, a, b)
            assert e.value.name == "HD_ERR_INVALID"
        with pytest.raises(hd.HdError) as e:            # a proper part cannot write over its inputs
            plan.convolve_residues(d, d[0], 0, 1)
        assert e.value.name == "HD_ERR_INVALID"


def test_sharded_convolve_one_rank(hd):
    """The sharding glue on one GPU: a world of one rank takes every residue and
    the all-reduce (NCCL) leaves the convolution."""
    import os
    import socket
    import torch
    import torch.distributed as dist
    from paper_2303_17510_gb300 import sharding
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        L, M = 1000, 1999
        fs = _inputs("complex", L, 1, 5)
        with hd.Plan(L, M, m=256) as plan:
            d = [to_dev(f[0], "f32") for f in fs]
            h = torch.zeros_like(d[0])
            sharding.convolve_sharded(plan, d, h)
            torch.cuda.synchronize()
            ref = cdirect.conv1d_batch(fs, L, "complex")[0]
            assert rel_l2(h.cpu().numpy(), ref) <= 1e-5
    finally:
        dist.destroy_process_group()
