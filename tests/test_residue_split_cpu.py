"""Residue-split convolution on the CPU: the oracle's partial sums and the
multi-rank host logic.

The residues of a hybrid-dealiased convolution are independent and their
backward transforms add into the output (Section 2.2), so the sum over
residues r_begin <= r < r_end is a well-defined part of the result: the
inverse padded DFT of the product spectrum restricted to the frequencies
k = r mod n.  The step-by-step oracle's partial sums (steps.convolve with
residues=...) are pinned here against that restricted explicit FFT
convolution -- a second formula -- and against the direct definition after
summing over a partition.  Two gloo ranks then run the sharding host logic
(paper_2303_17510_gb300.sharding) with the oracle as the partial computation.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import inputs
from oracle import direct, explicit, params, steps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sharding():
    # the host logic alone, loaded by path: the package itself loads libhd.so
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_hd_sharding", os.path.join(ROOT, "paper_2303_17510_gb300", "sharding.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod

# (kind, L, M, m): p = 1, 2 and > 2 for each kind
CASES = [
    ("complex", 16, 31, 16), ("complex", 16, 31, 8), ("complex", 24, 47, 4), ("complex", 13, 40, 8),
    ("centered", 16, 24, 8), ("centered", 17, 30, 4), ("centered", 20, 30, 2),
    ("hermitian", 15, 23, 8), ("hermitian", 16, 24, 4), ("hermitian", 21, 40, 2),
]


def _fs(kind, L, seed):
    if kind == "hermitian":
        return [inputs.hermitian_1d(1, L, seed + a)[0] for a in range(2)]
    return [inputs.uniform_complex(L, seed + a) for a in range(2)]


def _partial(kind, fs, L, M, m, r0, r1):
    if kind == "complex":
        return steps.convolve(fs, L, M, m, residues=(r0, r1))
    return steps.convolveX(fs, L, M, m, kind, residues=(r0, r1))


def _explicit_partial(kind, fs, L, M, m, r0, r1, sign=1):
    p, q, n = params.derive(kind, L, M, m)
    N = q * m
    if sign < 0:   # a planted convention slip: numpy's bins taken as the paper's frequencies
        k = np.arange(N)
        spec_keep = (k % n >= r0) & (k % n < r1)
        return _masked_numpy(kind, fs, N, spec_keep)
    return explicit.convnd_explicit(fs, [kind], [N], residues=(n, r0, r1))


def _masked_numpy(kind, fs, N, keep):
    lo = 0
    ex = fs
    if kind == "centered":
        lo = -(len(fs[0]) // 2)
    elif kind == "hermitian":
        ex = [direct.hermitian_expand(f) for f in fs]
        lo = -(len(fs[0]) - 1)
    P = []
    for e in ex:
        x = np.zeros(N, dtype=np.complex128)
        x[np.mod(np.arange(len(e)) + lo, N)] = e
        P.append(np.fft.fft(x))
    y = np.fft.ifft(np.where(keep, P[0] * P[1], 0))
    out_lo = 0 if kind == "hermitian" else lo
    return y[np.mod(np.arange(len(fs[0])) + out_lo, N)]


@pytest.mark.parametrize("kind,L,M,m", CASES)
def test_partial_sums_equal_restricted_explicit(kind, L, M, m):
    fs = _fs(kind, L, 31)
    p, q, n = params.derive(kind, L, M, m)
    ranges = [(0, n), (0, 1), (n - 1, n)] + [(r, min(n, r + 2)) for r in range(1, n)]
    for r0, r1 in ranges:
        got = _partial(kind, fs, L, M, m, r0, r1)
        want = _explicit_partial(kind, fs, L, M, m, r0, r1)
        assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want))), (r0, r1)


@pytest.mark.parametrize("kind,L,M,m", CASES)
def test_partition_sums_to_definition(kind, L, M, m):
    fs = _fs(kind, L, 47)
    p, q, n = params.derive(kind, L, M, m)
    ref = direct.conv1d(fs, kind)
    rng = np.random.default_rng(n * 1000 + L)
    cuts = sorted(set([0, n] + list(rng.integers(0, n + 1, size=3))))
    total = sum(_partial(kind, fs, L, M, m, a, b) for a, b in zip(cuts[:-1], cuts[1:]))
    assert np.max(np.abs(total - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_planted_frequency_convention_slip_fails():
    # with n >= 3 the residue classes of k and -k differ, so reading numpy's
    # bins as the paper's frequencies selects other residues and is caught
    kind, L, M, m = "complex", 16, 31, 8
    fs = _fs(kind, L, 5)
    p, q, n = params.derive(kind, L, M, m)
    assert n >= 3
    got = _partial(kind, fs, L, M, m, 1, 2)
    good = _explicit_partial(kind, fs, L, M, m, 1, 2)
    bad = _explicit_partial(kind, fs, L, M, m, 1, 2, sign=-1)
    assert np.max(np.abs(got - good)) < 1e-12
    assert np.max(np.abs(got - bad)) > 1e-3


def test_residue_share_partitions():
    sharding = _sharding()
    for n in range(0, 40):
        for world in range(1, 12):
            rs = [sharding.residue_share(n, k, world) for k in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (a0, a1), (b0, b1) in zip(rs[:-1], rs[1:]):
                assert a1 == b0 and a0 <= a1
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.residue_share(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    sharding = _sharding()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for kind, L, M, m in (("complex", 24, 47, 4), ("centered", 17, 30, 4), ("hermitian", 21, 40, 2)):
        fs = _fs(kind, L, 71)            # every rank holds the whole input
        n = params.derive(kind, L, M, m)[2]
        seen = []

        def partial(r0, r1, out):
            seen.append((r0, r1))
            out.copy_(torch.from_numpy(_partial(kind, fs, L, M, m, r0, r1)))

        out = torch.zeros(len(fs[0]), dtype=torch.complex128)
        sharding.reduce_partials(partial, n, out)
        out2 = torch.zeros(len(fs[0]) + (len(fs[0]) % world), dtype=torch.complex128)

        def partial2(r0, r1, o):
            o.zero_()
            o[:len(fs[0])] = torch.from_numpy(_partial(kind, fs, L, M, m, r0, r1))

        part = sharding.reduce_partials(partial2, n, out2, mode="reduce_scatter")
        res[kind] = (seen[0], out.numpy(), part.numpy())
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([res], dtype=object), allow_pickle=True)


@pytest.mark.timeout(180)
def test_two_gloo_ranks_residue_sharding(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"rank{r}.npy", allow_pickle=True)[0] for r in range(world)]
    for kind, L, M, m in (("complex", 24, 47, 4), ("centered", 17, 30, 4), ("hermitian", 21, 40, 2)):
        fs = _fs(kind, L, 71)
        ref = direct.conv1d(fs, kind)
        n = params.derive(kind, L, M, m)[2]
        ranges = [res[r][kind][0] for r in range(world)]
        assert ranges == [(0, n // 2 + n % 2), (n // 2 + n % 2, n)]      # each rank its own residues
        for r in range(world):
            assert np.max(np.abs(res[r][kind][1] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
        padded = np.concatenate([ref, np.zeros(len(ref) % world)])
        sl = len(padded) // world
        for r in range(world):
            assert np.max(np.abs(res[r][kind][2] - padded[r * sl:(r + 1) * sl])) < 1e-12 * max(1.0, np.max(np.abs(ref)))


class _OraclePlan:
    """Stand-in for a plan on the CPU: convolve_residues computes the oracle's
    partial sums (steps.convolve / convolveX over a residue range), so the
    sharding glue can run with gloo ranks and no GPU."""

    def __init__(self, kind, L, M, m, mult):
        self.kind, self.L, self.M, self.m, self.mult = kind, L, M, m, mult
        self.residues = params.derive(kind, L, M, m)[2]

    def convolve_residues(self, fs, h, r0, r1, count=1, batch_stride=0, stream=None):
        import torch
        f = [x.numpy() for x in fs]
        if self.kind == "complex":
            y = steps.convolve(f, self.L, self.M, self.m, self.mult, residues=(r0, r1))
        else:
            y = steps.convolveX(f, self.L, self.M, self.m, self.kind, self.mult, residues=(r0, r1))
        if isinstance(h, (list, tuple)):
            for b, t in enumerate(h):
                t.copy_(torch.from_numpy(y[b]))
        else:
            h.copy_(torch.from_numpy(y))


def _rank_main_sharded(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    sharding = _sharding()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for kind, L, M, m, mult in (("complex", 16, 31, 8, "product"), ("centered", 17, 30, 4, "basdevant2"),
                                ("complex", 13, 40, 8, "mhd3")):
        A = direct.MULTS[mult]
        fs = [torch.from_numpy(inputs.uniform_complex(L, 900 + a)) for a in range(A)]
        plan = _OraclePlan(kind, L, M, m, mult)
        B = direct.OUTPUTS[mult]
        if B == 1:
            h = torch.zeros(L, dtype=torch.complex128)
            sharding.convolve_sharded(plan, fs, h)
            res[mult] = h.numpy()
        else:
            hs = [torch.zeros(L, dtype=torch.complex128) for _ in range(B)]
            sharding.convolve_sharded(plan, fs, hs)
            res[mult] = np.stack([t.numpy() for t in hs])
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"s{rank}.npy"), np.array([res], dtype=object), allow_pickle=True)


@pytest.mark.timeout(180)
def test_two_gloo_ranks_convolve_sharded_single_and_multi_output(tmp_path):
    """sharding.convolve_sharded over two gloo ranks with the oracle standing in
    for the plan: one output (reduced in place) and the two- and eight-output
    mults (each output all-reduced) give the whole convolution on every rank."""
    world = 2
    mp.start_processes(_rank_main_sharded, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"s{r}.npy", allow_pickle=True)[0] for r in range(world)]
    for kind, L, mult in (("complex", 16, "product"), ("centered", 17, "basdevant2"), ("complex", 13, "mhd3")):
        A = direct.MULTS[mult]
        ref = direct.conv1d([inputs.uniform_complex(L, 900 + a) for a in range(A)], kind, mult)
        for r in range(world):
            assert np.max(np.abs(res[r][mult] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), (mult, r)
