"""CPU checks of the C ABI: the library loads, exports every symbol that
include/*.h declares, and its host-only logic (parameter derivation,
dealiasing bounds, argument validation) matches the oracle bit for bit."""
import glob
import os
import re

import pytest

from oracle import params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(hd_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def test_symbols_exported(hd):
    names = _declared_symbols()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(hd.lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_derive_params_matches_oracle(hd, kind):
    for L in list(range(1, 40)) + [64, 100, 1000, 1024, 2048, 4096, 65536]:
        for M in sorted({params.dealias_bound(kind, L), params.dealias_bound(kind, L) + 1, 2 * L, 3 * L + 7}):
            for m in list(range(1, 20)) + [32, 64, 127, 128, 1024, 3072, 4096, 8192]:
                assert hd.derive_params(kind, L, M, m) == params.derive(kind, L, M, m), (kind, L, M, m)


def test_paper_examples_through_abi(hd):
    assert hd.derive_params("complex", 6, 11, 4)[:2] == (2, 3)             # Fig. 1
    assert hd.derive_params("centered", 2048, 3072, 16)[:2] == (128, 192)  # Section 7.2 example


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("mult", ["product", "sum_pairs3", "basdevant2"])
def test_dealias_bound_matches_oracle(hd, kind, mult):
    for L in range(1, 300):
        assert hd.dealias_bound(kind, L, mult) == params.dealias_bound(kind, L, mult)


def test_invalid_arguments(hd):
    with pytest.raises(hd.HdError) as e:
        hd.derive_params("complex", 0, 10, 4)
    assert e.value.name == "HD_ERR_INVALID"
    with pytest.raises(hd.HdError):
        hd.derive_params("complex", 10, 19, 0)
    assert hd.dealias_bound("complex", 0) == -1
    assert hd.lib.hd_status_string(6).decode().startswith("HD_ERR_ALIASED")
    assert hd.lib.hd_plan_destroy(None) == 0


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_enumerated_candidates_are_legal(hd, kind, dtype):
    for L in (1, 7, 100, 1024, 4096):
        for M in (params.dealias_bound(kind, L), 3 * L):
            cands = hd.enumerate_candidates(L=L, M=M, kind=kind, dtype=dtype)
            assert cands, (kind, L, M)
            seen = set()
            for c in cands:
                m, p, q, S, n = c["m"], c["p"], c["q"], c["S"], c["n"]
                assert q * m >= M and S * n == q * m
                if (p, q) != (1, 1):
                    want = params.derive(kind, L, M, m)
                    # the paper's p, or explicit padding to a power-of-two multiple
                    assert p == want[0] or (p > want[0] and p & (p - 1) == 0)
                else:
                    assert m >= M
                key = (S, n, c["E"], c["minb"], c["D"])
                assert key not in seen
                seen.add(key)
            # at least one candidate with the paper's own p for the largest legal m
    with pytest.raises(hd.HdError):
        hd.enumerate_candidates(L=0, M=5)


def test_mult_counts_validated(hd):
    """(A, B) must be the counts of the mult, refused before any device work;
    the two-output mult also runs on the split path (transforms beyond the
    fused kernel)."""
    for A, B, mult in ((3, 2, None), (2, 2, "product"), (3, 1, "basdevant2"), (2, 3, None), (1, 1, "product")):
        with pytest.raises(hd.HdError) as e:
            hd.Plan(100, 199, A=A, B=B, mult=mult)
        assert e.value.name == "HD_ERR_INVALID", (A, B, mult)
    assert any(c["S"] > 4096 for c in hd.enumerate_candidates(L=40000, M=79999, A=2, B=2))
    # the default variant of FP32 two-output plans (E = 8, 255 registers) starts at S = 512;
    # smaller transforms are reachable through enumerated candidates
    with pytest.raises(hd.HdError) as e:
        hd.Plan(300, 450, m=128, A=2, B=2, kind="centered")
    assert e.value.name == "HD_ERR_UNSUPPORTED"
    small = [c for c in hd.enumerate_candidates(L=300, M=450, A=2, B=2, kind="centered") if c["S"] < 512]
    assert small and not any(c["E"] == 8 and c["minb"] == 1 for c in small)
    import ctypes
    out = ctypes.c_void_p()
    assert hd.lib.hd_plan_create(ctypes.byref(out), 100, 199, 3, 2, 0, 0, 0, 0) == 1   # HD_ERR_INVALID
    assert hd.lib.hd_plan_create(ctypes.byref(out), 100, 199, 2, 3, 0, 0, 0, 0) == 1
    assert out.value is None
    cands = hd.enumerate_candidates(L=20000, M=39999, A=2, B=2)
    assert cands and all(c["S"] > 4096 and c["D"] == 1 for c in cands)   # the split path only
    assert hd.enumerate_candidates(L=4096, M=8191, A=2, B=2)


def test_ragged_workload_same_with_library_or_oracle_bounds(hd):
    """The ragged workload takes its dealiasing bounds from the caller: the
    library's hd_dealias_bound and the oracle's definition give the same
    10,000 instances (both are pinned to the paper's bounds elsewhere)."""
    import inputs
    from oracle import params
    a = inputs.ragged_instances(10000, 4, hd.dealias_bound)
    b = inputs.ragged_instances(10000, 4, params.dealias_bound)
    assert a == b
    assert sum(d["clamped"] for d in a) > 0
    assert all(d["M"] >= params.dealias_bound(d["kind"], d["L"]) for d in a)


def test_cluster_candidates_enumerated(hd):
    """D > 1 residues per pass (one convolution on a thread-block cluster of
    D x A CTAs) is offered for complex and centered data with n >= D residues
    and at most 8 CTAs; Hermitian candidates keep D = 2 (residue pairs)."""
    cs = hd.enumerate_candidates(L=1024, M=2047, dtype="f64")
    cl = sorted((c["S"], c["n"], c["D"], c["E"]) for c in cs if c["D"] > 1)
    assert cl == [(512, 4, 2, 2), (512, 4, 2, 4), (512, 4, 2, 8), (512, 4, 4, 2), (512, 4, 4, 4), (512, 4, 4, 8),
                  (1024, 2, 2, 4), (1024, 2, 2, 8)]
    for c in hd.enumerate_candidates(L=1000, M=1500, A=3, kind="centered"):
        assert c["D"] * 3 <= 8 or c["D"] == 1
        assert c["D"] <= c["n"]
    assert all(c["D"] == 2 for c in hd.enumerate_candidates(L=1000, M=1500, kind="hermitian") if c["S"] <= 4096)
    for c in hd.enumerate_candidates(L=20000, M=39999):
        if c["S"] > 4096:
            assert c["D"] == 1                            # no cluster form of the split path


def test_mhd3_counts_and_bounds(hd):
    """The eight-output mult (A = 6, B = 8) has the binary dealiasing bounds,
    is inferred from (A, B) = (6, 8) by hd_plan_create, and is refused with
    other counts before any device work; long inputs take the split path."""
    from oracle import params
    for kind in ("complex", "centered", "hermitian"):
        for L in (1, 100, 257):
            assert hd.dealias_bound(kind, L, "mhd3") == params.dealias_bound(kind, L, "mhd3")
    for A, B in ((3, 8), (6, 5), (6, 1)):
        with pytest.raises(hd.HdError) as e:
            hd.Plan(100, 199, A=A, B=B, mult="mhd3")
        assert e.value.name == "HD_ERR_INVALID", (A, B)
    split = hd.enumerate_candidates(L=20000, M=39999, A=6, B=8)
    assert split and all(c["S"] > 4096 for c in split)
    cands = hd.enumerate_candidates(L=300, M=599, A=6, B=8)
    # fused transforms up to 1024 points (eight residue sums in shared memory), else the split path
    assert cands and all((c["S"] <= 1024 or c["S"] > 4096) and c["D"] <= 1 for c in cands)
    import ctypes
    out = ctypes.c_void_p()
    assert hd.lib.hd_plan_create(ctypes.byref(out), 100, 199, 6, 7, 0, 0, 0, 0) == 1   # HD_ERR_INVALID


def test_basdevant3_counts_and_bounds(hd):
    """The five-output mult (A = 3, B = 5) has the binary dealiasing bounds,
    is inferred from (A, B) = (3, 5), and is refused with other counts before
    any device work; long inputs take the split path."""
    from oracle import params
    for kind in ("complex", "centered", "hermitian"):
        for L in (1, 100, 257):
            assert hd.dealias_bound(kind, L, "basdevant3") == params.dealias_bound(kind, L, "basdevant3")
    for A, B in ((2, 5), (3, 4)):
        with pytest.raises(hd.HdError) as e:
            hd.Plan(100, 199, A=A, B=B, mult="basdevant3")
        assert e.value.name == "HD_ERR_INVALID", (A, B)
    split = hd.enumerate_candidates(L=20000, M=39999, A=3, B=5)
    assert split and all(c["S"] > 4096 for c in split)
    # fused transforms up to 2048 points (five residue sums in shared memory), else the split path
    assert all(c["S"] <= 2048 or c["S"] > 4096 for c in hd.enumerate_candidates(L=3000, M=5999, A=3, B=5))
    import ctypes
    out = ctypes.c_void_p()
    assert hd.lib.hd_plan_create(ctypes.byref(out), 100, 199, 3, 4, 0, 0, 0, 0) == 1   # HD_ERR_INVALID
