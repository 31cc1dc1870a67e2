"""Pins of the parameter derivation and dealiasing bounds (oracle/params.py)."""
import os

import numpy as np
import pytest

import inputs
from oracle import direct, explicit, params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "params_examples.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        kind, L, M, m, p, q = line.split()
        rows.append((kind, int(L), int(M), int(m), int(p), int(q)))
    return rows


@pytest.mark.parametrize("row", _golden())
def test_paper_examples(row):
    kind, L, M, m, p, q = row
    gp, gq, n = params.derive(kind, L, M, m)
    assert (gp, gq) == (p, q)


def test_explicit_plan_example():
    # Section 7.2: y direction explicit m = 3072, p = q = 1 for M = 3072
    assert params.explicit(2048, 3072, 3072) == (1, 1, 1)
    with pytest.raises(ValueError):
        params.explicit(2048, 3072, 2048)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_derivation_invariants(kind):
    for L in range(1, 70, 3):
        for M in range(L, 3 * L + 3, 5):
            for m in list(range(1, 40)) + [64, 100, 128, 3 * L]:
                p, q, n = params.derive(kind, L, M, m)
                assert p * m >= L
                assert q * m >= M
                if kind == "complex":
                    assert p == -(-L // m)
                    if p > 2:
                        assert q % p == 0 and n == q // p
                    else:
                        assert n == q
                    # q is the smallest admissible value of its family
                    if p <= 2:
                        assert (q - 1) * m < M
                    else:
                        assert (n - 1) * p * m < M
                else:
                    assert p % 2 == 0 and p * m // 2 >= (L + 1) // 2
                    assert q * 2 == n * p and (n - 1) * p * m < 2 * M


def _smallest_dealiasing_N(kind, L, mult="product"):
    """Exhaustive search: the smallest explicit padding length that reproduces
    the direct convolution."""
    A = 2 if mult == "product" else 3
    if kind == "hermitian":
        fs = [inputs.hermitian_1d(1, L, 70 + a)[0] for a in range(A)]
    else:
        fs = [inputs.uniform_complex(L, 70 + a) for a in range(A)]
    ref = direct.conv1d(fs, kind, mult)
    for N in range(1, 4 * L + 4):
        got = explicit.convnd_explicit(fs, (kind,), [N], mult)
        if np.allclose(got, ref, atol=1e-10):
            # every larger N must work too
            for N2 in range(N, N + 4):
                assert np.allclose(explicit.convnd_explicit(fs, (kind,), [N2], mult), ref, atol=1e-10)
            return N
    raise AssertionError("no dealiasing length found")


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_dealias_bound_is_tight(kind):
    for L in range(2, 26):
        assert _smallest_dealiasing_N(kind, L) == params.dealias_bound(kind, L), L


def test_dealias_bound_sum_pairs3():
    for L in (3, 8, 13):
        assert _smallest_dealiasing_N("complex", L, "sum_pairs3") == params.dealias_bound("complex", L, "sum_pairs3")


def test_work_memory_ratios():
    # Section 5: 1D, A=2, B=1, p/q = 1/2, m = L -> hybrid needs 3/4 of explicit;
    # d dimensions -> 3E/2^(d+1); 2/3 padding -> (2/3)^(d-1) E.
    L = 1024
    for d in (1, 2, 3):
        hyb = params.work_memory_words(2, 1, 1, L, L, d)
        E = params.explicit_memory_words(2, 1, 1, 2, L, d)
        assert hyb / E == pytest.approx(3 / 2 ** (d + 1))
        E23 = params.explicit_memory_words(2, 1, 2, 3, L, d)
        assert hyb / E23 == pytest.approx((2 / 3) ** (d - 1))
    assert params.work_memory_words(2, 1, 1, L, L, 1) / params.explicit_memory_words(2, 1, 1, 2, L, 1) == 0.75
