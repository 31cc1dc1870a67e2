"""Parameter derivation, dealiasing bounds and work-memory formulas.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Given the FFT size m, the paper derives the explicit padding factor p and the
implicit padding factor q (Eq. pqdef1, Section 2.1), then, per Alg. convolve
(Section 2.2) and the inner-loop redefinition (Section 6.1):
    p = ceil(L/m);   p <= 2: n = q = ceil(M/m)
                     p  > 2: n = ceil(M/(p m)), q = n p
and per Alg. convolveX (Section 3/4) with Section 6.2 for centered and
Hermitian data:
    p = 2 ceil(L/(2m)) (even);  n = ceil(2M/(p m)),  q = n p / 2.
n is the number of residue contributions the convolution loop visits.  An
explicit plan (m >= M, p = q = n = 1) is legal for every kind (Section 7, the
optimizer example at L = 2048).
"""
from __future__ import annotations


def ceil_div(a: int, b: int) -> int:
    return -(-int(a) // int(b))


def derive(kind: str, L: int, M: int, m: int):
    """Return (p, q, n) for the given kind, length L, dealiased length M and FFT size m."""
    if m <= 0 or L <= 0 or M <= 0:
        raise ValueError("L, M and m must be positive")
    if kind == "complex":
        p = ceil_div(L, m)
        if p <= 2:
            n = ceil_div(M, m)
            q = n
        else:
            n = ceil_div(M, p * m)
            q = n * p
        return p, q, n
    if kind in ("centered", "hermitian"):
        p = 2 * ceil_div(L, 2 * m)
        n = ceil_div(2 * M, p * m)
        q = n * p // 2
        return p, q, n
    raise ValueError(kind)


def explicit(L: int, M: int, m: int):
    """Explicit zero padding as a hybrid plan: legal when m >= M."""
    if m < M:
        raise ValueError("explicit padding needs m >= M")
    return 1, 1, 1


def dealias_bound(kind: str, L: int, mult: str = "product") -> int:
    """Smallest M for which the returned L outputs carry no aliases.

    complex:   2L-1 (Section 2: M = sum L_i - (A-1) for a binary product; the
               sum of pairwise products, and the Basdevant and MHD outputs,
               which are signed sums of binary products, have the same bound).
    centered:  L + floor(L/2): outputs c in [-H, L-H-1] with H = floor(L/2)
               receive no wrapped term when M >= L + H.
    hermitian: the centered bound of the odd expanded length 2 ceil(L/2) - 1.
    """
    if mult not in ("product", "sum_pairs3", "basdevant2", "basdevant3", "mhd3"):
        raise ValueError(mult)
    if kind == "complex":
        return 2 * L - 1
    if kind == "centered":
        return L + L // 2
    if kind == "hermitian":
        Le = 2 * ((L + 1) // 2) - 1
        return Le + Le // 2
    raise ValueError(kind)


def work_memory_words(A: int, B: int, p: int, m: int, L: int, d: int) -> int:
    """Hybrid work memory (A+B) p m L^(d-1) complex words (Section 5, memory)."""
    return (A + B) * p * m * L ** (d - 1)


def explicit_memory_words(A: int, B: int, p: int, q: int, L: int, d: int) -> float:
    """Explicit padding buffer E = C (q/p)^d L^d with C = max(A, B) (Section 5)."""
    return max(A, B) * (q / p) ** d * L ** d
