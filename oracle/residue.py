"""Per-residue forward transforms by their definition (naive FP64 DFT sums).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

zeta_N = exp(2 pi i / N) (Section 2).  The padded transform of an input
zero padded to length qm is F_k = sum_j zeta_{qm}^{k j} f_j (Section 2, with a
positive exponent); for centered data the sum runs over the centered indices
(Eq. centDFT); for Hermitian data over the expanded symmetric array, and F_k
is then real (Section 4).

Residue contributions, in the order the paper's transforms return them:
  p <= 2 (complex) or p = 2 (centered/Hermitian): residue r < q returns
       F_r[l] = F_{q l + r},            l < m          (Eq. forStan, Eq. forCent)
  p  > 2 (complex):  residue v < n returns
       F_v[u m + l] = F_{q l + u n + v},  u < p,  l < m  (Section 6.1)
  p  > 2 (centered/Hermitian): residue v < n returns
       F_v[u m + l] = F_{q l + u n + v},  u < p/2, l < m (Eq. forCentIn)
"""
from __future__ import annotations

import numpy as np

from .direct import hermitian_expand
from .params import derive


def padded_dft(values: np.ndarray, offsets: np.ndarray, N: int, ks: np.ndarray) -> np.ndarray:
    """F_k = sum_j zeta_N^{k c_j} v_j for the listed k, with exact integer reduction of k c_j mod N."""
    values = np.asarray(values, dtype=np.complex128)
    offsets = np.asarray(offsets, dtype=np.int64)
    ks = np.asarray(ks, dtype=np.int64)
    e = np.mod(np.outer(ks, offsets), N)
    return np.exp(2j * np.pi * e / N) @ values


def _index_and_values(kind: str, f: np.ndarray):
    f = np.asarray(f, dtype=np.complex128)
    if kind == "complex":
        return np.arange(f.shape[-1]), f
    if kind == "centered":
        L = f.shape[-1]
        return np.arange(L) - L // 2, f
    if kind == "hermitian":
        e = hermitian_expand(f)
        H = f.shape[-1]
        return np.arange(2 * H - 1) - (H - 1), e
    raise ValueError(kind)


def residue_order(kind: str, m: int, p: int, q: int, n: int):
    """List over residues of the frequency indices k each residue returns, in order."""
    out = []
    if kind == "complex":
        if p <= 2:
            for r in range(q):
                out.append(np.array([q * l + r for l in range(m)], dtype=np.int64))
        else:
            for v in range(n):
                out.append(np.array([q * l + u * n + v for u in range(p) for l in range(m)], dtype=np.int64))
        return out
    ph = p // 2
    if p == 2:
        for r in range(q):
            out.append(np.array([q * l + r for l in range(m)], dtype=np.int64))
    else:
        for v in range(n):
            out.append(np.array([q * l + u * n + v for u in range(ph) for l in range(m)], dtype=np.int64))
    return out


def residue_forward(kind: str, f: np.ndarray, L: int, M: int, m: int, p=None, q=None):
    """All residue contributions of one input, as a list of arrays (see module doc)."""
    if p is None:
        p, q, n = derive(kind, L, M, m)
    else:
        n = q if (kind == "complex" and p <= 2) or (kind != "complex" and p == 2) else (
            q // p if kind == "complex" else q // (p // 2))
    idx, vals = _index_and_values(kind, f)
    N = q * m
    return [padded_dft(vals, idx, N, ks) for ks in residue_order(kind, m, p, q, n)]
