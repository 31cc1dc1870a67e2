"""Seeded synthetic input generators.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It draws random numbers and lays them out in the shapes and value
distributions of the convolution workloads; it contains none of the
convolution arithmetic (no dealiasing, no residue transforms, no products).

Layouts (all arrays are numpy, C order):
  * 1D complex / centered input: ``(count, L)`` complex array.  For the
    centered kind, stored index ``j`` holds centered index ``j - L//2``.
  * 1D Hermitian input: ``(count, ceil(L/2))`` complex array holding the
    non-negative indices ``0 .. ceil(L/2)-1``; index 0 is real.
  * 2D complex input: ``(Lx, Ly)``.
  * 3D centered/Hermitian input: ``(Lx, Ly, ceil(Lz/2))``; x and y are
    centered (stored ``j`` <-> centered ``j - L//2``), z holds the
    non-negative half.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "uniform_complex",
    "integer_complex",
    "hermitian_1d",
    "spectral_2d",
    "hermitian_3d",
    "ragged_instances",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def uniform_complex(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """Real and imaginary parts i.i.d. uniform on [-1, 1]."""
    g = _rng(seed)
    re = g.uniform(-1.0, 1.0, size=shape)
    im = g.uniform(-1.0, 1.0, size=shape)
    return (re + 1j * im).astype(dtype)


def integer_complex(shape, seed: int, lo: int = -8, hi: int = 8, dtype=np.complex128) -> np.ndarray:
    """Real and imaginary parts i.i.d. uniform on the integers lo..hi."""
    g = _rng(seed)
    re = g.integers(lo, hi + 1, size=shape)
    im = g.integers(lo, hi + 1, size=shape)
    return (re + 1j * im).astype(dtype)


def hermitian_1d(count: int, L: int, seed: int, dtype=np.complex128, integer: bool = False) -> np.ndarray:
    """Stored non-negative half (ceil(L/2) values) of a Hermitian array; index 0 real."""
    H = (L + 1) // 2
    if integer:
        f = integer_complex((count, H), seed, dtype=dtype)
    else:
        f = uniform_complex((count, H), seed, dtype=dtype)
    f[:, 0] = f[:, 0].real
    return f


def spectral_2d(Lx: int, Ly: int, seed: int, alpha: float = 1.0, dtype=np.complex64) -> np.ndarray:
    """Complex field with amplitude (1+|k|)^-alpha times (u+iv), u,v ~ U[-1,1].

    |k| is the Euclidean norm of the (uncentered) array index (i, j).
    """
    g = _rng(seed)
    u = g.uniform(-1.0, 1.0, size=(Lx, Ly))
    v = g.uniform(-1.0, 1.0, size=(Lx, Ly))
    i = np.arange(Lx, dtype=np.float64)[:, None]
    j = np.arange(Ly, dtype=np.float64)[None, :]
    amp = (1.0 + np.sqrt(i * i + j * j)) ** (-alpha)
    return (amp * (u + 1j * v)).astype(dtype)


def hermitian_2d(L: int, seed: int, alpha: float = 5.0 / 3.0, dtype=np.complex64) -> np.ndarray:
    """Stored half of a 2D Hermitian-symmetric field, centered in x (the
    spectrum of a real field, e.g. one velocity component of a 2D flow).

    A seeded real field of odd size (2*ceil(L/2)-1)^2 through a real-to-complex
    FFT, scaled by |k|^-alpha (k = 0 scaled by 1), then made exactly symmetric
    on the y = 0 column: f(-x, 0) = conj f(x, 0) with f(0, 0) real.  For even
    L the centered index -L/2 is zero.  Returns shape (L, ceil(L/2)).
    """
    g = _rng(seed)
    H = (L + 1) // 2
    n = 2 * H - 1
    spec = np.fft.rfft2(g.standard_normal((n, n)))   # (n, H): uncentered kx, ky = 0..H-1
    kx = np.fft.fftfreq(n, d=1.0 / n)
    kk = np.sqrt(kx[:, None] ** 2 + np.arange(H, dtype=np.float64)[None, :] ** 2)
    kk[0, 0] = 1.0
    spec = spec * kk ** (-alpha) / n
    out = np.zeros((L, H), dtype=np.complex128)
    out[kx.astype(np.int64) + L // 2, :] = spec
    out = out.astype(dtype)
    c = np.arange(L) - L // 2
    partner = -c + L // 2
    valid = (partner >= 0) & (partner < L)
    col = out[:, 0].copy()
    take = (c < 0) & valid
    col[take] = np.conj(col[partner[take]])
    col[~valid] = 0
    col[L // 2] = col[L // 2].real
    out[:, 0] = col
    return out


def hermitian_3d(L: int, seed: int, alpha: float = 5.0 / 3.0, dtype=np.complex64) -> np.ndarray:
    """Stored half of a 3D Hermitian-symmetric field, centered in x and y.

    Built from a seeded real field of odd size (2*ceil(L/2)-1)^3 through a
    real-to-complex FFT, scaled by |k|^-alpha (k = 0 scaled by 1), then made
    exactly symmetric on the z = 0 plane: f(-x,-y,0) = conj f(x,y,0) with
    f(0,0,0) real.  For even L the centered index -L/2 (the Nyquist row of
    each outer axis) is zero.  Returns shape (L, L, ceil(L/2)).
    """
    g = _rng(seed)
    H = (L + 1) // 2          # stored length of the innermost (Hermitian) axis
    n = 2 * H - 1             # odd effective length of every axis
    field = g.standard_normal((n, n, n))
    spec = np.fft.rfftn(field)            # (n, n, H), uncentered kx, ky; kz = 0..H-1
    kx = np.fft.fftfreq(n, d=1.0 / n)     # integer wavenumbers -(H-1)..(H-1)
    kz = np.arange(H, dtype=np.float64)
    kk = np.sqrt(kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2)
    kk[0, 0, 0] = 1.0
    spec = spec * kk ** (-alpha) / (n ** 1.5)
    # centered layout: stored x index j <-> centered c = j - L//2
    out = np.zeros((L, L, H), dtype=np.complex128)
    c = kx.astype(np.int64)               # centered index of each uncentered slot
    jx = c + L // 2
    out[np.ix_(jx, jx, np.arange(H))] = spec
    # exact symmetry on the z = 0 plane: the canonical half keeps its value,
    # the other half is the conjugate of its partner; the origin is real
    out = out.astype(dtype)
    c_all = np.arange(L) - L // 2
    ca, cb = c_all[:, None], c_all[None, :]
    pa = np.broadcast_to(-ca + L // 2, (L, L))
    pb = np.broadcast_to(-cb + L // 2, (L, L))
    valid = (pa >= 0) & (pa < L) & (pb >= 0) & (pb < L)
    neg = (ca < 0) | ((ca == 0) & (cb < 0))
    plane = out[:, :, 0].copy()
    sym = plane.copy()
    take = neg & valid
    sym[take] = np.conj(plane[pa[take], pb[take]])
    sym[~valid] = 0
    sym[L // 2, L // 2] = sym[L // 2, L // 2].real
    out[:, :, 0] = sym
    return out


def ragged_instances(count: int, seed: int, bound, L_lo: int = 64, L_hi: int = 65536,
                     ratio_lo: float = 0.3, ratio_hi: float = 0.67):
    """Workload list for a ragged batch of 1D convolutions.

    L is log-uniform on [L_lo, L_hi]; the padding ratio L/M is uniform on
    [ratio_lo, ratio_hi]; A is 2 or 3 with probability 1/2 each; B = 1.
    Ratios above 1/2 cannot dealias the full complex product, so those
    instances use the centered kind; M is then raised, if needed, to the
    smallest dealiased length of the kind, which the caller's
    ``bound(kind, L, mult)`` gives (this module holds no dealiasing
    arithmetic).  Returns a list of dicts with keys L, M, A, B, kind
    ("complex"/"centered"), ratio and clamped (True when M was raised).
    """
    g = _rng(seed)
    Ls = np.floor(np.exp(g.uniform(math.log(L_lo), math.log(L_hi), size=count))).astype(np.int64)
    ratios = g.uniform(ratio_lo, ratio_hi, size=count)
    As = np.where(g.uniform(size=count) < 0.5, 2, 3)
    out = []
    for L, r, A in zip(Ls.tolist(), ratios.tolist(), As.tolist()):
        kind = "centered" if r > 0.5 else "complex"
        M0 = int(math.ceil(L / r))
        M = max(M0, int(bound(kind, int(L), "product" if A == 2 else "sum_pairs3")))
        out.append(dict(L=int(L), M=int(M), A=int(A), B=1, kind=kind, ratio=float(r), clamped=M != M0))
    return out
