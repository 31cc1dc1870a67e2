"""The paper's residue-at-a-time convolution, step by step, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

This follows Alg. convolve (complex) and Alg. convolveX (centered and
Hermitian): for each residue the A inputs are forward transformed, ``mult``
combines them, and the B backward transforms are accumulated; the sum is
divided by qm.  The per-residue transforms are written from the paper's
equations in the paper's order:

  forward1 / backward1   (p = 1)   Eq. forStan / invStan with t = 0
  forward2 / backward2   (p = 2)   the two blocks t = 0, 1 of Eq. forStan;
                                   backward2 uses zeta_qm^{-s r} for s >= m
                                   (Eq. invStan with t = 1; the printed
                                   exponent -(s-m) r drops zeta_q^{-r})
  forwardInner / backwardInner (p > 2)   Section 6.1: twist zeta_q^{vt}, size-p
                                   DFTs along t, twiddle zeta_qm^{(un+v)s},
                                   size-m FFTs; Eq. invInner backwards
  forward2C / backward2C (p = 2)   Eq. wDef with out-of-range f taken as 0;
                                   backward stores zeta_qm^{-r c} W_{c mod m} at
                                   each centered output c (Eq. invStan, Section 3)
  forwardInnerC / backwardInnerC   Section 6.2 (fold factor zeta_n^{-v})
  forward2H / backward2H,          as the centered transforms with
  forwardInnerH / backwardInnerH   f_{-j} = conj f_j (Eq. wHerDef); the size-m
                                   transforms are complex-to-real forward
                                   (crfft) and real-to-complex backward (rcfft).

The size-m (and size-p) DFTs call numpy's FFT (a library primitive):
fft(x)_l = sum_s zeta_m^{l s} x_s (positive exponent, as in Section 2) is
m * numpy.fft.ifft, and ifft(X)_s = sum_l zeta_m^{-s l} X_l is numpy.fft.fft.
"""
from __future__ import annotations

import numpy as np

from .params import derive


def zeta(N: int, e) -> np.ndarray:
    """zeta_N^e with the integer exponent reduced exactly mod N."""
    e = np.mod(np.asarray(e, dtype=np.int64), N)
    return np.exp(2j * np.pi * e / N)


def fft(x, axis=-1):
    x = np.asarray(x, dtype=np.complex128)
    return np.fft.ifft(x, axis=axis) * x.shape[axis]


def ifft(X, axis=-1):
    return np.fft.fft(np.asarray(X, dtype=np.complex128), axis=axis)


def crfft(w_half, m):
    """Complex-to-real size-m transform with positive exponent from e = m//2+1 values."""
    return np.fft.irfft(np.asarray(w_half, dtype=np.complex128), n=m) * m


def rcfft(F):
    """Real-to-complex size-m transform with negative exponent; returns m//2+1 values."""
    return np.fft.rfft(np.asarray(F, dtype=np.float64))


# ------------------------------------------------------------------ complex

def forward1(f, L, m, q, r):
    W = np.zeros(m, dtype=np.complex128)
    s = np.arange(L)
    W[:L] = zeta(q * m, r * s) * f[:L]
    return fft(W)


def backward1(F, L, m, q, r):
    W = ifft(F)
    s = np.arange(L)
    return zeta(q * m, -r * s) * W[:L]


def forward2(f, L, m, q, r):
    W = np.zeros(m, dtype=np.complex128)
    s = np.arange(L - m)
    W[:L - m] = zeta(q * m, r * s) * f[:L - m] + zeta(q * m, r * (m + s)) * f[m:L]
    s = np.arange(L - m, m)
    W[L - m:] = zeta(q * m, r * s) * f[L - m:m]
    return fft(W)


def backward2(F, L, m, q, r):
    W = ifft(F)
    V = np.zeros(L, dtype=np.complex128)
    s = np.arange(m)
    V[:m] = zeta(q * m, -s * r) * W
    s = np.arange(m, L)
    V[m:] = zeta(q * m, -s * r) * W[s - m]
    return V


def forwardInner(f, L, m, p, q, n, v):
    W = np.zeros((p, m), dtype=np.complex128)
    flat = np.zeros(p * m, dtype=np.complex128)
    flat[:L] = f[:L]
    t = np.arange(p)[:, None]
    W = zeta(q, v * t) * flat.reshape(p, m)
    W = fft(W, axis=0)                                 # size-p DFT along t -> u
    u = np.arange(p)[:, None]
    s = np.arange(m)[None, :]
    W = W * zeta(q * m, (u * n + v) * s)
    return fft(W, axis=1).reshape(p * m)               # F[u m + l]


def backwardInner(F, L, m, p, q, n, v):
    W = ifft(np.asarray(F).reshape(p, m), axis=1)
    u = np.arange(p)[:, None]
    s = np.arange(m)[None, :]
    W = W * zeta(q * m, -s * (u * n + v))
    W = ifft(W, axis=0)                                # size-p inverse along u -> t
    t = np.arange(p)[:, None]
    V = (zeta(q, -t * v) * W).reshape(p * m)
    return V[:L]


# ------------------------------------------------------------------ centered

def _centered_get(f, L, c):
    """f at centered indices c (array); zero outside [-H, L-H-1]."""
    H = L // 2
    c = np.asarray(c)
    j = c + H
    ok = (j >= 0) & (j < L)
    out = np.zeros(c.shape, dtype=np.complex128)
    out[ok] = f[j[ok]]
    return out


def forward2C(f, L, m, q, r, get=_centered_get):
    s = np.arange(m)
    w = zeta(q * m, r * s) * (get(f, L, s) + zeta(q, -r) * get(f, L, s - m))
    return fft(w)


def backward2C(F, L, m, q, r):
    W = ifft(F)
    H = L // 2
    c = np.arange(L) - H
    return zeta(q * m, -r * c) * W[np.mod(c, m)]


def forwardInnerC(f, L, m, p, q, n, v, get=_centered_get):
    ph = p // 2
    t = np.arange(ph)[:, None]
    s = np.arange(m)[None, :]
    j = t * m + s
    X = zeta(q, v * t) * (get(f, L, j) + zeta(n, -v) * get(f, L, j - p * m // 2))
    X = fft(X, axis=0)                                 # size-p/2 DFT along t -> u
    u = np.arange(ph)[:, None]
    X = X * zeta(q * m, (u * n + v) * s)
    return fft(X, axis=1).reshape(ph * m)


def backwardInnerC(F, L, m, p, q, n, v):
    ph = p // 2
    W = ifft(np.asarray(F).reshape(ph, m), axis=1)
    u = np.arange(ph)[:, None]
    s = np.arange(m)[None, :]
    W = W * zeta(q * m, -(u * n + v) * s)
    Y = ifft(W, axis=0)                                # -> t
    H = L // 2
    V = np.zeros(L, dtype=np.complex128)
    t = np.arange(ph)[:, None]
    for c0, fac in ((t * m + s, zeta(q, -v * t)), (t * m + s - p * m // 2, zeta(q, -v * (t - ph)))):
        val = fac * Y
        j = c0 + H
        ok = (j >= 0) & (j < L)
        V[j[ok]] += val[ok]
    return V


# ------------------------------------------------------------------ Hermitian

def _hermitian_get(f, L, c):
    """Stored half f_0..f_{H-1}; f_{-c} = conj f_c; zero beyond |c| >= H."""
    Hc = (L + 1) // 2
    c = np.asarray(c)
    a = np.abs(c)
    ok = a < Hc
    out = np.zeros(c.shape, dtype=np.complex128)
    vals = np.where(c >= 0, f[np.where(ok, a, 0)], np.conj(f[np.where(ok, a, 0)]))
    out[ok] = vals[ok]
    # index 0 is real
    z = c == 0
    out[z] = np.real(f[0])
    return out


def forward2H(f, L, m, q, r):
    e = m // 2 + 1
    s = np.arange(e)
    w = zeta(q * m, r * s) * (_hermitian_get(f, L, s) + zeta(q, -r) * _hermitian_get(f, L, s - m))
    return crfft(w, m)                                  # m real values


def backward2H(F, L, m, q, r):
    Hc = (L + 1) // 2
    Wh = rcfft(F)                                       # W_s, s < e
    e = m // 2 + 1
    c = np.arange(Hc)
    Wc = np.where(c < e, Wh[np.minimum(c, e - 1)], np.conj(Wh[np.clip(m - c, 0, e - 1)]))
    return zeta(q * m, -r * c) * Wc


def forwardInnerH(f, L, m, p, q, n, v):
    ph = p // 2
    e = m // 2 + 1
    t = np.arange(ph)[:, None]
    s = np.arange(e)[None, :]
    j = t * m + s
    X = zeta(q, v * t) * (_hermitian_get(f, L, j) + zeta(n, -v) * _hermitian_get(f, L, j - p * m // 2))
    X = fft(X, axis=0)
    u = np.arange(ph)[:, None]
    X = X * zeta(q * m, (u * n + v) * s)
    return np.concatenate([crfft(X[uu], m) for uu in range(ph)])


def backwardInnerH(F, L, m, p, q, n, v):
    ph = p // 2
    e = m // 2 + 1
    Hc = (L + 1) // 2
    W = np.stack([rcfft(np.asarray(F)[uu * m:(uu + 1) * m]) for uu in range(ph)])   # (u, s), s < e
    u = np.arange(ph)[:, None]
    s = np.arange(e)[None, :]
    W = W * zeta(q * m, -(u * n + v) * s)
    Y = ifft(W, axis=0)                                 # size-p/2 inverse along u -> (t, s)
    # Row t gives the output at c = t m + s for s < e.  The remaining columns
    # s' = m - s (1 <= s <= m - e) follow from the real residue values: the
    # output at c = (p/2 - t) m - s is zeta_q^{-v(p/2-t)} conj(Y[t, s]).
    V = np.zeros(Hc, dtype=np.complex128)
    for t in range(ph):
        for s_ in range(e):
            c = t * m + s_
            if c < Hc:
                V[c] += zeta(q, -v * t) * Y[t, s_]
        for s_ in range(1, m - e + 1):
            c = (ph - t) * m - s_
            if 0 <= c < Hc:
                V[c] += zeta(q, -v * (ph - t)) * np.conj(Y[t, s_])
    return V


# ------------------------------------------------------------------ drivers

def _mult(Fs, mult):
    """The B transformed outputs of one residue, pointwise in the A transformed
    inputs (the Basdevant forms of Section 9: velocity components in, the
    products of the nonlinear term out)."""
    if mult == "product":
        return [Fs[0] * Fs[1]]
    if mult == "sum_pairs3":
        return [Fs[0] * Fs[1] + Fs[1] * Fs[2] + Fs[2] * Fs[0]]
    if mult == "basdevant2":
        u, v = Fs
        return [u * v, u * u - v * v]
    if mult == "basdevant3":
        u, v, w = Fs
        return [u * v, v * w, w * u, u * u - w * w, v * v - w * w]
    if mult == "mhd3":   # traceless part of T_ij = Z-_i Z+_j (Elsasser components)
        p0, p1, p2, m0, m1, m2 = Fs
        return [m0 * p1, m0 * p2, m1 * p0, m1 * p2, m2 * p0, m2 * p1, m0 * p0 - m2 * p2, m1 * p1 - m2 * p2]
    raise ValueError(mult)


def _accumulate(h, Hs, backward):
    """h_b += backward(H_b) for each output b (Alg. convolve: every output
    accumulates its residue contribution)."""
    for b, Hb in enumerate(Hs):
        h[b] += backward(Hb)


def _outputs(h):
    return h[0] if h.shape[0] == 1 else h


def _residue_range(n, residues):
    """Residues r_begin <= r < r_end summed (all n by default): the residue
    contributions are independent and add up (Section 2.2), so a subset gives
    the partial sum that one share of a residue-split convolution computes."""
    if residues is None:
        return range(n)
    r0, r1 = residues
    assert 0 <= r0 <= r1 <= n
    return range(r0, r1)


def convolve(fs, L, M, m, mult="product", p=None, q=None, residues=None):
    """Alg. convolve: complex 1D convolution, one residue at a time
    (residues = (r_begin, r_end): that part of the residue sum only)."""
    if p is None:
        p, q, n = derive("complex", L, M, m)
    else:
        n = q if p <= 2 else q // p
    fs = [np.asarray(f, dtype=np.complex128) for f in fs]
    h = np.zeros((len(_mult([np.zeros(1)] * len(fs), mult)), L), dtype=np.complex128)
    for r in _residue_range(n, residues):
        if p == 1:
            Fs = [forward1(f, L, m, q, r) for f in fs]
            back = lambda F: backward1(F, L, m, q, r)
        elif p == 2:
            Fs = [forward2(f, L, m, q, r) for f in fs]
            back = lambda F: backward2(F, L, m, q, r)
        else:
            Fs = [forwardInner(f, L, m, p, q, n, r) for f in fs]
            back = lambda F: backwardInner(F, L, m, p, q, n, r)
        Hs = _mult(Fs, mult)
        _accumulate(h, Hs, back)
    return _outputs(h) / (q * m)


def convolveX(fs, L, M, m, kind="centered", mult="product", residues=None):
    """Alg. convolveX: centered (X = C) or Hermitian (X = H) 1D convolution
    (residues as in convolve)."""
    p, q, n = derive(kind, L, M, m)
    fs = [np.asarray(f, dtype=np.complex128) for f in fs]
    B = len(_mult([np.zeros(1)] * len(fs), mult))
    if kind == "centered":
        h = np.zeros((B, L), dtype=np.complex128)
        for r in _residue_range(n, residues):
            if p == 2:
                Fs = [forward2C(f, L, m, q, r) for f in fs]
                back = lambda F: backward2C(F, L, m, q, r)
            else:
                Fs = [forwardInnerC(f, L, m, p, q, n, r) for f in fs]
                back = lambda F: backwardInnerC(F, L, m, p, q, n, r)
            Hs = _mult(Fs, mult)
            _accumulate(h, Hs, back)
        return _outputs(h) / (q * m)
    if kind == "hermitian":
        Hc = (L + 1) // 2
        h = np.zeros((B, Hc), dtype=np.complex128)
        for r in _residue_range(n, residues):
            if p == 2:
                Fs = [forward2H(f, L, m, q, r) for f in fs]
                back = lambda F: backward2H(F, L, m, q, r)
            else:
                Fs = [forwardInnerH(f, L, m, p, q, n, r) for f in fs]
                back = lambda F: backwardInnerH(F, L, m, p, q, n, r)
            Hs = _mult(Fs, mult)
            _accumulate(h, Hs, back)
        return _outputs(h) / (q * m)
    raise ValueError(kind)
