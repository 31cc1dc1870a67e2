"""The fused kernels' formulation of one residue, restated in numpy and pinned
to the direct definition on the CPU.

With N = q m = n S, residue r needs one size-S FFT of the twisted input folded
modulo S, W_j = sum over i = j (mod S) of zeta_N^{r i} f_i, and contributes
zeta_N^{-r i} IFFT_S(mult(F))_{i mod S} to output i (Alg. convolve /
convolveX reorganized: forward1/forward2, forwardInner with its size-p DFTs
merged into one size-p m FFT, the centered fold with zeta_N^{-r S}, and the
Hermitian residues paired in one complex FFT).  The fold and twist follow the
kernels' two-block form: block 0 holds index j, block 1 index j + S (complex)
or j - S (centered, Hermitian), with the block-1 factor zeta_N^{r S} or its
conjugate.  numpy's FFT is the FFT step.  Every legal (m, p, q) of small L
must reproduce the direct convolution of oracle/direct.py, for every kind and
mult; this pins the sign, twist and fold conventions the kernels implement
(their GPU parity is tested against the same oracle in tests/*_gpu.py).
"""
import numpy as np
import pytest

import inputs
from oracle import direct, params


def zeta(N, e):
    return np.exp(2j * np.pi * np.asarray(e, dtype=np.float64) / N)


def geometry(kind, m, p, q):
    if p == 1 and q == 1:
        return m, 1
    if kind == "complex":
        return (m, q) if p <= 2 else (p * m, q // p)
    return p * m // 2, q // (p // 2)


def mult_outputs(F, mult):
    """B transformed outputs of one residue (pointwise in the A transforms)."""
    if mult == "product":
        return [F[0] * F[1]]
    if mult == "sum_pairs3":
        return [F[0] * F[1] + F[2] * (F[0] + F[1])]
    if mult == "basdevant2":
        return [F[0] * F[1], (F[0] + F[1]) * (F[0] - F[1])]
    if mult == "mhd3":
        p0, p1, p2, m0, m1, m2 = F
        return [m0 * p1, m0 * p2, m1 * p0, m1 * p2, m2 * p0, m2 * p1, m0 * p0 - m2 * p2, m1 * p1 - m2 * p2]
    raise ValueError(mult)


def blocks(kind, f, S):
    """(b0, b1): stored values folded to slot j from block 0 and block 1."""
    j = np.arange(S)
    b0 = np.zeros(S, complex)
    b1 = np.zeros(S, complex)
    if kind == "complex":
        L = len(f)
        b0[j < L] = f[j[j < L]]
        k = j + S < L
        b1[k] = f[j[k] + S]
    elif kind == "centered":
        L = len(f)
        H = L // 2
        k = j < L - H
        b0[k] = f[j[k] + H]
        k = j >= S - H
        b1[k] = f[j[k] - S + H]
    else:
        Ls = len(f)
        k = j < Ls
        b0[k] = f[j[k]]
        b0[0] = f[0].real
        k = (j > 0) & (S - j < Ls)
        b1[k] = np.conj(f[S - j[k]])
    return b0, b1


def convolve_formulation(fs, kind, mult, m, p, q, slip=None, conj_sym=False):
    """slip (planted mistakes): "fold_factor" (centered block-1 factor not
    conjugated), "sign" (forward transform with -zeta) or "csym_backward" (the
    paired residue's own backward twist after a conjugated forward one).
    conj_sym: residues r > n/2 (complex and centered kinds) twist with the
    conjugated twists of residue n - r, in both directions (Section 6.3, as the
    kernels do: their spectra come out shifted by one frequency)."""
    S, n = geometry(kind, m, p, q)
    N = n * S
    fs = [np.asarray(f, complex) for f in fs]
    Ls = len(fs[0])
    L = Ls if kind != "hermitian" else None
    B = direct.OUTPUTS[mult]
    acc0 = np.zeros((B, S), complex)   # block 0 outputs (slot j)
    acc1 = np.zeros((B, S), complex)   # block 1 outputs
    j = np.arange(S)
    bl = [blocks(kind, f, S) for f in fs]

    def twist(r):
        if conj_sym and 2 * r > n:
            return np.conj(zeta(N, (n - r) * j))
        return zeta(N, r * j)

    def twisted(r):
        cr = zeta(N, r * S)
        if kind != "complex" and slip != "fold_factor":
            cr = np.conj(cr)
        return [(b0 + cr * b1) * twist(r) for b0, b1 in bl], cr

    if kind != "hermitian":
        for r in range(n):
            W, cr = twisted(r)
            # forward with +zeta (Eq. forStan): F_l = sum_j zeta_S^{j l} W_j
            F = [np.fft.fft(w) if slip == "sign" else np.fft.ifft(w) * S for w in W]
            Y = [np.fft.fft(h) for h in mult_outputs(F, mult)]   # unnormalized inverse: zeta^{-}
            tb = zeta(N, r * j) if slip == "csym_backward" else twist(r)
            for b in range(B):
                y = Y[b] * np.conj(tb)
                acc0[b] += y
                acc1[b] += y * np.conj(cr)
    else:
        for r1 in range(0, n, 2):
            r2 = r1 + 1
            W1, _ = twisted(r1)
            W2, _ = twisted(r2) if r2 < n else ([np.zeros(S, complex)] * len(fs), 0)
            F = [np.fft.ifft(a + 1j * b) * S for a, b in zip(W1, W2)]
            # real parts carry residue r1, imaginary parts residue r2
            Fr = mult_outputs([x.real for x in F], mult)
            Fi = mult_outputs([x.imag for x in F], mult)
            for b in range(B):
                Y = np.fft.fft(Fr[b] + 1j * Fi[b])
                Ym = np.conj(Y[(S - j) % S])
                g1 = (Y + Ym) / 2
                g2 = (Y - Ym) / 2j
                y = g1 * np.conj(zeta(N, r1 * j))
                if r2 < n:
                    y = y + g2 * np.conj(zeta(N, r2 * j))
                acc0[b] += y
    out = np.zeros((B, Ls), complex)
    if kind == "complex":
        k = j < L
        out[:, j[k]] = acc0[:, k]
        k = j + S < L
        out[:, j[k] + S] = acc1[:, k]
    elif kind == "centered":
        H = L // 2
        k = j < L - H
        out[:, j[k] + H] = acc0[:, k]
        k = j >= S - H
        out[:, j[k] - S + H] = acc1[:, k]
    else:
        out[:, :] = acc0[:, :Ls]
    out /= N
    return out[0] if B == 1 else out


def legal_plans(kind, L, M):
    """(m, p, q) of every m with a power-of-two transform size, plus the explicit plan."""
    seen = set()
    for m in range(1, 2 * M + 1):
        p, q, n = params.derive(kind, L, M, m)
        S, nn = geometry(kind, m, p, q)
        if S & (S - 1) == 0 and (S, nn) not in seen:
            seen.add((S, nn))
            yield m, p, q
    S = 1
    while S < M:
        S *= 2
    yield S, 1, 1


def stored(kind, L, A, seed):
    if kind == "hermitian":
        return [inputs.hermitian_1d(1, L, seed + a)[0] for a in range(A)]
    return [inputs.uniform_complex(L, seed + a) for a in range(A)]


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("mult", ["product", "sum_pairs3", "basdevant2"])
def test_formulation_equals_definition_every_plan(kind, mult):
    A = direct.MULTS[mult]
    checked = 0
    for L in (1, 2, 3, 5, 8, 13, 16, 21):
        fs = stored(kind, L, A, 300 + L)
        ref = direct.conv1d(fs, kind, mult)
        bound = params.dealias_bound(kind, L, mult)
        for M in (bound, bound + 3, 2 * L + 5):
            for m, p, q in legal_plans(kind, L, M):
                got = convolve_formulation(fs, kind, mult, m, p, q)
                assert np.allclose(got, ref, atol=1e-10), (kind, mult, L, M, m, p, q)
                checked += 1
    assert checked >= 50


@pytest.mark.parametrize("slip", ["fold_factor", "sign"])
def test_formulation_planted_slips_fail(slip):
    """The same restatement with the centered block-1 factor not conjugated,
    or with the forward transform's sign flipped, misses the definition."""
    L, M = 13, 20
    fs = stored("centered", L, 2, 77)
    ref = direct.conv1d(fs, "centered")
    m, p, q = 4, 4, 6                        # S = 8, n = 3: both blocks of the fold are used
    assert params.derive("centered", L, M, m) == (p, q, 3)
    assert np.allclose(convolve_formulation(fs, "centered", "product", m, p, q), ref, atol=1e-10)
    bad = convolve_formulation(fs, "centered", "product", m, p, q, slip=slip)
    assert not np.allclose(bad, ref, atol=1e-6)


@pytest.mark.parametrize("kind", ["complex", "centered"])
@pytest.mark.parametrize("mult", ["product", "sum_pairs3", "basdevant2", "mhd3"])
def test_conjugate_symmetry_pairs_equal_definition(kind, mult):
    """Conjugate symmetry (Section 6.3) as the kernels use it: residue r > n/2
    takes the conjugated twists of residue n - r in both directions; every plan
    with n >= 3 (where some residue is paired) still gives the definition."""
    A = direct.MULTS[mult]
    checked = 0
    for L in (3, 8, 13, 21):
        fs = stored(kind, L, A, 500 + L)
        ref = direct.conv1d(fs, kind, mult)
        bound = params.dealias_bound(kind, L, mult)
        for M in (bound, 2 * L + 5, 3 * L + 1):
            for m, p, q in legal_plans(kind, L, M):
                S, n = geometry(kind, m, p, q)
                if n < 3:
                    continue
                got = convolve_formulation(fs, kind, mult, m, p, q, conj_sym=True)
                assert np.allclose(got, ref, atol=1e-10), (kind, mult, L, M, m, p, q)
                checked += 1
    assert checked >= 10


def test_conjugate_symmetry_planted_slip_fails():
    """Conjugated forward twists with the paired residue's own backward twist
    (the one-frequency shift left in place) miss the definition."""
    L, M = 13, 20
    fs = stored("centered", L, 2, 77)
    ref = direct.conv1d(fs, "centered")
    m, p, q = 4, 4, 6                        # S = 8, n = 3: residue 2 pairs with residue 1
    assert np.allclose(convolve_formulation(fs, "centered", "product", m, p, q, conj_sym=True), ref, atol=1e-10)
    bad = convolve_formulation(fs, "centered", "product", m, p, q, slip="csym_backward", conj_sym=True)
    assert not np.allclose(bad, ref, atol=1e-6)
