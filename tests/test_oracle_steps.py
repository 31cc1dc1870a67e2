"""Pins of the step-by-step oracle (oracle/steps.py) and of the per-residue
definition (oracle/residue.py).

* The paper's residue-at-a-time algorithm equals the direct definition for
  every m (hence every legal (m, p, q)) on small sizes.
* An explicit zero-padded FFT convolution at size qm equals the direct
  definition for every legal plan (the hybrid method is a reorganization of
  that length-qm transform).
* Each per-residue forward transform of the paper equals the naive length-qm
  DFT at k = q l + r (or q l + u n + v).
* Planted mistakes: the printed forms that the readings replace, and a few
  plausible slips, make a pin fail.
"""
import numpy as np
import pytest

import inputs
from oracle import direct, explicit, params, residue, steps


def _fs(kind, L, seed, A=2, integer=False):
    if kind == "hermitian":
        return [inputs.hermitian_1d(1, L, seed + a, integer=integer)[0] for a in range(A)]
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    return [gen(L, seed + a) for a in range(A)]


def _run_steps(kind, fs, L, M, m, mult="product"):
    if kind == "complex":
        return steps.convolve(fs, L, M, m, mult)
    return steps.convolveX(fs, L, M, m, kind, mult)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_steps_equal_definition_every_m(kind):
    for L in range(1, 13):
        fs = _fs(kind, L, 1000 + L)
        ref = direct.conv1d(fs, kind)
        lo = params.dealias_bound(kind, L)
        for M in range(lo, 3 * L + 1):
            for m in range(1, M + 2):
                got = _run_steps(kind, fs, L, M, m)
                assert np.allclose(got, ref, atol=1e-11), (kind, L, M, m)


@pytest.mark.parametrize("kind", ["complex", "centered"])
def test_steps_sum_pairs3(kind):
    for L in (5, 9):
        fs = _fs(kind, L, 77, A=3)
        ref = direct.conv1d(fs, kind, "sum_pairs3")
        for m in range(1, 2 * L):
            got = _run_steps(kind, fs, L, 2 * L, m, "sum_pairs3")
            assert np.allclose(got, ref, atol=1e-11)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("mult", ["basdevant2", "basdevant3", "mhd3"])
def test_steps_multi_output(kind, mult):
    """B > 1 outputs: each accumulates its own residue contributions; the
    algorithm equals the definition for every m."""
    A = direct.MULTS[mult]
    for L in (4, 7):
        fs = _fs(kind, L, 88, A=A)
        ref = direct.conv1d(fs, kind, mult)
        M = params.dealias_bound(kind, L, mult)
        for m in range(1, M + 2):
            got = _run_steps(kind, fs, L, M, m, mult)
            assert got.shape == ref.shape
            assert np.allclose(got, ref, atol=1e-11), (kind, mult, L, m)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_explicit_at_qm_equals_definition(kind):
    for L in range(1, 11):
        fs = _fs(kind, L, 2000 + L)
        ref = direct.conv1d(fs, kind)
        lo = params.dealias_bound(kind, L)
        for M in range(lo, 3 * L + 1):
            seen = set()
            for m in range(1, M + 2):
                p, q, n = params.derive(kind, L, M, m)
                if q * m in seen:
                    continue
                seen.add(q * m)
                got = explicit.convnd_explicit(fs, (kind,), [q * m])
                assert np.allclose(got, ref, atol=1e-11), (kind, L, M, m)


def test_integer_inputs_round_exactly():
    for kind in ("complex", "centered", "hermitian"):
        L, M = 40, 2 * 40
        fs = _fs(kind, L, 5, integer=True)
        ref = direct.conv1d(fs, kind)
        for m in (3, 8, 16, 20, 40, 80):
            got = _run_steps(kind, fs, L, M, m)
            assert np.array_equal(np.rint(got.real) + 1j * np.rint(got.imag), ref)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_residue_forward_steps_equal_definition(kind):
    L = 13
    f = _fs(kind, L, 3)[0]
    M = params.dealias_bound(kind, L) + 2
    for m in range(1, 2 * L):
        p, q, n = params.derive(kind, L, M, m)
        defs = residue.residue_forward(kind, f, L, M, m)
        assert len(defs) == n
        for r in range(n):
            if kind == "complex":
                got = {1: lambda: steps.forward1(f, L, m, q, r), 2: lambda: steps.forward2(f, L, m, q, r)}.get(
                    p, lambda: steps.forwardInner(f, L, m, p, q, n, r))()
            elif kind == "centered":
                got = steps.forward2C(f, L, m, q, r) if p == 2 else steps.forwardInnerC(f, L, m, p, q, n, r)
            else:
                got = steps.forward2H(f, L, m, q, r) if p == 2 else steps.forwardInnerH(f, L, m, p, q, n, r)
            assert np.allclose(got, defs[r], atol=1e-11), (kind, m, r)
            if kind == "hermitian":
                assert np.max(np.abs(defs[r].imag)) < 1e-11      # Section 4: real residues


def test_fig1_residue_layout():
    # Fig. 1: L=6, M=11, m=4 -> p=2, q=3: three residues of m=4 values each,
    # together the length-12 padded DFT.
    f = inputs.uniform_complex(6, 8)
    rs = residue.residue_forward("complex", f, 6, 11, 4)
    assert len(rs) == 3 and all(len(x) == 4 for x in rs)
    full = np.zeros(12, complex)
    for r in range(3):
        full[r::3] = rs[r]
    pad = np.zeros(12, complex)
    pad[:6] = f
    assert np.allclose(full, 12 * np.fft.ifft(pad), atol=1e-12)   # positive-exponent DFT


# ----------------------------------------------------------- planted mistakes

def test_printed_backward2_exponent_fails():
    """backward2 as printed (zeta^{-(s-m) r} for s >= m) is wrong; the reading
    zeta^{-s r} is what reproduces the definition."""
    L, M, m = 7, 13, 4
    fs = _fs("complex", L, 9)
    ref = direct.conv1d(fs, "complex")
    orig = steps.backward2

    def printed(F, L, m, q, r):
        W = steps.ifft(F)
        V = np.zeros(L, dtype=np.complex128)
        s = np.arange(m)
        V[:m] = steps.zeta(q * m, -s * r) * W
        s = np.arange(m, L)
        V[m:] = steps.zeta(q * m, -(s - m) * r) * W[s - m]
        return V

    try:
        steps.backward2 = printed
        bad = steps.convolve(fs, L, M, m)
    finally:
        steps.backward2 = orig
    assert not np.allclose(bad, ref, atol=1e-6)
    assert np.allclose(steps.convolve(fs, L, M, m), ref, atol=1e-11)


@pytest.mark.parametrize("slip", ["sign", "twiddle_index", "fold_factor", "norm"])
def test_planted_slips_fail(slip):
    L, M, m = 7, 13, 4                     # p = 2, q = 4: forward2 is on the path
    assert params.derive("complex", L, M, m)[0] == 2
    fs = _fs("complex", L, 12)
    ref = direct.conv1d(fs, "complex")
    orig_f2, orig_b2 = steps.forward2, steps.backward2
    orig_z = steps.zeta

    def f2(f, L, m, q, r):
        W = np.zeros(m, dtype=np.complex128)
        s = np.arange(L - m)
        fac = steps.zeta(q, r) if slip != "fold_factor" else steps.zeta(q, -r)
        idx = s if slip != "twiddle_index" else s + 1
        W[:L - m] = steps.zeta(q * m, r * idx) * (f[:L - m] + fac * f[m:L])
        s = np.arange(L - m, m)
        idx = s if slip != "twiddle_index" else s + 1
        W[L - m:] = steps.zeta(q * m, r * idx) * f[L - m:m]
        return steps.fft(W) if slip != "sign" else steps.ifft(W)

    try:
        steps.forward2 = f2
        if slip == "norm":
            # dividing by M instead of qm
            steps.forward2 = orig_f2
            p, q, n = params.derive("complex", L, M, m)
            bad = steps.convolve(fs, L, M, m) * (q * m) / M
        else:
            bad = steps.convolve(fs, L, M, m)
    finally:
        steps.forward2, steps.backward2 = orig_f2, orig_b2
        steps.zeta = orig_z
    assert not np.allclose(bad, ref, atol=1e-6), slip


def test_direct_planted_slip_fails():
    # a dropped term (sum_pairs3 without F3F1) is caught by the brute force
    from tests.test_oracle_direct import brute_1d
    fs = _fs("complex", 6, 4, A=3, integer=True)
    ref = brute_1d(fs, "complex", "sum_pairs3")
    dropped = direct.full_linear(fs[0], fs[1])[:6] + direct.full_linear(fs[1], fs[2])[:6]
    assert not np.array_equal(dropped, ref)
    assert np.array_equal(direct.conv1d(fs, "complex", "sum_pairs3"), ref)
