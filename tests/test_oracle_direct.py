"""Pins of the direct-definition oracle (oracle/direct.py, oracle/direct_conv.c).

Each pin is independent of the function it checks: a pure-Python brute force
over index pairs with exact integers, delta-function shifts, commutativity,
linearity, the sum rule of a product of transforms, and agreement of the
numpy and C implementations.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import inputs
from oracle import cdirect, direct, explicit


def brute_1d(fs, kind, mult):
    """Textbook definition with Python ints: every pair of input indices adds
    f_i g_k to the output index i + k; outputs are selected by kind."""
    def as_dict(f):
        f = [complex(x) for x in f]
        if kind == "complex":
            return {i: f[i] for i in range(len(f))}
        if kind == "centered":
            L = len(f)
            return {i - L // 2: f[i] for i in range(L)}
        H = len(f)
        d = {0: complex(f[0].real, 0)}
        for c in range(1, H):
            d[c] = f[c]
            d[-c] = f[c].conjugate()
        return d
    ds = [as_dict(f) for f in fs]

    def conv(a, b):
        out = {}
        for i, x in ds[a].items():
            for k, y in ds[b].items():
                out[i + k] = out.get(i + k, 0) + x * y
        return out

    def lin(*terms):   # sum of c * dict
        out = {}
        for c, d in terms:
            for k, v in d.items():
                out[k] = out.get(k, 0) + c * v
        return out

    if mult == "product":
        outs = [conv(0, 1)]
    elif mult == "sum_pairs3":
        outs = [lin((1, conv(0, 1)), (1, conv(1, 2)), (1, conv(2, 0)))]
    elif mult == "basdevant2":        # u v, u^2 - v^2
        outs = [conv(0, 1), lin((1, conv(0, 0)), (-1, conv(1, 1)))]
    elif mult == "basdevant3":        # u v, v w, w u, u^2 - w^2, v^2 - w^2
        outs = [conv(0, 1), conv(1, 2), conv(2, 0), lin((1, conv(0, 0)), (-1, conv(2, 2))),
                lin((1, conv(1, 1)), (-1, conv(2, 2)))]
    else:                             # mhd3: inputs z+ = (0, 1, 2), z- = (3, 4, 5); T_ij = z-_i z+_j
        T = {(i, j): conv(3 + i, j) for i in range(3) for j in range(3)}
        outs = [T[0, 1], T[0, 2], T[1, 0], T[1, 2], T[2, 0], T[2, 1],
                lin((1, T[0, 0]), (-1, T[2, 2])), lin((1, T[1, 1]), (-1, T[2, 2]))]
    n = len(fs[0])
    if kind == "complex":
        keys = range(n)
    elif kind == "centered":
        keys = range(-(n // 2), n - n // 2)
    else:
        keys = range(n)
    res = np.array([[o.get(k, 0) for k in keys] for o in outs], dtype=np.complex128)
    return res[0] if len(outs) == 1 else res


ALL_MULTS = ["product", "sum_pairs3", "basdevant2", "basdevant3", "mhd3"]


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("mult", ALL_MULTS)
def test_brute_force_tiny(kind, mult):
    A = direct.MULTS[mult]
    for L in range(1, 13):
        if kind == "hermitian":
            fs = [inputs.hermitian_1d(1, L, 100 + L + a, integer=True)[0] for a in range(A)]
        else:
            fs = [inputs.integer_complex(L, 100 + L + a) for a in range(A)]
        got = direct.conv1d(fs, kind, mult)
        ref = brute_1d(fs, kind, mult)
        assert np.array_equal(got, ref), (kind, mult, L)


@pytest.mark.parametrize("kind", ["complex", "centered"])
def test_delta_shift(kind):
    L = 17
    g = inputs.uniform_complex(L, 3)
    for k in range(L):
        f = np.zeros(L, complex)
        f[k] = 1.0
        h = direct.conv1d([f, g], kind)
        H = L // 2 if kind == "centered" else 0
        # centered delta at c_k = k - H shifts g by c_k: h_c = g_{c - c_k}
        for j in range(L):
            src = j - (k - H)
            want = g[src] if 0 <= src < L else 0
            assert h[j] == want


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_commutative_and_linear(kind):
    L = 23
    if kind == "hermitian":
        f, g, u = inputs.hermitian_1d(3, L, 5)
    else:
        f, g, u = inputs.uniform_complex((3, L), 5)
    a = direct.conv1d([f, g], kind)
    b = direct.conv1d([g, f], kind)
    assert np.allclose(a, b, rtol=0, atol=1e-13)
    lin = direct.conv1d([2.5 * f + u, g], kind)
    ref = 2.5 * a + direct.conv1d([u, g], kind)
    assert np.allclose(lin, ref, rtol=0, atol=1e-12)


def test_sum_rule_product():
    # full products fit in the L outputs when the inputs live on [0, ceil(L/2))
    for L in (8, 9, 40, 41):
        half = (L + 1) // 2
        f = np.zeros(L, complex)
        g = np.zeros(L, complex)
        f[:half] = inputs.integer_complex(half, L)
        g[:half] = inputs.integer_complex(half, L + 1000)
        h = direct.conv1d([f, g], "complex")
        assert h.sum() == f.sum() * g.sum()


def test_sum_rule_centered():
    # centered inputs supported on [-floor(L/4), floor(L/4)] keep the full product in range
    L = 41
    H = L // 2
    f = np.zeros(L, complex)
    g = np.zeros(L, complex)
    k = L // 4
    f[H - k:H + k + 1] = inputs.integer_complex(2 * k + 1, 1)
    g[H - k:H + k + 1] = inputs.integer_complex(2 * k + 1, 2)
    h = direct.conv1d([f, g], "centered")
    assert h.sum() == f.sum() * g.sum()


def test_hermitian_matches_centered_on_expanded():
    L = 31
    f, g = inputs.hermitian_1d(2, L, 9)
    ef, eg = direct.hermitian_expand(f), direct.hermitian_expand(g)
    c = direct.conv1d([ef, eg], "centered")
    h = direct.conv1d([f, g], "hermitian")
    Le = len(ef)
    assert np.allclose(h, c[Le // 2:], rtol=0, atol=1e-13)
    # the convolution of Hermitian arrays is Hermitian: h_0 is real and the
    # negative half mirrors the positive half
    assert abs(h[0].imag) < 1e-13
    assert np.allclose(c[:Le // 2][::-1], np.conj(c[Le // 2 + 1:]), atol=1e-13)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("mult", ALL_MULTS)
def test_c_oracle_equals_numpy(kind, mult):
    A = direct.MULTS[mult]
    for L in (1, 2, 7, 64, 129):
        if kind == "hermitian":
            fs = [inputs.hermitian_1d(3, L, 11 + a, integer=True) for a in range(A)]
        else:
            fs = [inputs.integer_complex((3, L), 11 + a) for a in range(A)]
        ref = direct.conv1d_batch(fs, kind, mult)
        got = cdirect.conv1d_batch(fs, L, kind, mult, nthreads=2)
        assert np.array_equal(got, ref), (kind, mult, L)
        idx = np.arange(fs[0].shape[1])[::3]
        pts = cdirect.conv1d_points([f[0] for f in fs], L, idx, kind, mult)
        assert np.array_equal(pts, ref[..., 0, idx])
        pts2 = direct.conv1d_points([f[0] for f in fs], kind, idx, mult)
        assert np.array_equal(pts2, ref[..., 0, idx])


def test_integer_exactness_large():
    # |h_j| <= 64 L per component for entries in {-8..8}: exact in FP64
    L = 4096
    f, g = inputs.integer_complex((2, 1, L), 21)
    h = cdirect.conv1d_batch([f, g], L, "complex")
    assert np.array_equal(h, np.rint(h))
    idx = np.array([0, 1, 2047, 4095])
    exact = []
    fi = [complex(x) for x in f[0]]
    gi = [complex(x) for x in g[0]]
    for j in idx:
        exact.append(sum(fi[i] * gi[j - i] for i in range(j + 1)))
    assert np.array_equal(h[0, idx], np.array(exact))


def brute_nd(fs, kinds):
    """N-D textbook definition with explicit index pairs (non-Hermitian)."""
    f, g = fs
    shape = f.shape
    lo = [-(n // 2) if k == "centered" else 0 for n, k in zip(shape, kinds)]
    out = {}
    for i in itertools.product(*[range(n) for n in shape]):
        for k in itertools.product(*[range(n) for n in shape]):
            key = tuple(a + lo[d] + b + lo[d] for d, (a, b) in enumerate(zip(i, k)))
            out[key] = out.get(key, 0) + f[i] * g[k]
    res = np.zeros(shape, dtype=np.complex128)
    for j in itertools.product(*[range(n) for n in shape]):
        res[j] = out.get(tuple(a + lo[d] for d, a in enumerate(j)), 0)
    return res


@pytest.mark.parametrize("kinds", [("complex", "complex"), ("centered", "centered"), ("centered", "complex")])
def test_nd_brute_and_points(kinds):
    f = inputs.integer_complex((5, 4), 31)
    g = inputs.integer_complex((5, 4), 32)
    ref = brute_nd([f, g], kinds)
    got = direct.convnd([f, g], kinds)
    assert np.array_equal(got, ref)
    pts = np.array(list(itertools.product(range(5), range(4))))
    pv = direct.convnd_points([f, g], kinds, pts)
    assert np.array_equal(pv, ref.reshape(-1))


def test_nd_separable_closed_form():
    # f(x,y) = a(x) b(y), g = c(x) d(y)  =>  h = (a*c)(x) (b*d)(y)
    a, b, c, d = inputs.uniform_complex((4, 9), 41)
    for kinds in [("complex", "complex"), ("centered", "centered")]:
        f = np.outer(a, b)
        g = np.outer(c, d)
        h = direct.convnd([f, g], kinds)
        ref = np.outer(direct.conv1d([a, c], kinds[0]), direct.conv1d([b, d], kinds[1]))
        assert np.allclose(h, ref, atol=1e-12)


def test_nd_hermitian_3d_small():
    # Hermitian in the last axis with centered outer axes: must equal the 1D
    # Hermitian result for a field that only varies along z at x = y = 0 ...
    L = 6
    f = inputs.hermitian_3d(L, 51).astype(np.complex128)
    g = inputs.hermitian_3d(L, 52).astype(np.complex128)
    h = direct.convnd([f, g], ("centered", "centered", "hermitian"))
    # ... and, in general, the centered 3D convolution of the expanded arrays
    ef = direct.hermitian_expand_nd(f, f.shape[:-1])
    eg = direct.hermitian_expand_nd(g, g.shape[:-1])
    full = direct.convnd([ef, eg], ("centered", "centered", "centered"))
    H = f.shape[-1]
    assert np.allclose(h, full[:, :, H - 1:], atol=1e-12)
    # the expansion really is Hermitian symmetric: e(-x) = conj e(x) where both exist
    n0, n1, n2 = ef.shape
    for i in range(1, n0):
        for j in range(1, n1):
            for k in range(n2):
                mi, mj, mk = n0 - i, n1 - j, n2 - 1 - k
                assert ef[i, j, k] == np.conj(ef[mi, mj, mk])
    pts = np.array([[0, 0, 0], [3, 3, 0], [5, 1, 2], [2, 4, 1]])
    assert np.allclose(direct.convnd_points([f, g], ("centered", "centered", "hermitian"), pts),
                       h[tuple(pts.T)], atol=1e-12)


@pytest.mark.parametrize("kinds", [("complex", "complex"), ("centered", "centered"),
                                   ("centered", "centered", "hermitian")])
def test_explicit_fft_equals_direct(kinds):
    if kinds[-1] == "hermitian":
        f = inputs.hermitian_3d(6, 61).astype(np.complex128)
        g = inputs.hermitian_3d(6, 62).astype(np.complex128)
        Ns = [9, 9, 9]
    else:
        f, g = inputs.uniform_complex((2, 6, 7), 63)
        Ns = [12 if k == "complex" else 9 for k in kinds]
        Ns[1] = 14 if kinds[1] == "complex" else 11
    ref = direct.convnd([f, g], kinds)
    got = explicit.convnd_explicit([f, g], kinds, Ns)
    assert np.allclose(got, ref, atol=1e-11)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_basdevant_special_cases(kind):
    """Basdevant outputs against the binary product: u v is the product
    convolution; with v = 0 the second output is u*u; with u = v it vanishes;
    swapping u and v keeps u v and negates u^2 - v^2."""
    L = 19
    if kind == "hermitian":
        u, v, w = inputs.hermitian_1d(3, L, 71)
    else:
        u, v, w = inputs.uniform_complex((3, L), 71)
    b = direct.conv1d([u, v], kind, "basdevant2")
    assert b.shape == (2, len(u))
    assert np.allclose(b[0], direct.conv1d([u, v], kind), atol=1e-13)
    z = np.zeros_like(v)
    b0 = direct.conv1d([u, z], kind, "basdevant2")
    assert np.allclose(b0[1], direct.conv1d([u, u], kind), atol=1e-13) and not np.any(b0[0])
    assert np.allclose(direct.conv1d([u, u], kind, "basdevant2")[1], 0, atol=1e-13)
    bs = direct.conv1d([v, u], kind, "basdevant2")
    assert np.allclose(bs[0], b[0], atol=1e-13) and np.allclose(bs[1], -b[1], atol=1e-13)
    # 3D form: with w = 0 it holds the 2D form's outputs (and zeros)
    b3 = direct.conv1d([u, v, np.zeros_like(w)], kind, "basdevant3")
    assert b3.shape == (5, len(u))
    assert np.allclose(b3[0], b[0], atol=1e-13) and not np.any(b3[1]) and not np.any(b3[2])
    assert np.allclose(b3[3] - b3[4], b[1], atol=1e-13)


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
def test_mhd_special_cases(kind):
    """The MHD mult (traceless part of z-_i z+_j): with z+ = z- = u it holds the
    3D Basdevant outputs of u (T symmetric, so T_10, T_21, T_02 repeat T_01,
    T_12, T_20); swapping z+ and z- transposes T; z- = 0 gives zeros."""
    L = 17
    if kind == "hermitian":
        u = list(inputs.hermitian_1d(3, L, 61))
        w = list(inputs.hermitian_1d(3, L, 62))
    else:
        u = list(inputs.uniform_complex((3, L), 61))
        w = list(inputs.uniform_complex((3, L), 62))
    b3 = direct.conv1d(u, kind, "basdevant3")
    m = direct.conv1d(u + u, kind, "mhd3")
    assert m.shape == (8, len(u[0]))
    for k, b in ((0, 0), (3, 1), (4, 2), (6, 3), (7, 4)):     # T_01, T_12, T_20, T_00 - T_22, T_11 - T_22
        assert np.allclose(m[k], b3[b], atol=1e-13), (k, b)
    for a, b in ((0, 2), (3, 5), (4, 1)):                      # T_01 = T_10, T_12 = T_21, T_20 = T_02
        assert np.allclose(m[a], m[b], atol=1e-13)
    mw = direct.conv1d(u + w, kind, "mhd3")
    mt = direct.conv1d(w + u, kind, "mhd3")
    for a, b in ((0, 2), (1, 4), (3, 5)):                      # transposed off-diagonal entries
        assert np.allclose(mw[a], mt[b], atol=1e-13)
    assert np.allclose(mw[6], mt[6], atol=1e-13) and np.allclose(mw[7], mt[7], atol=1e-13)
    z = [np.zeros_like(x) for x in u]
    assert not np.any(direct.conv1d(u + z, kind, "mhd3"))


@pytest.mark.parametrize("mult", ["basdevant2", "basdevant3", "mhd3"])
def test_multi_output_batch_points_and_nd(mult):
    """B > 1: the batch, point and N-D forms agree with the 1D definition and
    the explicit FFT convolution, output by output."""
    A, B = direct.MULTS[mult], direct.OUTPUTS[mult]
    fs = [inputs.integer_complex((3, 9), 81 + a) for a in range(A)]
    for kind in ("complex", "centered"):
        ref = direct.conv1d_batch(fs, kind, mult)
        assert ref.shape == (B, 3, 9)
        for i in range(3):
            assert np.array_equal(ref[:, i], brute_1d([f[i] for f in fs], kind, mult))
        idx = np.array([0, 4, 8])
        pts = direct.conv1d_points([f[1] for f in fs], kind, idx, mult)
        assert np.array_equal(pts, ref[:, 1, idx])
    f2 = [inputs.uniform_complex((5, 4), 91 + a) for a in range(A)]
    kinds = ("centered", "complex")
    h = direct.convnd(f2, kinds, mult)
    assert h.shape == (B, 5, 4)
    got = explicit.convnd_explicit(f2, kinds, [8, 7], mult)
    assert np.allclose(got, h, atol=1e-12)
    pts = np.array([[0, 0], [2, 3], [4, 1]])
    assert np.allclose(direct.convnd_points(f2, kinds, pts, mult), h[(slice(None),) + tuple(pts.T)], atol=1e-12)
    f3 = [inputs.hermitian_3d(6, 95 + a).astype(np.complex128) for a in range(A)]
    k3 = ("centered", "centered", "hermitian")
    h3 = direct.convnd(f3, k3, mult)
    assert np.allclose(explicit.convnd_explicit(f3, k3, [9, 9, 9], mult), h3, atol=1e-11)


def test_basdevant_planted_sign_fails(monkeypatch):
    """A slip in the Basdevant terms (u^2 + v^2 for u^2 - v^2) breaks the
    brute-force pin."""
    fs = [inputs.integer_complex(7, 97 + a) for a in range(2)]
    ok = direct.conv1d(fs, "centered", "basdevant2")
    assert np.array_equal(ok, brute_1d(fs, "centered", "basdevant2"))
    monkeypatch.setitem(direct.MULT_TERMS, "basdevant2", (2, [[(0, 1, 1)], [(0, 0, 1), (1, 1, 1)]]))
    bad = direct.conv1d(fs, "centered", "basdevant2")
    assert not np.array_equal(bad, brute_1d(fs, "centered", "basdevant2"))
