"""Direct (O(L^2)) FP64 linear convolutions: the definition the method must reproduce.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's general convolution (Section 2) maps A inputs of length L, zero
padded to at least the dealiasing length M, to B outputs whose DFT is a
pointwise function ``mult`` of the inputs' DFTs.  For a product of DFTs the
result is the linear convolution (f*g)_j = sum_i f_i g_{j-i} (Section 2); the
convolution returns L outputs (Alg. convolve and convolveX return one value per
input index).  Once the padding dealiases, the hybrid method's result does not
depend on m, p or q, so the oracle is the direct sum, written out:

  complex   (Section 2):   h_j = sum_{i=0}^{j} f_i g_{j-i},  j = 0..L-1
  centered  (Section 3):   stored j <-> centered c = j - floor(L/2);
                           h_c = sum_{c'} f_{c'} g_{c-c'} over the stored range
  Hermitian (Section 4):   stored c = 0..ceil(L/2)-1 of an array with
                           f_{-c} = conj(f_c); the expanded (odd length
                           2*ceil(L/2)-1) array is convolved as centered and
                           the non-negative half is returned.  Im f_0 is ignored.

Multiplication operators (``mult``); output b is a signed sum of pairwise
convolutions f_i*f_j, since a pointwise product of DFTs is the DFT of a
convolution:
  "product"     A=2, B=1:  F1*F2                    -> f1*f2
  "sum_pairs3"  A=3, B=1:  F1F2 + F2F3 + F3F1       -> f1*f2 + f2*f3 + f3*f1
  "basdevant2"  A=2, B=2:  (F1F2, F1^2 - F2^2)      -> (f1*f2, f1*f1 - f2*f2)
  "basdevant3"  A=3, B=5:  (F1F2, F2F3, F3F1, F1^2 - F3^2, F2^2 - F3^2)
  "mhd3"        A=6, B=8:  inputs the Elsasser components (Z+_0, Z+_1, Z+_2,
                Z-_0, Z-_1, Z-_2); outputs the eight entries of the traceless
                part of T_ij = Z-_i Z+_j: T_01, T_02, T_10, T_12, T_20, T_21,
                T_00 - T_22, T_11 - T_22
The Basdevant products are the nonlinear terms of incompressible
Navier-Stokes in Basdevant's form, which Section 9 counts as A = B = 2 in two
dimensions and A = 3, B = 5 in three (inputs: the velocity components).
Section 9 gives A = 6, B = 8 for incompressible 3D magnetohydrodynamics
without the form; "mhd3" is the reading that yields those counts: in
Elsasser variables z+- = u +- b the nonlinear term is the divergence of the
flux tensor z-_i z+_j, whose trace (like the velocity tensor's in
Basdevant's form) is absorbed by the pressure gradient, leaving 9 - 1 = 8
independent products of the 6 transformed components.  With
B > 1 the functions below return the B outputs stacked on a new first axis.
On integer-valued inputs every product and partial sum is an integer below
2^53, so these FP64 sums are exact.
"""
from __future__ import annotations

import itertools

import numpy as np

KINDS = ("complex", "centered", "hermitian")
# mult -> (A, terms): output b = sum of c * (f_i * f_j) over (i, j, c) in terms[b]
MULT_TERMS = {
    "product": (2, [[(0, 1, 1)]]),
    "sum_pairs3": (3, [[(0, 1, 1), (1, 2, 1), (2, 0, 1)]]),
    "basdevant2": (2, [[(0, 1, 1)], [(0, 0, 1), (1, 1, -1)]]),
    "basdevant3": (3, [[(0, 1, 1)], [(1, 2, 1)], [(2, 0, 1)], [(0, 0, 1), (2, 2, -1)], [(1, 1, 1), (2, 2, -1)]]),
    # T_ij = z-_i z+_j with z+_j = f_j and z-_i = f_{3+i}
    "mhd3": (6, [[(3, 1, 1)], [(3, 2, 1)], [(4, 0, 1)], [(4, 2, 1)], [(5, 0, 1)], [(5, 1, 1)],
                 [(3, 0, 1), (5, 2, -1)], [(4, 1, 1), (5, 2, -1)]]),
}
MULTS = {k: v[0] for k, v in MULT_TERMS.items()}             # inputs A
OUTPUTS = {k: len(v[1]) for k, v in MULT_TERMS.items()}      # outputs B


def full_linear(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Full linear convolution (length La+Lb-1) written as a sum of shifted copies."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    out = np.zeros(a.shape[-1] + b.shape[-1] - 1, dtype=np.complex128)
    Lb = b.shape[-1]
    for i in range(a.shape[-1]):
        out[i:i + Lb] += a[i] * b
    return out


def hermitian_expand(f: np.ndarray) -> np.ndarray:
    """Stored half f_0..f_{H-1} -> symmetric array over c = -(H-1)..(H-1)."""
    f = np.asarray(f, dtype=np.complex128).copy()
    f[0] = f[0].real
    return np.concatenate([np.conj(f[:0:-1]), f])


def _outputs(fs, mult, conv):
    """The B outputs of ``mult``: signed sums of conv(f_i, f_j), stacked when B > 1."""
    if mult not in MULT_TERMS:
        raise ValueError(mult)
    A, terms = MULT_TERMS[mult]
    assert len(fs) == A
    outs = [sum(c * conv(fs[i], fs[j]) for i, j, c in t) for t in terms]
    return outs[0] if len(outs) == 1 else np.stack(outs)


def conv1d(fs, kind: str = "complex", mult: str = "product") -> np.ndarray:
    """One 1D convolution of the A stored inputs ``fs``; returns the stored
    output (shape (B, ...) when B > 1)."""
    fs = [np.asarray(f, dtype=np.complex128) for f in fs]
    if kind == "hermitian":
        H = fs[0].shape[-1]
        ex = [hermitian_expand(f) for f in fs]
        full = _outputs(ex, mult, full_linear)
        # expanded length Le = 2H-1, centered offset H-1; full index k <-> c = k - 2(H-1)
        return full[..., 2 * (H - 1): 2 * (H - 1) + H]
    L = fs[0].shape[-1]
    full = _outputs(fs, mult, full_linear)
    if kind == "complex":
        return full[..., :L]
    if kind == "centered":
        Hc = L // 2
        return full[..., Hc:Hc + L]
    raise ValueError(kind)


def conv1d_batch(fs, kind="complex", mult="product") -> np.ndarray:
    """Row-wise conv1d over a batch: fs is a list of A arrays of shape (count, L);
    returns (count, L), or (B, count, L) when B > 1."""
    count = fs[0].shape[0]
    out = np.stack([conv1d([f[b] for f in fs], kind, mult) for b in range(count)])
    return out if OUTPUTS[mult] == 1 else np.moveaxis(out, 1, 0)


# ---------------------------------------------------------------------------
# N-D separable definition (Section 5): the N-D linear convolution, restricted
# per axis like the 1D kinds.  Axis kinds: "complex" or "centered"; the last
# axis may be "hermitian", in which case the input is Hermitian symmetric on
# the whole array, f(-x) = conj f(x), and only the non-negative half of the
# last axis is stored (Section 5, last paragraphs).
# ---------------------------------------------------------------------------

def hermitian_expand_nd(f: np.ndarray, outer_lengths) -> np.ndarray:
    """Expand a stored N-D Hermitian array (outer axes centered) to the full array.

    Outer axis i has stored length L_i with centered index j - L_i//2; the last
    axis stores c = 0..H-1.  The full array covers, for each outer axis, the
    stored range, and c = -(H-1)..(H-1) on the last axis; a value whose mirror
    index lies outside the stored range is taken as zero.
    """
    f = np.asarray(f, dtype=np.complex128)
    H = f.shape[-1]
    outer = f.shape[:-1]
    full = np.zeros(outer + (2 * H - 1,), dtype=np.complex128)
    full[..., H - 1:] = f
    # mirror: full(x, -z) = conj f(-x, z) for z = 1..H-1
    idx = []
    for L in outer:
        c = np.arange(L) - L // 2
        m = -c + L // 2
        idx.append(m)
    valid = np.ones(outer, dtype=bool)
    grids = np.meshgrid(*idx, indexing="ij")
    for L, g in zip(outer, grids):
        valid &= (g >= 0) & (g < L)
    src = tuple(np.clip(g, 0, L - 1) for g, L in zip(grids, outer))
    mirrored = np.conj(f[src])               # conj f(-x, z), shape outer + (H,)
    mirrored[~valid] = 0
    full[..., :H - 1] = mirrored[..., :0:-1]  # z = -(H-1)..-1
    # the z = 0 plane is taken as stored (it must already be symmetric)
    return full


def _full_linear_nd(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    out_shape = tuple(x + y - 1 for x, y in zip(a.shape, b.shape))
    out = np.zeros(out_shape, dtype=np.complex128)
    for idx in itertools.product(*[range(n) for n in a.shape]):
        v = a[idx]
        if v == 0:
            continue
        sl = tuple(slice(i, i + n) for i, n in zip(idx, b.shape))
        out[sl] += v * b
    return out


def convnd(fs, kinds, mult="product") -> np.ndarray:
    """Direct N-D convolution (O(prod L^2)); for small grids only."""
    fs = [np.asarray(f, dtype=np.complex128) for f in fs]
    if kinds[-1] == "hermitian":
        H = fs[0].shape[-1]
        ex = [hermitian_expand_nd(f, f.shape[:-1]) for f in fs]
        full = _outputs(ex, mult, _full_linear_nd)
        sl = [Ellipsis]
        for ax, k in enumerate(kinds[:-1]):
            L = fs[0].shape[ax]
            sl.append(slice(L // 2, L // 2 + L) if k == "centered" else slice(0, L))
        sl.append(slice(2 * (H - 1), 2 * (H - 1) + H))
        return full[tuple(sl)]
    full = _outputs(fs, mult, _full_linear_nd)
    sl = [Ellipsis]
    for ax, k in enumerate(kinds):
        L = fs[0].shape[ax]
        sl.append(slice(L // 2, L // 2 + L) if k == "centered" else slice(0, L))
    return full[tuple(sl)]


def convnd_points(fs, kinds, points, mult="product") -> np.ndarray:
    """Exact direct evaluation of selected output points of the N-D convolution.

    ``points`` is an (npts, ndim) integer array of STORED output indices.  Each
    point costs O(prod L): h(c) = sum_{c'} f(c') g(c - c') over the stored
    (expanded, for Hermitian) ranges.
    """
    fs = [np.asarray(f, dtype=np.complex128) for f in fs]
    nd = len(kinds)
    herm = kinds[-1] == "hermitian"
    if herm:
        H = fs[0].shape[-1]
        ex = [hermitian_expand_nd(f, f.shape[:-1]) for f in fs]
        lo = [-(fs[0].shape[a] // 2) if kinds[a] == "centered" else 0 for a in range(nd - 1)] + [-(H - 1)]
        out_lo = lo[:-1] + [0]
    else:
        ex = fs
        lo = [-(fs[0].shape[a] // 2) if kinds[a] == "centered" else 0 for a in range(nd)]
        out_lo = lo
    shape = ex[0].shape
    A, terms = MULT_TERMS[mult]
    assert len(ex) == A
    res = np.zeros((len(terms), len(points)), dtype=np.complex128)
    for pi, pt in enumerate(np.asarray(points)):
        c = [int(pt[a]) + out_lo[a] for a in range(nd)]       # centered output index
        # c' ranges over the stored range of axis a: lo_a .. lo_a + n_a - 1
        # c - c' must be in the same range -> c' in [c - (lo+n-1), c - lo]
        sl_a, sl_b = [], []
        empty = False
        for a in range(nd):
            n = shape[a]
            c1 = max(lo[a], c[a] - (lo[a] + n - 1))
            c2 = min(lo[a] + n - 1, c[a] - lo[a])
            if c1 > c2:
                empty = True
                break
            sl_a.append(slice(c1 - lo[a], c2 - lo[a] + 1))
            # g index (c - c') - lo runs from c - c1 - lo down to c - c2 - lo
            sl_b.append(slice(c[a] - c1 - lo[a], c[a] - c2 - lo[a] - 1 if c[a] - c2 - lo[a] - 1 >= 0 else None, -1))
        if empty:
            continue
        for b, t in enumerate(terms):
            res[b, pi] = sum(c * np.sum(ex[i][tuple(sl_a)] * ex[j][tuple(sl_b)]) for i, j, c in t)
    return res[0] if len(terms) == 1 else res


def conv1d_points(fs, kind, points, mult="product") -> np.ndarray:
    """Selected stored output indices of one 1D convolution, O(L) per point."""
    return convnd_points([np.asarray(f) for f in fs], (kind,), np.asarray(points).reshape(-1, 1), mult)
