"""Explicit zero-padded FFT convolution in FP64 (the paper's comparison method).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Explicit dealiasing pads every input with zeros to a length N >= M, takes
length-N FFTs, applies ``mult`` pointwise and inverse transforms (Section 1,
Section 7).  numpy's FFT is the FFT step.  For centered data the zero
padding is applied symmetrically by transforming at the centered offsets;
for Hermitian data the expanded symmetric array is used.  Used as the
full-field oracle of the multidimensional workloads, where the direct sum is
too slow, and pinned against the direct sum on small grids.
"""
from __future__ import annotations

import numpy as np

from .direct import MULT_TERMS, hermitian_expand_nd


def convnd_explicit(fs, kinds, Ns, mult="product", residues=None) -> np.ndarray:
    """N-D convolution by explicit padding to sizes Ns (one per axis).

    residues = (n, r_begin, r_end): only the frequencies k of axis 0 with
    k mod n in [r_begin, r_end) enter the inverse transform -- the part of the
    convolution that residues r_begin <= r < r_end of a hybrid plan with n
    residues on axis 0 compute (Section 2.2: residue r holds the padded
    frequencies q l + r, or q l + u n + r for p > 2, all of them = r mod n;
    frequency k in the paper's positive-exponent convention is numpy's bin
    -k mod N).  N[0] must be a multiple of n."""
    fs = [np.asarray(f, dtype=np.complex128) for f in fs]
    herm = kinds[-1] == "hermitian"
    if herm:
        H = fs[0].shape[-1]
        ex = [hermitian_expand_nd(f, f.shape[:-1]) for f in fs]
        lo = [-(fs[0].shape[a] // 2) if kinds[a] == "centered" else 0 for a in range(len(kinds) - 1)] + [-(H - 1)]
    else:
        ex = fs
        lo = [-(fs[0].shape[a] // 2) if kinds[a] == "centered" else 0 for a in range(len(kinds))]
    axes = tuple(range(len(kinds)))
    # place each array at its (possibly negative) centered offsets modulo N
    padded = []
    for e in ex:
        P = np.zeros(tuple(Ns), dtype=np.complex128)
        idx = np.ix_(*[np.mod(np.arange(e.shape[a]) + lo[a], Ns[a]) for a in axes])
        P[idx] = e
        padded.append(np.fft.fftn(P, axes=axes))
    A, terms = MULT_TERMS[mult]
    assert len(padded) == A
    out_lo = lo[:-1] + [0] if herm else lo
    out_shape = fs[0].shape
    idx = np.ix_(*[np.mod(np.arange(out_shape[a]) + out_lo[a], Ns[a]) for a in axes])
    keep = None
    if residues is not None:
        n, r0, r1 = residues
        assert Ns[0] % n == 0
        k = np.mod(-np.arange(Ns[0]), Ns[0])   # paper frequency of numpy bin j along axis 0
        keep = ((k % n >= r0) & (k % n < r1)).reshape((-1,) + (1,) * (len(kinds) - 1))
    outs = []
    for t in terms:   # mult, pointwise on the padded spectra
        spec = sum(c * padded[i] * padded[j] for i, j, c in t)
        if keep is not None:
            spec = np.where(keep, spec, 0)
        outs.append(np.fft.ifftn(spec, axes=axes)[idx])
    return outs[0] if len(outs) == 1 else np.stack(outs)
