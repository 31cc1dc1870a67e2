"""ctypes wrapper of direct_conv.c (the direct definition in plain C).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  ``build()`` compiles the
C file with gcc into oracle/_build/liboracle_direct.so.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import direct

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct_conv.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_direct.so")
_lib = None

KIND = {"complex": 0, "centered": 1, "hermitian": 2}
MULT = {"product": 0, "sum_pairs3": 1}


def build(force: bool = False) -> str:
    import fcntl
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    with open(os.path.join(os.path.dirname(_OUT), ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)   # one builder at a time (several processes may call this)
        try:
            if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
                tmp = _OUT + f".tmp{os.getpid()}"
                subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
                os.replace(tmp, _OUT)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_conv1d_batch.restype = ctypes.c_int
        _lib.oracle_conv1d_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int]
        _lib.oracle_conv1d_points.restype = ctypes.c_int
        _lib.oracle_conv1d_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p]
    return _lib


def _multi(fn, fs, mult, *args):
    """B > 1 outputs (the Basdevant forms): each output is a signed sum of
    binary product convolutions, computed by the C product one pair at a time."""
    A, terms = direct.MULT_TERMS[mult]
    assert len(fs) == A
    return np.stack([sum(c * fn([fs[i], fs[j]], *args) for i, j, c in t) for t in terms])


def conv1d_batch(fs, L: int, kind="complex", mult="product", nthreads=None) -> np.ndarray:
    """fs: list of A arrays of shape (count, n) -> (count, n) complex128 output,
    or (B, count, n) for a mult with B > 1 outputs."""
    if mult not in MULT:
        return _multi(lambda g: conv1d_batch(g, L, kind, "product", nthreads), fs, mult)
    lib = _load()
    fs = [np.ascontiguousarray(f, dtype=np.complex128) for f in fs]
    count = fs[0].shape[0]
    h = np.zeros_like(fs[0])
    ptrs = (ctypes.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    nt = nthreads or os.cpu_count() or 1
    rc = lib.oracle_conv1d_batch(KIND[kind], MULT[mult], int(L), int(count), ptrs, h.ctypes.data, int(nt))
    if rc != 0:
        raise ValueError("oracle_conv1d_batch rejected its arguments")
    return h


def conv1d_points(fs, L: int, idx, kind="complex", mult="product") -> np.ndarray:
    if mult not in MULT:
        return _multi(lambda g: conv1d_points(g, L, idx, kind, "product"), fs, mult)
    lib = _load()
    fs = [np.ascontiguousarray(f, dtype=np.complex128) for f in fs]
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(len(idx), dtype=np.complex128)
    ptrs = (ctypes.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    rc = lib.oracle_conv1d_points(KIND[kind], MULT[mult], int(L), ptrs, idx.ctypes.data, len(idx), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_conv1d_points rejected its arguments")
    return out
