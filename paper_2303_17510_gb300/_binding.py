"""ctypes binding of libhd.so (argument marshalling only).

Every computation runs in the CUDA library.  Importing this module loads
``_build/libhd.so`` and raises ``ImportError`` when it is missing: there is
no fallback of any kind.  Build it with ``python -m paper_2303_17510_gb300.build``
or ``__graft_entry__.build()``.

Tensors are torch CUDA tensors (complex64 for f32 plans, complex128 for f64
plans); only their ``data_ptr()`` and the current CUDA stream handle cross the
boundary.  Raw integer device addresses are accepted too.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhd.so not built ({LIB_PATH}); run paper_2303_17510_gb300.build.build()")

lib = ctypes.CDLL(LIB_PATH)

KIND = {"complex": 0, "centered": 1, "hermitian": 2}
DTYPE = {"f32": 0, "f64": 1}
MULT = {"product": 0, "sum_pairs3": 1, "basdevant2": 2, "basdevant3": 3, "mhd3": 4}
PLAN_NO_WORK_BUFFER = 1   # HD_PLAN_NO_WORK_BUFFER
MULT_AB = {"product": (2, 1), "sum_pairs3": (3, 1), "basdevant2": (2, 2), "basdevant3": (3, 5), "mhd3": (6, 8)}   # inputs A, outputs B


def _mult_of(A, B, mult):
    """The mult name (from (A, B) when not given) and B (from the mult when
    not given); the library validates the counts against the mult."""
    if mult is None:
        mult = {2: "basdevant2", 5: "basdevant3", 8: "mhd3"}.get(B) or ("product" if A == 2 else "sum_pairs3")
    if B is None:
        B = MULT_AB[mult][1]
    return mult, A, B
STATUS = {0: "HD_OK", 1: "HD_ERR_INVALID", 2: "HD_ERR_UNSUPPORTED", 3: "HD_ERR_NOMEM", 4: "HD_ERR_CUDA",
          5: "HD_ERR_TIMEOUT", 6: "HD_ERR_ALIASED", 7: "HD_ERR_SCRATCH_LIMIT"}
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p


class hd_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("L", _i64 * 3), ("M", _i64 * 3), ("A", ctypes.c_int), ("B", ctypes.c_int),
                ("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("mult", ctypes.c_int), ("m", _i64 * 3),
                ("p", _i64 * 3), ("q", _i64 * 3), ("D", ctypes.c_int * 3), ("row_pitch", _i64 * 3),
                ("flags", ctypes.c_int)]


class hd_candidate(ctypes.Structure):
    _fields_ = [("m", _i64), ("p", _i64), ("q", _i64), ("D", ctypes.c_int), ("S", _i64), ("n", _i64),
                ("E", ctypes.c_int), ("minb", ctypes.c_int), ("comp", ctypes.c_int), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HdError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        self.name = STATUS.get(self.code, str(code))
        super().__init__(f"{where}: {lib.hd_status_string(self.code).decode()}")


def _sig(name, res, args):
    fn = getattr(lib, name)
    fn.restype = res
    fn.argtypes = args
    return fn


_sig("hd_status_string", ctypes.c_char_p, [ctypes.c_int])
_sig("hd_derive_params", ctypes.c_int, [ctypes.c_int, _i64, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                        ctypes.POINTER(_i64)])
_sig("hd_dealias_bound", _i64, [ctypes.c_int, ctypes.c_int, _i64])
_sig("hd_plan_create", ctypes.c_int, [ctypes.POINTER(_vp), _i64, _i64, ctypes.c_int, ctypes.c_int, _i64, _i64, _i64,
                                      ctypes.c_int])
_sig("hd_plan_create_ex", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(hd_desc)])
_sig("hd_convolve", ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp])
_sig("hd_convolve_batched", ctypes.c_int, [_vp, _i64, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64, _vp])
_sig("hd_convolve_residues", ctypes.c_int, [_vp, _i64, _i64, _i64, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64,
                                            _vp])
_sig("hd_plan_get_params", ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)])
_sig("hd_forward_residue", ctypes.c_int, [_vp, _vp, _i64, _vp, _vp])
_sig("hd_plan_get_axis_params", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                               ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64),
                                               ctypes.POINTER(_i64)])
_sig("hd_plan_destroy", ctypes.c_int, [_vp])
_sig("hd_device_status", ctypes.c_int, [])
_sig("hd_enumerate_candidates", ctypes.c_int, [ctypes.POINTER(hd_desc), ctypes.POINTER(hd_candidate), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)])
_sig("hd_autotune", ctypes.c_int, [ctypes.POINTER(hd_desc), _i64, ctypes.c_int, ctypes.POINTER(hd_candidate),
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(hd_candidate)])
_sig("hd_plan_create_candidate", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(hd_desc),
                                                ctypes.POINTER(hd_candidate)])
_sig("hd_tune_cache_put", ctypes.c_int, [ctypes.POINTER(hd_desc), ctypes.POINTER(hd_candidate)])
_sig("hd_tune_cache_get", ctypes.c_int, [ctypes.POINTER(hd_desc), ctypes.POINTER(hd_candidate)])
_sig("hd_tune_cache_clear", ctypes.c_int, [])
_sig("hd_alu_peak", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)])
_sig("hd_convolve_batched_noalloc", ctypes.c_int, [_vp, _i64, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64, _vp])
_sig("hd_mlp_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int)])
_sig("hd_mlp_num_params", _i64, [_vp])
_sig("hd_mlp_set_params", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)])
_sig("hd_mlp_get_params", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)])
_sig("hd_mlp_forward", ctypes.c_int, [_vp, _vp, _i64, _vp, _vp])
_sig("hd_mlp_gradients", ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float), _vp])
_sig("hd_mlp_train_step", ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _vp])
_sig("hd_mlp_destroy", ctypes.c_int, [_vp])
_sig("hd_selector_features", ctypes.c_int, [ctypes.POINTER(hd_desc), ctypes.POINTER(hd_candidate),
                                            ctypes.POINTER(ctypes.c_float)])
_sig("hd_selector_install", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_int])
_sig("hd_selector_clear", ctypes.c_int, [])
_sig("hd_selector_choose", ctypes.c_int, [ctypes.POINTER(hd_desc), ctypes.POINTER(hd_candidate),
                                          ctypes.POINTER(ctypes.c_int)])
_sig("hd_ragged_create", ctypes.c_int, [ctypes.POINTER(_vp), _i64, ctypes.POINTER(hd_desc)])
_sig("hd_ragged_create_candidates", ctypes.c_int, [ctypes.POINTER(_vp), _i64, ctypes.POINTER(hd_desc),
                                                   ctypes.POINTER(hd_candidate)])
_sig("hd_ragged_bind", ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)])
_sig("hd_ragged_run", ctypes.c_int, [_vp, _vp])
_sig("hd_ragged_status", ctypes.c_int, [_vp])
_sig("hd_ragged_get_params", ctypes.c_int, [_vp, _i64, ctypes.POINTER(hd_candidate)])
_sig("hd_ragged_set_wait_limit", ctypes.c_int, [_vp, _i64])
_sig("hd_ragged_inject_stall", ctypes.c_int, [_vp, _i64])


def _check(rc, where):
    if rc != 0:
        raise HdError(rc, where)


def device_status() -> str:
    """Synchronizes the current device; "HD_ERR_TIMEOUT" if a persistent batched
    kernel's bounded wait ran out since the last call, else "HD_OK"."""
    return STATUS[lib.hd_device_status()]


PEAK_KINDS = {"f32": 0, "f64": 1, "f32x2": 2}


def alu_peak(kind="f32") -> float:
    """Measured FMA throughput of the current device in TFLOP/s: "f32" (scalar
    FP32 FMA), "f64" or "f32x2" (packed two-lane FP32 FMA)."""
    v = ctypes.c_double()
    _check(lib.hd_alu_peak(PEAK_KINDS[kind], ctypes.byref(v)), "hd_alu_peak")
    return v.value


def status_string(code: int) -> str:
    return lib.hd_status_string(int(code)).decode()


def derive_params(kind: str, L: int, M: int, m: int):
    p, q, n = _i64(), _i64(), _i64()
    _check(lib.hd_derive_params(KIND[kind], L, M, m, ctypes.byref(p), ctypes.byref(q), ctypes.byref(n)),
           "hd_derive_params")
    return p.value, q.value, n.value


def dealias_bound(kind: str, L: int, mult: str = "product") -> int:
    return int(lib.hd_dealias_bound(KIND[kind], MULT[mult], L))


def _ptr(x) -> int:
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_desc(L, M, A=2, B=None, m=0, p=0, q=0, D=0, kind="complex", dtype="f32", mult=None, ndim=None, flags=0):
    mult, A, B = _mult_of(A, B, mult)
    Ls = list(L) if isinstance(L, (list, tuple)) else [L]
    Ms = list(M) if isinstance(M, (list, tuple)) else [M]
    ms = list(m) if isinstance(m, (list, tuple)) else [m] * len(Ls)
    ps = list(p) if isinstance(p, (list, tuple)) else [p] * len(Ls)
    qs = list(q) if isinstance(q, (list, tuple)) else [q] * len(Ls)
    Ds = list(D) if isinstance(D, (list, tuple)) else [D] * len(Ls)
    nd = ndim or len(Ls)
    d = hd_desc()
    d.ndim = nd
    for i in range(nd):
        d.L[i], d.M[i], d.m[i], d.p[i], d.q[i], d.D[i] = Ls[i], Ms[i], ms[i], ps[i], qs[i], Ds[i]
    d.A, d.B, d.kind, d.dtype, d.mult = A, B, KIND[kind], DTYPE[dtype], MULT[mult]
    d.flags = int(flags)
    return d


def enumerate_candidates(**kw):
    """Legal, supported parameter candidates of a 1D description (host only)."""
    d = make_desc(**kw)
    n = ctypes.c_int()
    _check(lib.hd_enumerate_candidates(ctypes.byref(d), None, 0, ctypes.byref(n)), "hd_enumerate_candidates")
    arr = (hd_candidate * max(1, n.value))()
    _check(lib.hd_enumerate_candidates(ctypes.byref(d), arr, n.value, ctypes.byref(n)), "hd_enumerate_candidates")
    return [arr[i].as_dict() for i in range(n.value)]


def autotune(count, reps=5, **kw):
    """Times every candidate for a batch of `count`; returns (best, all) as dicts
    and records the best in the library's tuning cache."""
    d = make_desc(**kw)
    arr = (hd_candidate * 256)()
    n = ctypes.c_int()
    best = hd_candidate()
    _check(lib.hd_autotune(ctypes.byref(d), int(count), int(reps), arr, 256, ctypes.byref(n), ctypes.byref(best)),
           "hd_autotune")
    return best.as_dict(), [arr[i].as_dict() for i in range(min(n.value, 256))]


def tune_cache_put(cand: dict, **kw):
    d = make_desc(**kw)
    c = hd_candidate(**{k: cand[k] for k, _ in hd_candidate._fields_})
    _check(lib.hd_tune_cache_put(ctypes.byref(d), ctypes.byref(c)), "hd_tune_cache_put")


def tune_cache_get(**kw):
    d = make_desc(**kw)
    c = hd_candidate()
    if lib.hd_tune_cache_get(ctypes.byref(d), ctypes.byref(c)) != 0:
        return None
    return c.as_dict()


def tune_cache_clear():
    lib.hd_tune_cache_clear()


class Plan:
    """A convolution plan (owns device twiddle tables and scratch)."""

    def __init__(self, L, M, A=2, B=None, m=0, p=0, q=0, D=0, kind="complex", dtype="f32", mult=None, ndim=None,
                 candidate=None, flags=0):
        """flags: 0, or PLAN_NO_WORK_BUFFER (a 1D split-path plan without its own
        work buffer, for convolve_batched_noalloc only)."""
        mult, A, B = _mult_of(A, B, mult)
        d = make_desc(L, M, A, B, m, p, q, D, kind, dtype, mult, ndim, flags)
        self._h = _vp()
        if candidate is None:
            _check(lib.hd_plan_create_ex(ctypes.byref(self._h), ctypes.byref(d)), "hd_plan_create_ex")
        else:
            c = hd_candidate(**{k: candidate[k] for k, _ in hd_candidate._fields_})
            _check(lib.hd_plan_create_candidate(ctypes.byref(self._h), ctypes.byref(d), ctypes.byref(c)),
                   "hd_plan_create_candidate")
        self.L = list(L) if isinstance(L, (list, tuple)) else [L]
        self.M = list(M) if isinstance(M, (list, tuple)) else [M]
        self.A, self.B = A, B
        self.kind, self.dtype, self.mult, self.ndim = kind, dtype, mult, d.ndim

    @property
    def handle(self) -> int:
        return self._h.value

    def params(self):
        m, p, q, D, s = _i64(), _i64(), _i64(), ctypes.c_int(), ctypes.c_size_t()
        _check(lib.hd_plan_get_params(self._h, ctypes.byref(m), ctypes.byref(p), ctypes.byref(q), ctypes.byref(D),
                                      ctypes.byref(s)), "hd_plan_get_params")
        return dict(m=m.value, p=p.value, q=q.value, D=D.value, scratch_bytes=s.value)

    def axis_params(self, axis):
        m, p, q, S, n = _i64(), _i64(), _i64(), _i64(), _i64()
        D = ctypes.c_int()
        _check(lib.hd_plan_get_axis_params(self._h, int(axis), ctypes.byref(m), ctypes.byref(p), ctypes.byref(q),
                                           ctypes.byref(D), ctypes.byref(S), ctypes.byref(n)), "hd_plan_get_axis_params")
        return dict(m=m.value, p=p.value, q=q.value, D=D.value, S=S.value, n=n.value)

    def convolve(self, fs, h, stream=None):
        """One convolution: fs = A device arrays (tensors or addresses), h = the
        output (or a list of the B outputs)."""
        fa = (_vp * self.A)(*[_ptr(x) for x in fs])
        ha = (_vp * self.B)(*[_ptr(h)] if not isinstance(h, (list, tuple)) else [_ptr(x) for x in h])
        _check(lib.hd_convolve(self._h, fa, ha, _stream(stream)), "hd_convolve")

    def convolve_batched(self, fs, h, count, batch_stride, stream=None):
        fa = (_vp * self.A)(*[_ptr(x) for x in fs])
        ha = (_vp * self.B)(*[_ptr(h)] if not isinstance(h, (list, tuple)) else [_ptr(x) for x in h])
        _check(lib.hd_convolve_batched(self._h, int(count), fa, ha, int(batch_stride), _stream(stream)),
               "hd_convolve_batched")

    @property
    def residues(self) -> int:
        """n: the residue count of the outermost axis (the range of convolve_residues)."""
        return self.axis_params(0)["n"]

    def convolve_residues(self, fs, h, r_begin, r_end, count=1, batch_stride=0, stream=None):
        """Partial sums over residues r_begin <= r < r_end of the outermost axis
        (hd_convolve_residues); over a partition of [0, n) they add up to the
        convolution."""
        fa = (_vp * self.A)(*[_ptr(x) for x in fs])
        ha = (_vp * self.B)(*[_ptr(h)] if not isinstance(h, (list, tuple)) else [_ptr(x) for x in h])
        _check(lib.hd_convolve_residues(self._h, int(r_begin), int(r_end), int(count), fa, ha, int(batch_stride),
                                        _stream(stream)), "hd_convolve_residues")

    def convolve_batched_noalloc(self, fs, h, count, batch_stride, stream=None):
        """As convolve_batched, over the library's fixed work buffer (no device allocation)."""
        fa = (_vp * self.A)(*[_ptr(x) for x in fs])
        ha = (_vp * self.B)(*[_ptr(h)] if not isinstance(h, (list, tuple)) else [_ptr(x) for x in h])
        _check(lib.hd_convolve_batched_noalloc(self._h, int(count), fa, ha, int(batch_stride), _stream(stream)),
               "hd_convolve_batched_noalloc")

    def forward_residue(self, f, r, out, stream=None):
        _check(lib.hd_forward_residue(self._h, _ptr(f), int(r), _ptr(out), _stream(stream)), "hd_forward_residue")

    def close(self):
        if self._h and self._h.value:
            lib.hd_plan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class RaggedPlan:
    """A ragged batch of 1D convolutions run by one persistent kernel launch
    replayed from a CUDA graph.  `descs`: list of dicts with L, M, A (2 or 3),
    kind ("complex" or "centered") and optionally m, p, q."""

    def __init__(self, descs, candidates=None):
        n = len(descs)
        arr = (hd_desc * n)()
        for i, d in enumerate(descs):
            arr[i] = make_desc(d["L"], d["M"], A=d.get("A", 2), m=d.get("m", 0), p=d.get("p", 0), q=d.get("q", 0),
                               kind=d.get("kind", "complex"), dtype="f32")
        self._h = _vp()
        if candidates is None:
            _check(lib.hd_ragged_create(ctypes.byref(self._h), n, arr), "hd_ragged_create")
        else:
            ca = (hd_candidate * n)(*[hd_candidate(**{k: c[k] for k, _ in hd_candidate._fields_}) for c in candidates])
            _check(lib.hd_ragged_create_candidates(ctypes.byref(self._h), n, arr, ca), "hd_ragged_create_candidates")
        self.n = n
        self.descs = descs

    @property
    def handle(self) -> int:
        return self._h.value

    def bind(self, fs, hs):
        """fs[i]: list of A device arrays of instance i; hs[i]: its output."""
        fa = (_vp * (3 * self.n))()
        for i, row in enumerate(fs):
            for a, x in enumerate(row):
                fa[3 * i + a] = _ptr(x)
        ha = (_vp * self.n)(*[_ptr(x) for x in hs])
        _check(lib.hd_ragged_bind(self._h, fa, ha), "hd_ragged_bind")

    def run(self, stream=None):
        _check(lib.hd_ragged_run(self._h, _stream(stream)), "hd_ragged_run")

    def status(self):
        """Synchronizes the last run; returns the status name."""
        return STATUS[lib.hd_ragged_status(self._h)]

    def params(self, i):
        c = hd_candidate()
        _check(lib.hd_ragged_get_params(self._h, int(i), ctypes.byref(c)), "hd_ragged_get_params")
        return c.as_dict()

    def set_wait_limit(self, ns):
        _check(lib.hd_ragged_set_wait_limit(self._h, int(ns)), "hd_ragged_set_wait_limit")

    def inject_stall(self, i):
        _check(lib.hd_ragged_inject_stall(self._h, int(i)), "hd_ragged_inject_stall")

    def close(self):
        if self._h and self._h.value:
            lib.hd_plan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


SELECTOR_FEATURES = 13


def selector_features(cand, **kw):
    d = make_desc(**kw)
    c = hd_candidate(**{k: cand[k] for k, _ in hd_candidate._fields_})
    out = (ctypes.c_float * SELECTOR_FEATURES)()
    _check(lib.hd_selector_features(ctypes.byref(d), ctypes.byref(c), out), "hd_selector_features")
    return list(out)


class MLP:
    """Device MLP (tanh hidden layers, linear scalar output) trained with the
    library's kernels.  dims: layer sizes, the last one 1."""

    def __init__(self, dims):
        self.dims = list(dims)
        arr = (ctypes.c_int * len(dims))(*dims)
        self._h = _vp()
        _check(lib.hd_mlp_create(ctypes.byref(self._h), len(dims) - 1, arr), "hd_mlp_create")
        self.nparams = int(lib.hd_mlp_num_params(self._h))

    @property
    def handle(self):
        return self._h.value

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        _check(lib.hd_mlp_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "hd_mlp_set_params")

    def get_params(self):
        import numpy as np
        a = np.zeros(self.nparams, dtype=np.float32)
        _check(lib.hd_mlp_get_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "hd_mlp_get_params")
        return a

    def forward(self, X, Y, stream=None):
        _check(lib.hd_mlp_forward(self._h, _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)), "hd_mlp_forward")

    def gradients(self, X, t, stream=None):
        import numpy as np
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib.hd_mlp_gradients(self._h, _ptr(X), _ptr(t), int(X.shape[0]), ctypes.byref(loss),
                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(stream)),
               "hd_mlp_gradients")
        return float(loss.value), g

    def train_step(self, X, t, lr, stream=None, want_loss=False):
        loss = ctypes.c_float()
        _check(lib.hd_mlp_train_step(self._h, _ptr(X), _ptr(t), int(X.shape[0]), float(lr),
                                     ctypes.byref(loss) if want_loss else None, _stream(stream)), "hd_mlp_train_step")
        return float(loss.value) if want_loss else None

    def close(self):
        if self._h and self._h.value:
            lib.hd_mlp_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selector_install(models, tau=0.05, sigma=0.25, fallback=True):
    arr = (_vp * len(models))(*[m.handle for m in models])
    _check(lib.hd_selector_install(arr, len(models), float(tau), float(sigma), 1 if fallback else 0),
           "hd_selector_install")


def selector_clear():
    lib.hd_selector_clear()


def selector_choose(**kw):
    d = make_desc(**kw)
    c = hd_candidate()
    conf = ctypes.c_int()
    _check(lib.hd_selector_choose(ctypes.byref(d), ctypes.byref(c), ctypes.byref(conf)), "hd_selector_choose")
    return c.as_dict(), bool(conf.value)
