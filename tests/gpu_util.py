"""Helpers shared by the GPU parity tests: device transfer and error norms."""
import numpy as np


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    nr = np.linalg.norm(ref)
    if nr == 0:
        return float(np.linalg.norm(got))
    return float(np.linalg.norm(got - ref) / nr)


def rel_l2_rows(got, ref):
    """Largest rel-L2 over the instances of a batch: every axis but the last
    indexes an instance, the last one runs along it.  A wrong instance, or a
    wrong stretch of one, cannot hide under the norm of the others."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    if ref.ndim <= 1:
        return rel_l2(got, ref)
    g = got.reshape(-1, got.shape[-1])
    r = ref.reshape(-1, ref.shape[-1])
    return max(rel_l2(a, b) for a, b in zip(g, r))


def to_dev(x, dtype):
    import torch
    npdt = np.complex64 if dtype == "f32" else np.complex128
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).astype(npdt))).cuda()


def run_conv(hd, plan, fs, count=None, stride=None, h=None):
    """fs: list of A numpy arrays, shape (count, n) or (n,).  Returns numpy output."""
    import torch
    dts = [to_dev(f, plan.dtype) for f in fs]
    out = torch.zeros_like(dts[0]) if h is None else h
    if dts[0].dim() == 1 and count is None:
        plan.convolve(dts, out)
    else:
        cnt = dts[0].shape[0] if count is None else count
        st = dts[0].shape[-1] if stride is None else stride
        plan.convolve_batched(dts, out, cnt, st)
    torch.cuda.synchronize()
    return out.cpu().numpy()
