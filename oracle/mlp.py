"""FP64 reference of the parameter-selector MLP (forward, loss, gradients, Adam).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The selector is not in the
paper; this is the textbook definition of a fully connected network that the
GPU training kernels must reproduce:

    h_0 = x;   z_l = h_l W_l^T + b_l;   h_{l+1} = tanh(z_l) (hidden layers),
    y = z_{K-1} (linear output, one value);   loss = mean((y - t)^2).

Gradients by reverse-mode differentiation written out layer by layer; Adam as
in Kingma & Ba (2015) with bias correction.
"""
from __future__ import annotations

import numpy as np


def forward(params, X):
    """params: list of (W, b); returns (outputs, cache of (h_l, z_l))."""
    h = np.asarray(X, dtype=np.float64)
    cache = []
    K = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        cache.append((h, z))
        h = np.tanh(z) if l < K - 1 else z
    return h[:, 0], cache


def loss(params, X, t):
    y, _ = forward(params, X)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def gradients(params, X, t):
    """Analytic gradients of the mean squared error: list of (dW, db)."""
    y, cache = forward(params, X)
    N = len(y)
    delta = (2.0 / N) * (y - np.asarray(t, np.float64))[:, None]        # d loss / d z_{K-1}
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        h, z = cache[l]
        W = np.asarray(params[l][0], np.float64)
        grads[l] = (delta.T @ h, delta.sum(axis=0))
        if l > 0:
            _, zp = cache[l - 1]
            delta = (delta @ W) * (1.0 - np.tanh(zp) ** 2)
    return grads


def numeric_gradients(params, X, t, eps=1e-6):
    """Central finite differences (for pinning `gradients` on small nets)."""
    out = []
    for l, (W, b) in enumerate(params):
        gW = np.zeros_like(np.asarray(W, np.float64))
        gb = np.zeros_like(np.asarray(b, np.float64))
        for arr, g in ((W, gW), (b, gb)):
            base = np.asarray(arr, np.float64)
            it = np.nditer(base, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                p_plus = [(np.array(w, np.float64), np.array(bb, np.float64)) for w, bb in params]
                p_minus = [(np.array(w, np.float64), np.array(bb, np.float64)) for w, bb in params]
                tgt_plus = p_plus[l][0] if arr is W else p_plus[l][1]
                tgt_minus = p_minus[l][0] if arr is W else p_minus[l][1]
                tgt_plus[idx] += eps
                tgt_minus[idx] -= eps
                g[idx] = (loss(p_plus, X, t) - loss(p_minus, X, t)) / (2 * eps)
        out.append((gW, gb))
    return out


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; state = dict(step, m, v) (m, v lists like params)."""
    state["step"] += 1
    k = state["step"]
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        mW, mb = state["m"][l]
        vW, vb = state["v"][l]
        mW = beta1 * mW + (1 - beta1) * gW
        mb = beta1 * mb + (1 - beta1) * gb
        vW = beta2 * vW + (1 - beta2) * gW * gW
        vb = beta2 * vb + (1 - beta2) * gb * gb
        state["m"][l] = (mW, mb)
        state["v"][l] = (vW, vb)
        c1 = 1 - beta1 ** k
        c2 = 1 - beta2 ** k
        W = np.asarray(W, np.float64) - lr * (mW / c1) / (np.sqrt(vW / c2) + eps)
        b = np.asarray(b, np.float64) - lr * (mb / c1) / (np.sqrt(vb / c2) + eps)
        new.append((W, b))
    return new


def adam_state(params):
    z = [(np.zeros_like(np.asarray(W, np.float64)), np.zeros_like(np.asarray(b, np.float64))) for W, b in params]
    return {"step": 0, "m": [tuple(x.copy() for x in p) for p in z], "v": [tuple(x.copy() for x in p) for p in z]}
