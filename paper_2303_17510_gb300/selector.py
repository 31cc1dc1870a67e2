"""Training data, training and installation of the learned parameter selector.

The selector predicts the log time of one convolution for a (problem,
candidate) pair (features: ``hd_selector_features``) with an ensemble of small
MLPs that run on the GPU (``hd_mlp_*`` kernels).  Its training data are the
library's own autotuner timings (``hd_autotune``); this module only moves data
and drives the loops.

Run as a script on a GPU to regenerate the committed training set:
    python -m paper_2303_17510_gb300.selector --out paper_2303_17510_gb300/data/selector_gb300.json
    python -m paper_2303_17510_gb300.selector --append --kind hermitian --problems 120 --seed 7 --L-hi 8192
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

from . import _binding as b

DIMS = (b.SELECTOR_FEATURES, 32, 32, 1)
HERE = os.path.dirname(os.path.abspath(__file__))
DATA = os.path.join(HERE, "data", "selector_gb300.json")


def problem_set(n, seed, L_lo=64, L_hi=65536, ratio_lo=0.3, ratio_hi=0.67, kind=None):
    """Random 1D FP32 problems of the ragged workload's distribution: L
    log-uniform, L/M uniform, A in {2, 3}; ratios above 1/2 use the centered
    kind and M is raised to the kind's dealiasing bound when needed.  `kind`
    forces one kind for every problem (e.g. "hermitian", the innermost axis
    of Hermitian N-D data)."""
    g = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = int(math.floor(math.exp(g.uniform(math.log(L_lo), math.log(L_hi)))))
        r = float(g.uniform(ratio_lo, ratio_hi))
        A = 2 if g.uniform() < 0.5 else 3
        k = kind or ("centered" if r > 0.5 else "complex")
        M = max(int(math.ceil(L / r)), b.dealias_bound(k, L, "product" if A == 2 else "sum_pairs3"))
        out.append(dict(L=L, M=M, A=A, kind=k))
    return out


def batch_count(L, work=1 << 21):
    return max(1, min(4096, work // max(L, 64)))


def collect(problems, reps=3, work=1 << 21):
    """Times every candidate of every problem; returns rows of features, the
    log of microseconds per convolution, and the problem index."""
    X, y, pid, cands = [], [], [], []
    for i, p in enumerate(problems):
        count = batch_count(p["L"], work)
        _, allc = b.autotune(count, reps=reps, L=p["L"], M=p["M"], A=p["A"], kind=p["kind"], dtype="f32")
        for c in allc:
            if c["ms"] <= 0:
                continue
            if c["D"] > 1 and p["kind"] != "hermitian":   # cluster variants: not selector candidates
                continue
            X.append(b.selector_features(c, L=p["L"], M=p["M"], A=p["A"], kind=p["kind"], dtype="f32"))
            y.append(math.log(c["ms"] * 1e3 / count))
            pid.append(i)
            cands.append(c)
        b.tune_cache_clear()
    return dict(X=np.asarray(X, np.float32), y=np.asarray(y, np.float32), pid=np.asarray(pid, np.int64),
                cands=cands, problems=problems)


def init_params(dims, seed):
    """Xavier-uniform weights, zero biases (seeded)."""
    g = np.random.default_rng(seed)
    out = []
    for l in range(len(dims) - 1):
        fan_in, fan_out = dims[l], dims[l + 1]
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        out.append(g.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32).ravel())
        out.append(np.zeros(fan_out, np.float32))
    return np.concatenate(out)


def train(data, k=4, steps=3000, lr=3e-3, seed=0, dims=DIMS):
    """Trains k networks on the GPU with the library's kernels (full batch, Adam)."""
    import torch
    X = torch.from_numpy(data["X"]).cuda()
    t = torch.from_numpy(data["y"]).cuda()
    models, losses = [], []
    for i in range(k):
        m = b.MLP(dims)
        m.set_params(init_params(dims, seed + i))
        for s in range(steps):
            cur = lr * (0.1 if s > 0.8 * steps else 1.0)
            m.train_step(X, t, cur)
        loss, _ = m.gradients(X, t)
        models.append(m)
        losses.append(loss)
    return models, losses


def predict(models, X):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    outs = []
    for m in models:
        Y = torch.empty(Xd.shape[0], dtype=torch.float32, device="cuda")
        m.forward(Xd, Y)
        outs.append(Y.cpu().numpy())
    return np.stack(outs)


def evaluate(models, data, cost_pick=None):
    """Per problem: time of the ensemble's pick, of the best candidate and of
    the cost-model pick (from the timed table), in microseconds per conv."""
    P = predict(models, data["X"]).mean(axis=0)
    res = []
    for i in np.unique(data["pid"]):
        rows = np.where(data["pid"] == i)[0]
        t = np.exp(data["y"][rows])
        sel = rows[np.argmin(P[rows])]
        row = dict(problem=int(i), selector=float(np.exp(data["y"][sel])), best=float(t.min()))
        if cost_pick is not None:
            row["cost_model"] = float(cost_pick(int(i), rows))
        res.append(row)
    return res


def save(models, path):
    json.dump({"dims": list(models[0].dims), "params": [m.get_params().tolist() for m in models]}, open(path, "w"))


def load(path):
    d = json.load(open(path))
    models = []
    for p in d["params"]:
        m = b.MLP(d["dims"])
        m.set_params(np.asarray(p, np.float32))
        models.append(m)
    return models


def save_data(data, path):
    json.dump({"X": data["X"].tolist(), "y": data["y"].tolist(), "pid": data["pid"].tolist(),
               "cands": data["cands"], "problems": data["problems"]}, open(path, "w"))


def load_data(path=DATA):
    d = json.load(open(path))
    return dict(X=np.asarray(d["X"], np.float32), y=np.asarray(d["y"], np.float32),
                pid=np.asarray(d["pid"], np.int64), cands=d["cands"], problems=d["problems"])


def merge_data(a, c):
    """Training sets a and c as one (problem indices of c shifted past a's)."""
    off = len(a["problems"])
    return dict(X=np.concatenate([a["X"], c["X"]]), y=np.concatenate([a["y"], c["y"]]),
                pid=np.concatenate([a["pid"], c["pid"] + off]), cands=list(a["cands"]) + list(c["cands"]),
                problems=list(a["problems"]) + list(c["problems"]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DATA)
    ap.add_argument("--problems", type=int, default=400)
    ap.add_argument("--seed", type=int, default=123)
    ap.add_argument("--kind", default=None, help="one kind for every problem (default: the ragged mix)")
    ap.add_argument("--L-hi", type=int, default=65536)
    ap.add_argument("--append", action="store_true", help="add the new problems to the existing set in --out")
    args = ap.parse_args()
    data = collect(problem_set(args.problems, args.seed, L_hi=args.L_hi, kind=args.kind))
    if args.append and os.path.exists(args.out):
        data = merge_data(load_data(args.out), data)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    save_data(data, args.out)
    print("rows", len(data["y"]), "problems", len(data["problems"]))


if __name__ == "__main__":
    main()
