"""GPU checks of the selector MLP kernels against the FP64 reference
(oracle/mlp.py), and of what the trained selector gains over the cost model,
judged by the exhaustive (timed) optimum on held-out problems."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def _split(flat, dims):
    out, o = [], 0
    for l in range(len(dims) - 1):
        W = flat[o:o + dims[l + 1] * dims[l]].reshape(dims[l + 1], dims[l]).astype(np.float64)
        o += dims[l + 1] * dims[l]
        b = flat[o:o + dims[l + 1]].astype(np.float64)
        o += dims[l + 1]
        out.append((W, b))
    return out


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def test_forward_and_gradients_match_reference(hd):
    import torch
    from paper_2303_17510_gb300 import selector
    dims = (13, 32, 32, 1)
    m = hd.MLP(dims)
    flat = selector.init_params(dims, 7)
    m.set_params(flat)
    g = np.random.default_rng(0)
    X = g.uniform(-1, 1, (200, 13)).astype(np.float32)
    t = g.standard_normal(200).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    Y = torch.empty(200, device="cuda")
    m.forward(Xd, Y)
    torch.cuda.synchronize()
    params = _split(flat, dims)
    y_ref, _ = ref.forward(params, X.astype(np.float64))
    assert np.max(np.abs(Y.cpu().numpy() - y_ref)) <= 1e-5 * (1 + np.max(np.abs(y_ref)))
    loss, grads = m.gradients(Xd, td)
    assert abs(loss - ref.loss(params, X, t)) <= 1e-5 * (1 + abs(loss))
    gref = _flat(ref.gradients(params, X.astype(np.float64), t.astype(np.float64)))
    err = np.max(np.abs(grads - gref)) / np.max(np.abs(gref))
    assert err <= 1e-4, err


def test_adam_step_matches_reference(hd):
    import torch
    from paper_2303_17510_gb300 import selector
    dims = (13, 16, 1)
    m = hd.MLP(dims)
    flat = selector.init_params(dims, 3)
    m.set_params(flat)
    g = np.random.default_rng(1)
    X = g.uniform(-1, 1, (64, 13)).astype(np.float32)
    t = g.standard_normal(64).astype(np.float32)
    params = _split(flat, dims)
    st = ref.adam_state(params)
    for _ in range(3):
        m.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), 1e-2)
        params = ref.adam_step(params, ref.gradients(params, X.astype(np.float64), t.astype(np.float64)), st, 1e-2)
    assert np.max(np.abs(m.get_params() - _flat(params))) <= 1e-5


def test_selector_gain_over_cost_model(hd):
    """Trained on the autotuner's timings of 48 problems; on 24 held-out
    problems the ensemble's picks must cost at most 10% more than the timed
    optimum, and no more than the cost model's picks."""
    from paper_2303_17510_gb300 import selector
    probs = selector.problem_set(72, 2024, L_lo=64, L_hi=16384)
    train = selector.collect(probs[:48])
    test = selector.collect(probs[48:])
    models, losses = selector.train(train, k=3, steps=1500)

    def cost_pick(i, rows):
        p = test["problems"][i]
        with hd.Plan(p["L"], p["M"], A=p["A"], kind=p["kind"]) as plan:
            pr = plan.params()
        for r in rows:
            c = test["cands"][r]
            if c["m"] * c["q"] == pr["m"] * pr["q"] and c["p"] * c["m"] == pr["p"] * pr["m"] and \
                    c["minb"] == (2 if c["S"] <= 2048 else 1) and c["E"] == min(8, c["S"]):
                return float(np.exp(test["y"][r]))
        return float(np.exp(test["y"][rows]).min())

    res = selector.evaluate(models, test, cost_pick)
    sel = sum(r["selector"] for r in res)
    best = sum(r["best"] for r in res)
    cost = sum(r["cost_model"] for r in res)
    assert sel <= 1.10 * best, (sel, best, cost)
    assert sel <= cost * 1.02, (sel, best, cost)
    # installed: plans with m = 0 take the ensemble's choice (or the timed fallback)
    hd.tune_cache_clear()
    selector.b.selector_install(models, tau=0.05, sigma=0.5, fallback=False)
    try:
        p = probs[50]
        c, conf = hd.selector_choose(L=p["L"], M=p["M"], A=p["A"], kind=p["kind"])
        with hd.Plan(p["L"], p["M"], A=p["A"], kind=p["kind"]) as plan:
            pr = plan.params()
        assert (pr["m"], pr["p"], pr["q"]) == (c["m"], c["p"], c["q"])
    finally:
        hd.selector_clear()


def test_selector_picks_innermost_axis_of_nd_plans(hd):
    """With a selector installed, the innermost axis of a 2D plan takes the
    ensemble's choice for that axis's 1D problem, and the 2D result still
    matches the oracle."""
    import inputs
    from oracle import direct
    from paper_2303_17510_gb300 import selector
    from tests.gpu_util import rel_l2, to_dev
    import torch
    models, _ = selector.train(selector.load_data(), k=2, steps=300)
    hd.tune_cache_clear()
    selector.b.selector_install(models, tau=0.0, sigma=1e9, fallback=False)
    try:
        Lx, Ly = 24, 600
        My = 2 * Ly - 1 + 5
        c, conf = hd.selector_choose(L=Ly, M=My)
        assert conf == 1
        fs = [inputs.uniform_complex((Lx, Ly), 61 + a) for a in range(2)]
        with hd.Plan([Lx, Ly], [2 * Lx - 1, My]) as plan:
            ax = plan.axis_params(1)
            assert (ax["m"], ax["p"], ax["q"], ax["S"], ax["n"]) == (c["m"], c["p"], c["q"], c["S"], c["n"])
            d = [to_dev(f, "f32") for f in fs]
            out = torch.zeros_like(d[0])
            plan.convolve(d, out)
            torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), direct.convnd(fs, ("complex", "complex"))) <= 1e-5
    finally:
        hd.selector_clear()
