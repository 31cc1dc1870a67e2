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


def _time_ragged(plan, fs, hs, reps=5):
    import torch
    plan.bind(fs, hs)
    for _ in range(2):
        plan.run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.run()
    e1.record()
    torch.cuda.synchronize()
    assert plan.status() == "HD_OK"
    return e0.elapsed_time(e1) / reps


def test_selector_plans_ragged_sample_100x_faster_than_search(hd):
    """What the learned selector gains over the exhaustive timed search on a
    2,000-instance sample of the ragged workload: it plans the batch at least
    100 times faster (inference instead of timing every candidate of every
    instance) and the plan runs within 10% of the searched plan's time."""
    import time
    import torch
    import inputs
    from paper_2303_17510_gb300 import selector
    descs = inputs.ragged_instances(2000, 13, hd.dealias_bound)
    tot = sum(d["L"] for d in descs)
    base = [torch.from_numpy(inputs.uniform_complex(tot, 80 + a, dtype=np.complex64)).cuda() for a in range(3)]
    out = torch.empty(tot, dtype=torch.complex64, device="cuda")
    fs, hs, off = [], [], 0
    for d in descs:
        fs.append([base[a][off:off + d["L"]] for a in range(d["A"])])
        hs.append(out[off:off + d["L"]])
        off += d["L"]
    models, _ = selector.train(selector.load_data(), k=4, steps=2000)
    hd.tune_cache_clear()
    hd.selector_clear()
    t0 = time.perf_counter()
    for d in descs:
        hd.autotune(selector.batch_count(d["L"]), reps=3, L=d["L"], M=d["M"], A=d["A"], kind=d["kind"], dtype="f32")
    with hd.RaggedPlan(descs) as plan:       # each instance's timed optimum, from the tuning cache
        t_search = time.perf_counter() - t0
        ms_search = _time_ragged(plan, fs, hs)
    hd.tune_cache_clear()
    selector.b.selector_install(models, tau=0.05, sigma=0.25, fallback=False)
    try:
        t0 = time.perf_counter()
        with hd.RaggedPlan(descs) as plan:
            t_sel = time.perf_counter() - t0
            ms_sel = _time_ragged(plan, fs, hs)
    finally:
        hd.selector_clear()
    stats = dict(t_search=t_search, t_sel=t_sel, ms_search=ms_search, ms_sel=ms_sel)
    print("ragged sample", stats)
    assert t_search >= 100 * t_sel, stats
    assert ms_sel <= 1.10 * ms_search, stats


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
