"""GPU parity of ragged batches (one persistent kernel launch replayed from a
CUDA graph) against the FP64 direct oracle, plus the bounded-wait failure
path of the persistent kernel."""
import os

import numpy as np
import pytest

import inputs
from oracle import cdirect
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def make_batch(descs, seed):
    import torch
    fs, hs, host = [], [], []
    for i, d in enumerate(descs):
        xs = [inputs.uniform_complex(d["L"], seed + 7 * i + a, dtype=np.complex64) for a in range(d["A"])]
        host.append(xs)
        fs.append([torch.from_numpy(x).cuda() for x in xs])
        hs.append(torch.full((d["L"],), float("nan"), dtype=torch.complex64, device="cuda"))
    return fs, hs, host


def oracle_of(d, xs):
    mult = "product" if d["A"] == 2 else "sum_pairs3"
    return cdirect.conv1d_batch([x[None, :].astype(np.complex128) for x in xs], d["L"], d["kind"], mult)[0]


def test_ragged_matches_oracle_and_replays(hd):
    import torch
    descs = inputs.ragged_instances(240, 11, hd.dealias_bound, L_lo=64, L_hi=24000)
    fs, hs, host = make_batch(descs, 100)
    with hd.RaggedPlan(descs) as plan:
        kinds = set()
        for i in range(len(descs)):
            c = plan.params(i)
            kinds.add("split" if c["S"] > 4096 else "fused")
            assert c["q"] * c["m"] >= descs[i]["M"]
        assert kinds == {"split", "fused"}
        plan.bind(fs, hs)
        plan.run()
        assert plan.status() == "HD_OK"
        first = [h.cpu().numpy() for h in hs]
        for i, d in enumerate(descs):
            e = rel_l2(first[i], oracle_of(d, host[i]))
            assert e <= 1e-5, (i, d, plan.params(i), e)
        for h in hs:
            h.fill_(float("nan"))
        plan.run()
        assert plan.status() == "HD_OK"
        for i in range(len(descs)):
            assert np.array_equal(hs[i].cpu().numpy(), first[i])


def test_ragged_explicit_candidates(hd):
    descs = [dict(L=3000, M=5999, A=2, kind="complex"), dict(L=1000, M=1500, A=3, kind="centered"),
             dict(L=9000, M=17999, A=2, kind="complex")]
    cands = []
    for d in descs:
        cs = hd.enumerate_candidates(L=d["L"], M=d["M"], A=d["A"], kind=d["kind"])
        cands.append(max(cs, key=lambda c: c["S"]))          # the largest transform of each
    fs, hs, host = make_batch(descs, 5)
    with hd.RaggedPlan(descs, candidates=cands) as plan:
        plan.bind(fs, hs)
        plan.run()
        assert plan.status() == "HD_OK"
        for i, d in enumerate(descs):
            assert rel_l2(hs[i].cpu().numpy(), oracle_of(d, host[i])) <= 1e-5


def test_ragged_wait_timeout_is_reported(hd):
    """A split instance whose row tiles wait for a column tile that never
    comes: the wait runs out after the limit, the run reports HD_ERR_TIMEOUT,
    and the context stays usable for the next run."""
    descs = [dict(L=9000, M=17999, A=2, kind="complex"), dict(L=500, M=999, A=2, kind="complex")]
    fs, hs, host = make_batch(descs, 9)
    with hd.RaggedPlan(descs) as plan:
        assert plan.params(0)["S"] > 4096
        plan.bind(fs, hs)
        plan.set_wait_limit(200_000_000)
        plan.inject_stall(0)
        plan.run()
        assert plan.status() == "HD_ERR_TIMEOUT"
        # the fused instance still completed
        assert rel_l2(hs[1].cpu().numpy(), oracle_of(descs[1], host[1])) <= 1e-5
    with hd.RaggedPlan(descs) as plan:
        plan.bind(fs, hs)
        plan.run()
        assert plan.status() == "HD_OK"
        assert rel_l2(hs[0].cpu().numpy(), oracle_of(descs[0], host[0])) <= 1e-5


def test_ragged_full_size(hd):
    """10,000 instances, L log-uniform on [64, 65536], L/M on [0.3, 0.67],
    A in {2, 3}.  For every class of instances present (transform size S,
    kind, A) the shortest instance is compared in full with the FP64 direct
    sum; nine more instances (shortest, median, longest L) on 64 points."""
    import concurrent.futures as cf
    import torch
    descs = inputs.ragged_instances(10000, 4, hd.dealias_bound)
    tot = sum(d["L"] for d in descs)
    base = [torch.from_numpy(inputs.uniform_complex(tot, 50 + a, dtype=np.complex64)).cuda() for a in range(3)]
    out = torch.empty(tot, dtype=torch.complex64, device="cuda")
    fs, hs, off = [], [], 0
    for d in descs:
        fs.append([base[a][off:off + d["L"]] for a in range(d["A"])])
        hs.append(out[off:off + d["L"]])
        off += d["L"]
    with hd.RaggedPlan(descs) as plan:
        plan.bind(fs, hs)
        plan.run()
        assert plan.status() == "HD_OK"
        params = [plan.params(i) for i in range(len(descs))]
    got_all = out.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([d["L"] for d in descs])])
    host = [x.cpu().numpy() for x in base]
    classes = {}
    for i, d in enumerate(descs):
        key = (params[i]["S"], d["kind"], d["A"])
        if key not in classes or d["L"] < descs[classes[key]]["L"]:
            classes[key] = i
    split_sizes = {k[0] for k in classes if k[0] > 4096}
    assert len(split_sizes) >= 3 and split_sizes <= {8192, 16384, 32768, 65536}, sorted(split_sizes)
    assert {(k[1], k[2]) for k in classes if k[0] > 4096} == {("complex", 2), ("complex", 3),
                                                              ("centered", 2), ("centered", 3)}

    def full_check(i):
        d = descs[i]
        xs = [host[a][offs[i]:offs[i + 1]][None, :].astype(np.complex128) for a in range(d["A"])]
        mult = "product" if d["A"] == 2 else "sum_pairs3"
        want = cdirect.conv1d_batch(xs, d["L"], d["kind"], mult, nthreads=1)[0]
        return i, rel_l2(got_all[offs[i]:offs[i + 1]], want)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        errs = dict(ex.map(full_check, sorted(classes.values(), key=lambda i: -descs[i]["L"])))
    bad = {i: (descs[i], params[i], e) for i, e in errs.items() if not e <= 1e-5}
    assert not bad, bad
    order = np.argsort([d["L"] for d in descs])
    pick = list(order[:3]) + list(order[len(order) // 2: len(order) // 2 + 3]) + list(order[-3:])
    for i in pick:
        d = descs[i]
        xs = [host[a][offs[i]:offs[i + 1]] for a in range(d["A"])]
        idx = np.unique(np.linspace(0, d["L"] - 1, 64).astype(np.int64))
        mult = "product" if d["A"] == 2 else "sum_pairs3"
        want = cdirect.conv1d_points([x.astype(np.complex128) for x in xs], d["L"], idx, d["kind"], mult)
        got = got_all[offs[i]:offs[i + 1]][idx]
        assert rel_l2(got, want) <= 1e-5, (i, d, params[i])
