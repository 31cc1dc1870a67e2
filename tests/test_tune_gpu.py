"""GPU checks of the parameter candidates and the device-timed autotuner."""
import numpy as np
import pytest

from oracle import direct, params
from tests.gpu_util import rel_l2_rows, run_conv
from tests.test_conv1d_gpu import check, make_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


@pytest.mark.parametrize("kind", ["complex", "centered", "hermitian"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_every_candidate_variant_matches_oracle(hd, kind, dtype):
    """Results are the same, within the FP tolerance, whatever candidate (m, p,
    q and kernel variant) is used."""
    for L, M in ((300, None), (1500, None), (4096, None)):
        M = params.dealias_bound(kind, L) + 5 if M is None else M
        fs = make_inputs(kind, L, 2, 5, 40 + L)
        ref = direct.conv1d_batch(fs, kind)
        for c in hd.enumerate_candidates(L=L, M=M, kind=kind, dtype=dtype):
            with hd.Plan(L, M, kind=kind, dtype=dtype, candidate=c) as plan:
                got = run_conv(hd, plan, fs)
                check(got, ref, dtype, False, (kind, dtype, L, c))


def test_sum_pairs3_variants(hd):
    L, M = 2000, 3999
    fs = make_inputs("complex", L, 3, 3, 8)
    ref = direct.conv1d_batch(fs, "complex", "sum_pairs3")
    for c in hd.enumerate_candidates(L=L, M=M, A=3):
        with hd.Plan(L, M, A=3, candidate=c) as plan:
            got = run_conv(hd, plan, fs)
            assert rel_l2_rows(got, ref) <= 1e-5, c


def test_autotune_populates_cache_and_plans_use_it(hd):
    hd.tune_cache_clear()
    kw = dict(L=2048, M=3072, kind="centered", dtype="f32")
    assert hd.tune_cache_get(**kw) is None
    best, allc = hd.autotune(256, reps=3, **kw)
    timed = [c for c in allc if c["ms"] > 0]
    assert timed and best["ms"] > 0
    assert best["ms"] <= min(c["ms"] for c in timed) * 1.0101
    assert hd.tune_cache_get(**kw)["S"] == best["S"]
    with hd.Plan(2048, 3072, kind="centered") as plan:
        p = plan.params()
        assert (p["m"], p["p"], p["q"]) == (best["m"], best["p"], best["q"])
        fs = make_inputs("centered", 2048, 2, 3, 77)
        got = run_conv(hd, plan, fs)
        assert rel_l2_rows(got, direct.conv1d_batch(fs, "centered")) <= 1e-5
    hd.tune_cache_clear()
    assert hd.tune_cache_get(**kw) is None
