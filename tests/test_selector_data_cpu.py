"""Integrity of the committed selector training data against the library's
host logic: every row's 13 features are what hd_selector_features computes
for its (problem, candidate) today (to the 6 decimals stored), its target is
the log of microseconds per convolution of its timing, and its candidate is
one the library still enumerates for that problem.  The one known exception: candidates with
S = 4096 and E = 8 for three inputs with long staged rows, which the second
pad element of the radix-8 exchanges (S/16 more shared memory) pushed past
227 KB; the selector only ever picks among enumerated candidates."""
import json
import math
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("m", "p", "q", "S", "n", "E", "minb")


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def test_selector_data_matches_library(hd):
    from paper_2303_17510_gb300 import selector
    d = json.load(open(os.path.join(ROOT, "paper_2303_17510_gb300", "data", "selector_gb300.json")))
    X, y, pid, cands, probs = d["X"], d["y"], d["pid"], d["cands"], d["problems"]
    assert len(X) == len(y) == len(pid) == len(cands) > 5000
    enum = {}
    stale = []
    for i in range(len(X)):
        p, c = probs[pid[i]], cands[i]
        f = hd.selector_features(c, L=p["L"], M=p["M"], A=p["A"], kind=p["kind"], dtype="f32")
        assert np.allclose(np.float32(f), np.float32(X[i]), rtol=0, atol=1e-6), i   # stored to 6 decimals
        assert abs(np.float32(math.log(c["ms"] * 1e3 / selector.batch_count(p["L"]))) - y[i]) <= 1e-5, i
        if pid[i] not in enum:
            enum[pid[i]] = {tuple(e[k] for k in KEYS)
                            for e in hd.enumerate_candidates(L=p["L"], M=p["M"], A=p["A"], kind=p["kind"])}
        if tuple(c[k] for k in KEYS) not in enum[pid[i]]:
            stale.append((p, c))
    assert len(stale) <= 2
    for p, c in stale:
        assert c["S"] == 4096 and c["E"] == 8 and p["A"] == 3, (p, c)
