"""Golden fixtures (tests/golden, written by tests/golden/make_golden.py from
the oracle): the oracle must keep reproducing them, they must satisfy what
the paper fixes (the k nearest inside a returned set of at most k+h), and the
GPU path must reproduce them through the C ABI."""

import json
import os

import numpy as np
import pytest

import oracle
from paper_1902_09465_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _inputs():
    return synth.gaussian_planted(2000, 256, 5, seed=0)


def test_oracle_reproduces_single_query_fixture():
    g = _load("single_query_gaussian_n2000_m256_k5.json")
    X, Q, planted = _inputs()
    assert [int(v) for v in planted[0]] == g["planted"]
    ti, td = oracle.exact_knn(X, Q, 5)
    assert ti[0].tolist() == g["exact_idx"]
    np.testing.assert_allclose(td[0], g["exact_dist"], rtol=1e-15)
    for run in g["runs"]:
        p = oracle.make_params(5, delta=0.01, bound=run["bound"], c_alpha=run["c_alpha"], B0=run["B0"], B=run["B"],
                               grow=run["grow"], seed=0)
        r = oracle.adaptive(X, Q, p)
        st = r["stats"][0]
        assert r["idx"][0].tolist() == run["idx"]
        assert (st["count"], st["evals"], st["rounds"], st["term"]) == (run["count"], run["evals"], run["rounds"],
                                                                        run["term"])


def test_single_query_fixture_meets_the_guarantee():
    g = _load("single_query_gaussian_n2000_m256_k5.json")
    assert set(g["exact_idx"]) == set(g["planted"])  # the planted rows are the 5 nearest
    for run in g["runs"]:
        got = run["idx"][: run["count"]]
        assert run["count"] <= 10 and all(v == -1 for v in run["idx"][run["count"]:])
        assert set(g["exact_idx"]) <= set(got)
        assert run["evals"] <= 2 * 2000 * 256


@pytest.mark.gpu
def test_gpu_reproduces_single_query_fixture():
    import torch
    from paper_1902_09465_gb300 import knn
    g = _load("single_query_gaussian_n2000_m256_k5.json")
    X, Q, _ = _inputs()
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    for run in g["runs"]:
        r = knn.adaptive(Xd, Qd, 5, 0.01, 0, bound=run["bound"], c_alpha=run["c_alpha"], B0=run["B0"], B=run["B"],
                         grow=run["grow"])
        c = int(r["count"][0])
        assert c == run["count"] and int(r["evals"][0]) == run["evals"] and int(r["rounds"][0]) == run["rounds"]
        assert set(r["idx"][0, :c].cpu().tolist()) == set(run["idx"][:c])
    ei, ed = knn.exact(Xd, Qd, 5)
    assert ei[0].cpu().tolist() == g["exact_idx"]
