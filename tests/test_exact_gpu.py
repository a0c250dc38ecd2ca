"""GPU exact path (screen + select + FP64 rerank) and rerank against the
oracle's brute force, through the C ABI."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()



@pytest.mark.parametrize("n,m,nq,k", [(1000, 64, 5, 1), (3001, 100, 130, 10), (20000, 784, 64, 10),
                                      (777, 3, 9, 7), (5000, 257, 3, 100)])
def test_exact_matches_bruteforce(n, m, nq, k):
    X, Q = synth.pixel_mixture(n, m, nq, seed=n)
    gi, gd = knn.exact(_cuda(X), _cuda(Q), k)
    oi, od = oracle.exact_knn(X, Q, k)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=1e-12)


def test_exact_gaussian_and_integer_data():
    X, Q, _ = synth.gap_planted(6000, 128, 20, 10, 1.05, seed=2, background="int255")
    gi, gd = knn.exact(_cuda(X), _cuda(Q), 10)
    oi, od = oracle.exact_knn(X, Q, 10)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)   # integer data: ties broken by index on both sides
    X, Q, _ = synth.gaussian_planted(4000, 300, 5, nq=7, seed=3)
    gi, gd = knn.exact(_cuda(X), _cuda(Q), 5)
    oi, od = oracle.exact_knn(X, Q, 5)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)


def test_exact_many_duplicates_takes_full_scan():
    # 5000 identical rows: the screen cannot narrow the set, rerank scans all
    X = np.zeros((5000, 32), dtype=np.float32)
    X[::7] = 1.0
    Q = np.zeros((2, 32), dtype=np.float32)
    gi, gd = knn.exact(_cuda(X), _cuda(Q), 5)
    oi, od = oracle.exact_knn(X, Q, 5)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)


def test_rerank_candidates():
    rng = np.random.default_rng(0)
    X, Q = synth.pixel_mixture(3000, 50, 6, seed=9)
    cand = np.stack([rng.choice(3000, 40, replace=False) for _ in range(6)]).astype(np.int64)
    cand[:, -3:] = -1
    gi, gd = knn.rerank(_cuda(X), _cuda(Q), _cuda(cand), 8)
    for q in range(6):
        c = cand[q][cand[q] >= 0]
        d = ((X[c].astype(np.float64) - Q[q].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((c, d))[:8]
        np.testing.assert_array_equal(gi[q].cpu().numpy(), c[order])
        np.testing.assert_allclose(gd[q].cpu().numpy(), d[order], rtol=1e-12)
