"""The l1 distance on the GPU (Section 3's generalisation): the rounds replay
in the oracle under l1 (per-pair draws, blocks, stored copies, shared
coordinates, the round-0 pass), l1 equals squared l2 on +-1/2 data bit for
bit, and the exact l1 method and the l1 rerank match the oracle's brute force."""

import numpy as np
import pytest
import torch

import oracle
from _parity import run_gpu
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def replay(X, Q, g, k, storage="f32", qid_base=0, delta=0.01, seed=0, **opt):
    g = {key: v.cpu().numpy() if hasattr(v, "cpu") else v for key, v in g.items()}
    oopt = {kk: v for kk, v in opt.items() if kk in ("h", "bound", "c_alpha", "B0", "B", "grow", "block",
                                                     "share_points", "share_queries")}
    for q in range(Q.shape[0]):
        p = oracle.make_params(k, delta=delta, seed=seed, qid=qid_base + q, tol=TOL, storage=storage, metric="l1",
                               **oopt)
        o = oracle.adaptive(X, Q[q:q + 1], p, replay=g["code"][q:q + 1])
        st = o["stats"][0]
        assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (storage, q, st)
        np.testing.assert_array_equal(o["code"][0], g["code"][q])
        assert int(g["evals"][q]) == st["evals"] and int(g["count"][q]) == st["count"], (q, st)
        So, Sg = o["S"][0], g["S"][q].astype(np.float64)
        rel = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-300)
        rel[(So == 0) & (Sg == 0)] = 0
        assert rel.max() <= TOL, (storage, q, rel.max())


@pytest.mark.parametrize("opt", [dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1),
                                 dict(bound="footnote", B0=16, B=16),
                                 dict(bound="exp", c_alpha=3e-4, B0=4, B=2, grow=1, block=8)])
def test_l1_rounds_replay(opt):
    X, Q = synth.pixel_mixture(6000, 300, 5, seed=3)
    g = run_gpu(X, Q, 10, 0.01, 2, metric="l1", **opt)
    replay(X, Q, g, 10, seed=2, **opt)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_l1_rounds_over_copies_and_the_round0_pass(storage):
    X, Q = synth.pixel_mixture(8000, 256, 6, seed=4)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1)
    with knn.Dataset(Xd, copies=(storage,)) as ds:
        a = ds.adaptive(Qd, 10, 0.01, 1, storage="f32", trace=True, metric="l1", **opt)
        b = knn.adaptive(Xd, Qd, 10, 0.01, 1, trace=True, metric="l1", **opt)     # no round-0 pass
        for key in a:
            assert torch.equal(a[key], b[key]), key
        c = ds.adaptive(Qd, 10, 0.01, 1, storage=storage, trace=True, metric="l1", **opt)
    replay(X, Q, c, 10, storage=storage, seed=1, **opt)


def test_l1_shared_coordinates():
    X, Q, _ = synth.gaussian_planted(7000, 128, 5, nq=4, seed=5)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=16, B=16, grow=1, share_points=True, share_queries=True)
    with knn.Dataset(Xd, copies=()) as ds:
        ds.share(3, copies=("f32",))
        a = ds.adaptive(Qd, 5, 0.01, 3, trace=True, metric="l1", **opt)
    b = knn.adaptive(Xd, Qd, 5, 0.01, 3, trace=True, metric="l1", **opt)
    for key in a:
        assert torch.equal(a[key], b[key]), key
    replay(X, Q, a, 5, seed=3, **opt)


def test_l1_equals_squared_l2_on_half_binary_data():
    X, q, _ = synth.binary_half(3000, 512, 3, 0.1, 0.4, seed=8)
    Q = np.repeat(q, 3, axis=0)
    for opt in (dict(bound="footnote", B0=16, B=16, grow=1), dict(bound="exp", c_alpha=1e-2, B0=8, B=8, grow=1)):
        a = run_gpu(X, Q, 3, 0.05, 4, **opt)
        b = run_gpu(X, Q, 3, 0.05, 4, metric="l1", **opt)
        for key in a:
            np.testing.assert_array_equal(a[key], b[key])


@pytest.mark.parametrize("n,m,nq,k", [(3000, 64, 17, 10), (1000, 3, 5, 7), (20000, 300, 130, 25)])
def test_exact_l1_and_rerank_match_bruteforce(n, m, nq, k):
    X, Q = synth.pixel_mixture(n, m, nq, seed=n)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    oi, od = oracle.exact_knn(X, Q, k, metric="l1")
    gi, gd = knn.exact(Xd, Qd, k, metric="l1")
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=1e-12)
    # rerank of a candidate set holding the true neighbours and others
    g = np.random.default_rng(1)
    cand = np.stack([np.concatenate([oi[q], g.permutation(np.setdiff1d(np.arange(n), oi[q]))[:40]])
                     for q in range(nq)])   # distinct candidates
    ri, rd = knn.rerank(Xd, Qd, torch.from_numpy(cand).cuda(), k, metric="l1")
    np.testing.assert_array_equal(ri.cpu().numpy(), oi)


def test_exact_l1_integer_data_with_ties():
    X, Q, _ = synth.gap_planted(6000, 32, 12, 10, 1.05, seed=2, background="int255")
    X[100:160] = X[5]
    oi, od = oracle.exact_knn(X, Q, 10, metric="l1")
    gi, gd = knn.exact(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), 10, metric="l1")
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
