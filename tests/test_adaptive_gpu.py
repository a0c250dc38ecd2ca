"""GPU parity of the adaptive rounds against the oracle, through the C ABI."""

import numpy as np
import pytest
import torch

import oracle
from _parity import check, run_gpu
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bound,c_alpha", [("footnote", 1.0), ("lemma", 1.0), ("exp", 1e-3), ("exp", 1e-4)])
def test_gaussian_single_query(bound, c_alpha):
    # n=2000 points in m=256, 5 planted neighbours, delta=0.01, seed 0
    X, Q, _ = synth.gaussian_planted(2000, 256, 5, seed=0)
    summ, gpu = check(X, Q, 5, delta=0.01, seed=0, bound=bound, c_alpha=c_alpha)
    ti, _ = oracle.exact_knn(X, Q, 5)
    assert set(ti[0]) <= set(gpu["idx"][0][: gpu["count"][0]])


@pytest.mark.parametrize("B0,B,grow", [(16, 16, 0), (8, 8, 1), (1, 3, 0), (12, 20, 1), (64, 32, 0)])
def test_schedules(B0, B, grow):
    X, Q, _ = synth.gaussian_planted(3000, 200, 6, nq=3, seed=1)
    check(X, Q, 6, delta=0.05, seed=7, bound="exp", c_alpha=3e-4, B0=B0, B=B, grow=grow)


def test_pixel_mixture_several_tiles_ragged_tail():
    # 5000 points (two full 2048-slot decide tiles and a ragged one), m=784
    X, Q = synth.pixel_mixture(5000, 784, 16, seed=3)
    summ, gpu = check(X, Q, 10, delta=0.01, seed=3, bound="exp", c_alpha=3e-3, B0=16, B=16, grow=1)
    assert summ["queries"] == 16


@pytest.mark.parametrize("k", [1, 10, 100])
def test_integer_valued_gap_planted(k):
    X, Q, _ = synth.gap_planted(8000, 128, 6, k, [3.0, 1.05, 3.0, 1.05, 2.0, 1.2], seed=4, background="int255")
    check(X, Q, k, delta=0.01, seed=11, bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1)


def test_shared_coordinates_mask():
    X, Q, _ = synth.gaussian_planted(2500, 160, 4, nq=4, seed=5)
    check(X, Q, 4, delta=0.01, seed=2, bound="exp", c_alpha=1e-3, share_points=True)
    check(X, Q, 4, delta=0.01, seed=2, bound="exp", c_alpha=1e-3, share_points=True, share_queries=True)


def test_query_id_base_selects_the_stream():
    X, Q, _ = synth.gaussian_planted(1500, 96, 3, nq=4, seed=6)
    a = run_gpu(X, Q, 3, 0.01, 0, bound="exp", c_alpha=1e-3, qid_base=100)
    b = run_gpu(X, Q[2:3], 3, 0.01, 0, bound="exp", c_alpha=1e-3, qid_base=102)
    np.testing.assert_array_equal(a["code"][2], b["code"][0])
    np.testing.assert_array_equal(a["idx"][2], b["idx"][0])
    check(X, Q, 3, 0.01, 0, bound="exp", c_alpha=1e-3, qid_base=100)


def test_edge_cases():
    # n <= k + h: every point returned, nothing sampled
    X, Q, _ = synth.gaussian_planted(9, 16, 4, seed=1)
    check(X, Q, 4, h=5)
    # h = 0, k = 1
    X, Q, _ = synth.gaussian_planted(700, 33, 1, nq=2, seed=2)
    check(X, Q, 1, h=0, bound="exp", c_alpha=1e-3, B0=5, B=7)
    # k = n - h exactly at the limit
    X, Q, _ = synth.gaussian_planted(40, 12, 2, seed=3)
    check(X, Q, 30, h=9, bound="exp", c_alpha=1e-2)
    # m = 1 and m = 3 (rows not 16-byte multiples)
    for m in (1, 3):
        X, Q, _ = synth.gaussian_planted(300, m, 2, nq=2, seed=4)
        check(X, Q, 2, bound="exp", c_alpha=1e-2, B0=1, B=1)
    # first round already exact (B0 >= m)
    X, Q, _ = synth.gaussian_planted(1000, 24, 3, nq=2, seed=5)
    check(X, Q, 3, B0=24)
    # all points identical: nothing separates, the exact round decides ties by index
    X = np.ones((100, 8), dtype=np.float32)
    check(X, X[:2].copy(), 3, h=2)


def test_non_finite_data_gives_empty_result():
    X, Q, _ = synth.gaussian_planted(200, 16, 2, nq=2, seed=1)
    X[17, 3] = np.nan
    g = run_gpu(X, Q, 2, 0.01, 0)
    assert np.all(g["count"] == 0) and np.all(g["idx"] == -1)


def test_workspace_argument_and_repeat_calls_identical():
    X, Q, _ = synth.gaussian_planted(4000, 128, 5, nq=8, seed=8)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    o = knn.make_opts(5, bound="exp", c_alpha=1e-3)
    ws = torch.empty(knn.adaptive_workspace_size(4000, 128, 8, 5, o), dtype=torch.uint8, device="cuda")
    a = knn.adaptive(Xd, Qd, 5, 0.01, 3, bound="exp", c_alpha=1e-3, workspace=ws)
    b = knn.adaptive(Xd, Qd, 5, 0.01, 3, bound="exp", c_alpha=1e-3)
    for key in ("idx", "count", "evals", "rounds"):
        assert torch.equal(a[key], b[key])
    with pytest.raises(knn.KnnError):
        knn.adaptive(Xd, Qd, 5, 0.01, 3, bound="exp", c_alpha=1e-3, workspace=ws[:100])


def test_containment_binary_data_gpu():
    """Theorem 1 on the GPU path: failures at most the binomial quantile."""
    from scipy import stats
    trials, fails = 60, 0
    Xs, Qs, nears = [], [], []
    for t in range(trials):
        X, q, near = synth.binary_half(150, 2048, 3, 0.05, 0.45, seed=1000 + t)
        g = run_gpu(X, q, 3, 0.05, t, bound="footnote", B0=32, B=32, grow=1)
        ti, _ = oracle.exact_knn(X, q, 3)
        fails += not set(ti[0]) <= set(g["idx"][0][: g["count"][0]])
    assert fails <= stats.binom.ppf(0.999, trials, 0.05)


def test_full_size_pixel_workload_sampled_queries():
    """The benchmark workload at full size (n=100,000, d=784, 1,024 queries,
    k=10) in the benchmark's launch configuration; three queries replayed."""
    import bench
    X, Q, _ = bench.make_inputs(0)
    summ, gpu = check(X, Q, 10, delta=0.01, seed=0, queries=[0, 511, 1023], bound="exp", c_alpha=1e-3,
                      B0=16, B=16, grow=1)
    assert summ["queries"] == 3
    assert np.all(gpu["count"] <= 20) and np.all(gpu["count"] >= 10)
    ti, _ = oracle.exact_knn(X, Q[[0, 511, 1023]], 10)
    for j, q in enumerate([0, 511, 1023]):
        assert set(ti[j]) <= set(gpu["idx"][q][: gpu["count"][q]])
