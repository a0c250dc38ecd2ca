"""Algorithm 1 with the seven heaps of Section 4.1 against the version that
scans the sets: the same iterations, evaluations and returned set on every
case (the two share the sampling and the arithmetic of an iteration, and
differ in how q1, q2 and b2 are found and the order is kept), and the
heap version's containment of the k nearest on easy and binary data."""

import time

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1902_09465_gb300 import synth


@pytest.mark.parametrize("n,m,k,h,bound,c,seed", [
    (300, 64, 3, 3, "exp", 1e-3, 0), (500, 128, 5, 0, "exp", 3e-4, 1), (400, 33, 1, 4, "footnote", 1.0, 2),
    (250, 200, 10, 10, "exp", 1e-2, 3), (120, 1, 2, 2, "exp", 1e-3, 4), (600, 96, 7, 2, "lemma", 1.0, 5)])
def test_heaps_equal_scans(n, m, k, h, bound, c, seed):
    X, Q, _ = synth.gaussian_planted(n, m, k, seed=seed)
    p = oracle.make_params(k, h=h, delta=0.05, bound=bound, c_alpha=c, seed=seed)
    a = oracle.sequential(X, Q[0], p)
    b = oracle.sequential(X, Q[0], p, heaps=True)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1:] == b[1:]


def test_heaps_equal_scans_with_ties():
    # duplicated rows and integer data: many equal estimates, the rank order decides
    X, Q, _ = synth.gap_planted(400, 16, 2, 4, [3.0, 1.05], seed=7, background="int255")
    X[50:80] = X[10]
    for qi in range(2):
        p = oracle.make_params(4, h=3, delta=0.05, bound="exp", c_alpha=1e-3, seed=qi)
        a = oracle.sequential(X, Q[qi], p)
        b = oracle.sequential(X, Q[qi], p, heaps=True)
        np.testing.assert_array_equal(a[0], b[0])
        assert a[1:] == b[1:]


def test_heaps_contain_the_knn_and_scale():
    """Theorem 1 on +-1/2 data, and a run the scan version would take far
    longer on (n = 20,000)."""
    fails = 0
    for t in range(60):
        X, q, near = synth.binary_half(150, 2048, 3, 0.05, 0.45, seed=4000 + t)
        p = oracle.make_params(3, delta=0.05, bound="footnote", seed=t)
        idx, ev, it = oracle.sequential(X, q, p, heaps=True)
        ti, _ = oracle.exact_knn(X, q, 3)
        fails += not set(ti[0]) <= set(idx.tolist())
    assert fails <= stats.binom.ppf(0.999, 60, 0.05)
    X, Q, _ = synth.gaussian_planted(20000, 128, 5, seed=9)
    p = oracle.make_params(5, delta=0.01, bound="exp", c_alpha=1e-4, seed=1)
    t0 = time.perf_counter()
    idx, ev, it = oracle.sequential(X, Q[0], p, heaps=True)
    assert time.perf_counter() - t0 < 30
    ti, _ = oracle.exact_knn(X, Q, 5)
    assert set(ti[0]) <= set(idx.tolist())
    assert ev < 0.2 * 20000 * 128


# ------------------------------------------------ closed-form limits of Algorithm 1

@pytest.mark.parametrize("heaps", [False, True])
@pytest.mark.parametrize("n,m,k", [(40, 12, 3), (25, 7, 1), (30, 1, 4)])
def test_wide_bounds_compute_every_distance(heaps, n, m, k):
    """With h = 0 and a huge C_alpha no sampled bound separates anything, so
    Algorithm 1 stops only once every point is exact: each point costs its
    initial draw, m - 1 more and the m of its exact distance (2m; a point of
    m = 1 is exact from its only draw, 1), and the result is the exact k
    nearest by (distance, index)."""
    X, Q, _ = synth.gaussian_planted(n, m, k, seed=n + m)
    p = oracle.make_params(k, h=0, delta=0.05, bound="exp", c_alpha=1e12, seed=2)
    idx, evals, iters = oracle.sequential(X, Q[0], p, heaps=heaps)
    ti, _ = oracle.exact_knn(X, Q[0:1], k)
    np.testing.assert_array_equal(idx, ti[0])
    assert evals == (n if m == 1 else 2 * m * n)


@pytest.mark.parametrize("heaps", [False, True])
def test_vanishing_bounds_stop_before_the_first_iteration(heaps):
    """With C_alpha -> 0 every bound is its estimate, and the estimates are in
    order, so the termination test holds at once: no iteration, one draw per
    point, and the k + h smallest single-draw estimates by (estimate, index)
    (the draws are orc_coordinate's, pinned to the documented Philox4x32 stream)."""
    n, m, k, h = 60, 50, 4, 3
    X, Q, _ = synth.gaussian_planted(n, m, k, seed=11)
    q = Q[0]
    p = oracle.make_params(k, h=h, delta=0.05, bound="exp", c_alpha=1e-300, seed=5, qid=7)
    idx, evals, iters = oracle.sequential(X, q, p, heaps=heaps)
    assert iters == 0 and evals == n
    est = np.array([(float(X[i, j]) - float(q[j])) ** 2
                    for i, j in ((i, oracle.coordinate(5, 7, i, 0, m)) for i in range(n))])
    want = np.lexsort((np.arange(n), est))[: k + h]
    np.testing.assert_array_equal(idx, want)


def _cost_table(name, gen, k, h, delta, c_alpha, trials, schedules):
    """Medians of evaluations / (n m) of Algorithm 1 (seven heaps) and of the
    batched rounds at each schedule, with how often the k nearest came back."""
    rows = {"sequential": [], **{s: [] for s in schedules}}
    hits = {key: 0 for key in rows}
    for t in range(trials):
        X, Q = gen(t)
        n, m = X.shape
        true = set(oracle.exact_knn(X, Q[:1], k)[0][0].tolist())
        p = oracle.make_params(k, h=h, delta=delta, bound="exp", c_alpha=c_alpha, seed=t)
        idx, ev, _ = oracle.sequential(X, Q[0], p, heaps=True)
        rows["sequential"].append(ev / (n * m))
        hits["sequential"] += true <= set(idx.tolist())
        for b0, b, g in schedules:
            pb = oracle.make_params(k, h=h, delta=delta, bound="exp", c_alpha=c_alpha, seed=t, B0=b0, B=b, grow=g)
            st = oracle.adaptive(X, Q[:1], pb, want_state=False)
            s0 = st["stats"][0]
            rows[(b0, b, g)].append(s0["evals"] / (n * m))
            hits[(b0, b, g)] += true <= set(st["idx"][0][: s0["count"]].tolist())
    med = {key: float(np.median(v)) for key, v in rows.items()}
    print(f"\n{name}: " + ", ".join(f"{key}: {med[key]:.4f} ({hits[key]}/{trials})" for key in rows))
    return med, hits


def test_two_arms_per_iteration_spend_fewer_evaluations_than_batched_rounds():
    """The cost of batching (Section 4's Algorithm 1 samples only q1 and b2 per
    iteration): on the same inputs and bound, Algorithm 1 spends fewer
    coordinate evaluations than rounds that sample every undecided point,
    and both return the k nearest. (python -m pytest -s prints the medians.)"""
    sched = ((1, 1, 0), (8, 8, 1), (16, 16, 1))
    med, hits = _cost_table("gaussian planted n = 2,000, m = 256, k = h = 5, C_alpha = 1e-3",
                            lambda t: synth.gaussian_planted(2000, 256, 5, seed=t)[:2], 5, 5, 0.01, 1e-3, 6, sched)
    for s in sched:
        assert med["sequential"] < med[s]
    assert all(v == 6 for v in hits.values())
    med, hits = _cost_table("subspace p = 10, n = 1,000, m = 12,288, k = h = 10, C_alpha = 1e-3",
                            lambda t: synth.subspace(1000, 12288, 10, nq=1, seed=t), 10, 10, 0.001, 1e-3, 3, sched)
    for s in sched:
        assert med["sequential"] < med[s]
    assert all(v == 3 for v in hits.values())
