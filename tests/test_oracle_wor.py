"""Pins of the oracle's sampling without replacement (footnote to Section 4:
a cipher on [m]; a Feistel network with cycle walking). Nothing here
re-derives the permutation: it is checked through what any keyed permutation
sampled uniformly must satisfy — a bijection of [0, m), uniform positions
across keys, the finite-population variance of a sample mean, exactly the
undrawn coordinates missing from a sum — and through Theorem 1's guarantee."""

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1902_09465_gb300 import synth

FULL = (1 << 64) - 1


@pytest.mark.parametrize("m", [1, 2, 3, 5, 7, 16, 17, 77, 100, 255, 256, 784, 1025, 4097])
def test_each_pair_draws_a_permutation(m):
    for seed, qid, point in ((0, 0, 0), (7, 3, 11), (2**40 + 5, 12345, 999999)):
        got = [oracle.coordinate_wor(seed, qid, point, s, m) for s in range(m)]
        assert sorted(got) == list(range(m)), (m, seed, qid, point)


def test_keys_separate_pairs_and_masks_share_them():
    m = 100
    perm = lambda seed, q, p, mp=FULL, mq=FULL: [oracle.coordinate_wor(seed, q, p, s, m, mp, mq) for s in range(m)]
    base = perm(1, 2, 3)
    assert perm(1, 2, 4) != base and perm(1, 3, 3) != base and perm(2, 2, 3) != base
    # both counter fields masked: every pair follows the same permutation
    assert perm(1, 2, 3, 0, 0) == perm(1, 9, 50, 0, 0)
    # the stream is disjoint from the with-replacement draws (whose first
    # 100 draws of a pair repeat coordinates)
    wr = [oracle.coordinate(1, 2, 3, s, m) for s in range(m)]
    assert len(set(wr)) < m


@pytest.mark.parametrize("m,s", [(10, 0), (10, 7), (37, 3)])
def test_positions_are_uniform_across_keys(m, s):
    """The s-th draw over 6,000 pairs: a chi-square test of uniformity on
    [0, m) (a badly mixing round function or a dropped round fails it)."""
    pairs = 6000
    counts = np.bincount([oracle.coordinate_wor(5, q, p, s, m) for q in range(60) for p in range(pairs // 60)],
                         minlength=m)
    chi2 = ((counts - pairs / m) ** 2 / (pairs / m)).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, m - 1), counts


def test_consecutive_draws_are_not_a_progression():
    """Draws s and s + 1 of a pair: the difference mod m is spread over
    [1, m) (an affine rule s -> a s + c would give one value per key)."""
    m, pairs = 16, 4000
    diffs = [(oracle.coordinate_wor(9, 0, p, 1, m) - oracle.coordinate_wor(9, 0, p, 0, m)) % m for p in range(pairs)]
    counts = np.bincount(diffs, minlength=m)
    assert counts[0] == 0
    expect = pairs / (m - 1)
    chi2 = ((counts[1:] - expect) ** 2 / expect).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, m - 2), counts


def test_first_two_draws_are_uniform_over_ordered_pairs():
    """(draw 0, draw 1) over 6,000 pairs for m = 6 (cycle walking from a
    16-value domain): uniform over the 30 ordered pairs of distinct values."""
    m, pairs = 6, 6000
    cells = np.zeros((m, m))
    for p in range(pairs):
        cells[oracle.coordinate_wor(13, 1, p, 0, m), oracle.coordinate_wor(13, 1, p, 1, m)] += 1
    assert np.trace(cells) == 0
    expect = pairs / (m * (m - 1))
    off = cells[~np.eye(m, dtype=bool)]
    chi2 = ((off - expect) ** 2 / expect).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, m * (m - 1) - 1), cells


def test_sample_mean_has_the_finite_population_variance():
    """Mean of T draws without replacement from m values: variance
    sigma^2 / T * (m - T) / (m - 1), half of the with-replacement variance at
    T = m / 2 (the with-replacement draws are checked against sigma^2 / T)."""
    m, T, pairs = 64, 32, 4000
    v = np.random.default_rng(3).standard_normal(m)
    sig2 = v.var()
    wor = np.array([v[[oracle.coordinate_wor(11, 0, p, s, m) for s in range(T)]].mean() for p in range(pairs)])
    wr = np.array([v[[oracle.coordinate(11, 0, p, s, m) for s in range(T)]].mean() for p in range(pairs)])
    want_wor = sig2 / T * (m - T) / (m - 1)
    want_wr = sig2 / T
    # sampling error of a variance over 4,000 trials: about 2.2% (1 sd)
    assert abs(wor.var() / want_wor - 1) < 0.1, (wor.var(), want_wor)
    assert abs(wr.var() / want_wr - 1) < 0.1, (wr.var(), want_wr)
    assert abs(wor.mean() - v.mean()) < 4 * np.sqrt(want_wor / pairs)


def test_round_sum_misses_exactly_the_undrawn_coordinate():
    """B0 = m - 1 (one draw short of the exact cap): each point's round-0
    sum is its distance less exactly one coordinate's term, the one at
    draw m - 1 of its permutation."""
    X, Q, _ = synth.gaussian_planted(40, 33, 3, nq=2, seed=4)
    m = X.shape[1]
    p = oracle.make_params(3, delta=0.01, bound="exp", c_alpha=1e-9, B0=m - 1, B=1, seed=6, qid=10, replace=False)
    r = oracle.adaptive(X, Q, p)
    for qi in range(2):
        for i in range(40):
            if r["T"][qi][i] != m - 1:
                continue
            j = oracle.coordinate_wor(6, 10 + qi, i, m - 1, m)
            terms = (X[i].astype(np.float64) - Q[qi].astype(np.float64)) ** 2
            assert r["S"][qi][i] == pytest.approx(terms.sum() - terms[j], rel=1e-12, abs=1e-12)


def test_containment_rate_without_replacement():
    """Theorem 1 with the draws taken without replacement (Hoeffding's
    inequality holds for sampling without replacement, so the bounds keep
    their level): containment at rate >= 1 - delta on +-1/2 data."""
    trials, delta, k = 120, 0.05, 3
    fails = saved = 0
    for t in range(trials):
        X, q, _ = synth.binary_half(150, 2048, k, 0.05, 0.45, seed=3000 + t)
        p = oracle.make_params(k, delta=delta, bound="footnote", B0=32, B=32, grow=1, seed=t, replace=False)
        r = oracle.adaptive(X, q, p)
        st = r["stats"][0]
        ti, _ = oracle.exact_knn(X, q, k)
        fails += not set(ti[0]) <= set(r["idx"][0][: st["count"]])
        saved += st["evals"] < 150 * 2048
        assert st["count"] <= 2 * k
    assert fails <= stats.binom.ppf(0.999, trials, delta)
    assert saved >= 0.9 * trials


def test_without_replacement_needs_single_coordinates():
    X, Q, _ = synth.gaussian_planted(50, 16, 2, nq=1, seed=1)
    with pytest.raises(ValueError):
        oracle.adaptive(X, Q, oracle.make_params(2, block=4, replace=False))
