"""Pins for the oracle's block samples (a sample is one of M = ceil(m/g)
blocks of g consecutive coordinates; its value the block's sum of squared
differences). Each test checks the oracle against the documented Philox stream and
block sums, the exact distance, Theorem 1's guarantee or the coherent example
of Section 4.2 -- never against the oracle itself."""

import numpy as np
import pytest
from scipy import stats

import _philox_ref
import oracle
from paper_1902_09465_gb300 import synth

def _numpy_block(seed, qid, point, s, M):
    """Block index of draw s of the documented Philox4x32 stream."""
    return _philox_ref.scaled(seed, qid, point, s, M)


def _p(**kw):
    base = dict(k=4, delta=0.01, bound="exp", c_alpha=1e-3, B0=4, B=4, grow=0, seed=0)
    base.update(kw)
    return oracle.make_params(**base)


@pytest.mark.parametrize("m,g", [(77, 8), (64, 16), (100, 32), (5, 8)])
def test_all_blocks_give_the_exact_distance(m, g):
    """M block samples make the distance exact (Algorithm 1's cap)."""
    M = -(-m // g)
    X, Q, _ = synth.gaussian_planted(200, m, 4, seed=m + g)
    r = oracle.adaptive(X, Q, _p(B0=M, block=g, bound="footnote"))
    st = r["stats"][0]
    d = ((X.astype(np.float64) - Q[0].astype(np.float64)) ** 2).sum(1)
    assert st["rounds"] == 1 and st["evals"] == 200 * m
    np.testing.assert_allclose(r["S"][0], d, rtol=1e-12)
    assert np.all(r["T"][0] == M)
    true4 = np.lexsort((np.arange(200), d))[:4]
    assert set(true4) <= set(r["idx"][0][: st["count"]])


@pytest.mark.parametrize("m,g", [(77, 8), (96, 16), (300, 32)])
def test_estimates_are_sums_of_the_drawn_blocks(m, g):
    """S is the sum, over the T blocks the documented Philox stream selects, of the
    block's squared differences; the last block of a ragged row is shorter."""
    M = -(-m // g)
    X, Q, _ = synth.gaussian_planted(40, m, 3, seed=9)
    r = oracle.adaptive(X, Q, _p(k=3, B0=2, B=1, c_alpha=1e-4, seed=13, qid=5, block=g))
    Xd, q = X.astype(np.float64), Q[0].astype(np.float64)
    checked = 0
    for i in range(40):
        T = int(r["T"][0, i])
        if T >= M:
            exp = ((Xd[i] - q) ** 2).sum()
        else:
            exp = 0.0
            for s in range(T):
                b = _numpy_block(13, 5, i, s, M)
                sl = slice(b * g, min(b * g + g, m))
                exp += ((Xd[i, sl] - q[sl]) ** 2).sum()
            checked += 1
        assert r["S"][0, i] == pytest.approx(exp, rel=1e-12, abs=0)
    assert checked > 10


def test_block_one_is_the_single_coordinate_estimator():
    X, Q, _ = synth.gaussian_planted(300, 64, 4, nq=2, seed=3)
    a = oracle.adaptive(X, Q, _p(block=0))
    b = oracle.adaptive(X, Q, _p(block=1))
    for key in ("idx", "code", "S", "T"):
        np.testing.assert_array_equal(a[key], b[key])


def test_evaluation_count_counts_block_coordinates():
    """evals = g per block drawn + m per exact distance (an exact point also
    drew every block of the rounds before its exact round)."""
    for m, g, B0, B, grow in ((77, 8, 2, 1, 0), (128, 16, 1, 1, 1), (40, 32, 1, 1, 0)):
        M = -(-m // g)
        X, Q, _ = synth.gaussian_planted(400, m, 5, seed=m)
        p = _p(k=5, B0=B0, B=B, grow=grow, block=g, c_alpha=1e-3)
        r = oracle.adaptive(X, Q, p)
        T = r["T"][0]
        tb, rr = 0, 0
        while True:
            br = B0 if rr == 0 else (max(B, tb) if grow else B)
            if tb + br >= M:
                break
            tb, rr = tb + br, rr + 1
        ex = T == M
        assert r["stats"][0]["evals"] == g * T[~ex].sum() + ex.sum() * (g * tb + m)


def test_containment_rate_binary_data_with_blocks():
    """Theorem 1 with block samples: a block mean of +-1/2 data lies in [0, 1]
    (normalised), so the returned set contains the k nearest with probability
    >= 1 - delta. The bound counts blocks, so the rows hold 2,048 blocks of 8."""
    trials, delta, k, m = 120, 0.05, 3, 2048 * 8
    fails, saved = 0, 0
    for t in range(trials):
        X, q, near = synth.binary_half(150, m, k, 0.05, 0.45, seed=3000 + t)
        p = oracle.make_params(k, delta=delta, bound="footnote", B0=32, B=32, grow=1, seed=t, block=8)
        r = oracle.adaptive(X, q, p)
        st = r["stats"][0]
        ti, _ = oracle.exact_knn(X, q, k)
        fails += not set(ti[0]) <= set(r["idx"][0][: st["count"]])
        saved += st["evals"] < 150 * m
    assert fails <= stats.binom.ppf(0.999, trials, delta)
    assert saved >= 0.9 * trials


def test_coherent_axis_gives_no_savings_with_blocks():
    """Section 4.2's coherent example: one coordinate differs, so with blocks
    one of M blocks carries the whole distance and nothing is decided before
    the exact round (theory bound)."""
    X, q = synth.coherent_axis(200, 256, axis=17, seed=2)
    r = oracle.adaptive(X, q, _p(k=5, bound="footnote", B0=2, B=2, block=16))
    st = r["stats"][0]
    assert st["rounds"] == 8                            # 7 sampled rounds of 2 blocks, then exact
    assert np.all((r["code"][0] >> 2) == 7)
    assert st["evals"] == 200 * (14 * 16 + 256)
    ti, _ = oracle.exact_knn(X, q, 5)
    assert set(ti[0]) <= set(r["idx"][0][: st["count"]])


def test_lossless_bf16_copy_with_blocks_reproduces_f32():
    """Integer data below 256 are exact in BF16: the copy's run must equal the
    FP32 run (copy error 0, no widening)."""
    X, Q, _ = synth.gap_planted(3000, 64, 3, 5, [3.0, 1.5, 1.05], seed=6, background="int255")
    a = oracle.adaptive(X, Q, _p(k=5, B0=2, B=1, grow=1, block=16, storage="f32"))
    b = oracle.adaptive(X, Q, _p(k=5, B0=2, B=1, grow=1, block=16, storage="bf16"))
    for key in ("idx", "code", "S", "T"):
        np.testing.assert_array_equal(a[key], b[key])


@pytest.mark.parametrize("w,decided", [(0.3, True), (0.7, False)])
def test_estimate_is_the_per_coordinate_mean_of_the_blocks(w, decided):
    """Closed-form case: the query and point 0 are all zeros, points 1 and 2
    all ones (span 1), so every block of point 1 or 2 sums to g and its
    estimate S / (T g) is exactly 1, point 0's exactly 0. With half-width w
    after round 0, points 1 and 2 are eliminated and point 0 accepted in
    round 0 iff 1 - w > w, i.e. w < 1/2 (k = 1, h = 0)."""
    m, g, u, n, delta = 64, 8, 2, 3, 0.01
    X = np.zeros((n, m), dtype=np.float32)
    X[1:] = 1.0
    q = np.zeros((1, m), dtype=np.float32)
    # C_alpha giving alpha(u) = w for the Section 5 form sqrt(C log(1 + (1 + log u) n / delta) / u)
    c = w * w * u / np.log(1.0 + (1.0 + np.log(u)) * n / delta)
    r = oracle.adaptive(X, q, oracle.make_params(1, h=0, delta=delta, bound="exp", c_alpha=c, B0=u, B=u,
                                                 block=g))
    rounds = r["code"][0] >> 2
    kind = r["code"][0] & 3
    if decided:
        assert r["stats"][0]["rounds"] == 1 and list(r["idx"][0]) == [0]
        assert kind[0] == oracle.ACCEPTED and np.all(kind[1:] == oracle.ELIMINATED)
    else:
        assert np.all(rounds >= 1)
