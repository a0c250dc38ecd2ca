"""Pins for the oracle's l1 metric (Section 3 names l1 as the generalisation
of the method): brute force against numpy, the exact cap, samples against
the documented Philox stream, the identity with squared l2 on +-1/2 data (where
|d| = d^2), Theorem 1's containment, and a closed-form case that separates
the l1 width span*alpha from the l2 width span^2*alpha."""

import numpy as np
import pytest
from scipy import stats

import _philox_ref
import oracle
from paper_1902_09465_gb300 import synth

def _coord(seed, qid, point, s, m):
    return _philox_ref.scaled(seed, qid, point, s, m)


def test_l1_brute_force_matches_numpy_with_ties():
    g = np.random.default_rng(3)
    X = g.integers(-3, 4, size=(400, 7)).astype(np.float32)   # many equal l1 distances
    Q = g.integers(-3, 4, size=(5, 7)).astype(np.float32)
    idx, dist = oracle.exact_knn(X, Q, 12, metric="l1")
    for q in range(5):
        d = np.abs(X.astype(np.float64) - Q[q]).sum(1)
        order = np.lexsort((np.arange(400), d))[:12]
        np.testing.assert_array_equal(idx[q], order)
        np.testing.assert_array_equal(dist[q], d[order])


def test_l1_all_coordinates_give_the_exact_distance():
    X, Q, _ = synth.gaussian_planted(300, 24, 4, seed=3)
    r = oracle.adaptive(X, Q, oracle.make_params(4, B0=24, bound="footnote", metric="l1"))
    d = np.abs(X.astype(np.float64) - Q[0].astype(np.float64)).sum(1)
    np.testing.assert_allclose(r["S"][0], d, rtol=1e-12)
    assert r["stats"][0]["evals"] == 300 * 24


def test_l1_estimates_are_sums_of_absolute_differences_at_drawn_coordinates():
    X, Q, _ = synth.gaussian_planted(40, 64, 3, seed=4)
    r = oracle.adaptive(X, Q, oracle.make_params(3, B0=8, B=8, bound="exp", c_alpha=1e-3, seed=11, metric="l1"))
    for i in range(40):
        T = int(r["T"][0, i])
        if T >= 64:
            exp = np.abs(X[i].astype(np.float64) - Q[0]).sum()
        else:
            js = np.array([_coord(11, 0, i, s, 64) for s in range(T)])
            exp = np.abs(X[i, js].astype(np.float64) - Q[0, js].astype(np.float64)).sum()
        assert r["S"][0, i] == pytest.approx(exp, rel=1e-12, abs=0)


def test_l1_equals_squared_l2_on_half_binary_data():
    """On +-1/2 coordinates every difference is 0 or 1, so |d| = d^2 and the
    span is 1: the two metrics take the same samples, sums, widths and
    decisions."""
    for t in range(6):
        X, q, _ = synth.binary_half(200, 512, 3, 0.1, 0.4, seed=500 + t)
        for bound, c in (("footnote", 1.0), ("exp", 1e-2)):
            a = oracle.adaptive(X, q, oracle.make_params(3, bound=bound, c_alpha=c, B0=16, B=16, grow=1, seed=t))
            b = oracle.adaptive(X, q, oracle.make_params(3, bound=bound, c_alpha=c, B0=16, B=16, grow=1, seed=t,
                                                         metric="l1"))
            for key in ("idx", "code", "S", "T"):
                np.testing.assert_array_equal(a[key], b[key])


def test_l1_containment_rate_binary_data():
    trials, delta, k = 100, 0.05, 3
    fails = 0
    for t in range(trials):
        X, q, near = synth.binary_half(150, 2048, k, 0.05, 0.45, seed=6000 + t)
        r = oracle.adaptive(X, q, oracle.make_params(k, delta=delta, bound="footnote", B0=32, B=32, grow=1, seed=t,
                                                     metric="l1"))
        st = r["stats"][0]
        ti, _ = oracle.exact_knn(X, q, k, metric="l1")
        fails += not set(ti[0]) <= set(r["idx"][0][: st["count"]])
    assert fails <= stats.binom.ppf(0.999, trials, delta)


@pytest.mark.parametrize("w,decided", [(0.2, True), (0.3, False)])
def test_l1_width_scales_with_span(w, decided):
    """Query and point 0 at 0, points 1 and 2 at 1, point 3 at 2 in every
    coordinate: span 2, estimates exactly 0, 1, 1, 2. The l1 half-width is
    span*alpha = 2w: points 1-3 are eliminated and point 0 accepted in round 0
    iff 1 - 2w > 2w (w < 1/4); the l2 scaling span^2 would need w < 1/6."""
    m, u, n, delta = 32, 2, 4, 0.01
    X = np.zeros((n, m), dtype=np.float32)
    X[1:3] = 1.0
    X[3] = 2.0
    q = np.zeros((1, m), dtype=np.float32)
    c = w * w * u / np.log(1.0 + (1.0 + np.log(u)) * n / delta)  # alpha(u) = w, Section 5 form
    r = oracle.adaptive(X, q, oracle.make_params(1, h=0, delta=delta, bound="exp", c_alpha=c, B0=u, B=u,
                                                 metric="l1"))
    kind = r["code"][0] & 3
    if decided:
        assert r["stats"][0]["rounds"] == 1 and list(r["idx"][0]) == [0]
        assert kind[0] == oracle.ACCEPTED and np.all(kind[1:] == oracle.ELIMINATED)
    else:
        assert np.all((r["code"][0][:3] >> 2) >= 1)


@pytest.mark.parametrize("slack,decided", [(1.5, True), (0.5, False)])
def test_l1_copy_term_is_the_element_error(slack, decided):
    """Under l1 a stored copy moves a sample |x - q| by at most e, so the
    width is (span + e) alpha + e. Query and point 0 at 0, points 1 and 2 at
    257 (BF16 copy 256: e = 1), point 3 at 4096 (span 4096): estimates 0, 256,
    256, 4096; round 0 decides everything iff the width is below 128. With
    (span + e) alpha = 128 - slack the width is 128.5 - slack: decided for
    slack 1.5, not for 0.5 (a dropped e would decide both; the l2 term
    e (2 span + e) = 8193 would decide neither)."""
    m, u, n, delta, e, span = 32, 2, 4, 0.01, 1.0, 4096.0
    X = np.zeros((n, m), dtype=np.float32)
    X[1:3] = 257.0
    X[3] = span
    q = np.zeros((1, m), dtype=np.float32)
    _, _, emax = oracle.quantize(X, "bf16")
    assert emax == e
    a = (128.0 - slack) / (span + e)
    c = a * a * u / np.log(1.0 + (1.0 + np.log(u)) * n / delta)  # alpha(u) = a, Section 5 form
    r = oracle.adaptive(X, q, oracle.make_params(1, h=0, delta=delta, bound="exp", c_alpha=c, B0=u, B=u,
                                                 metric="l1", storage="bf16"))
    kind = r["code"][0] & 3
    if decided:
        assert r["stats"][0]["rounds"] == 1 and list(r["idx"][0]) == [0]
        assert kind[0] == oracle.ACCEPTED and np.all(kind[1:] == oracle.ELIMINATED)
    else:
        assert np.all((r["code"][0][:3] >> 2) >= 1)
