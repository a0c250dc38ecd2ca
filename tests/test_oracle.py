"""Pins for the CPU oracle: each test checks it against something other than
itself (Philox4x32-10's published known answers and triton's implementation,
numpy's sort, closed-form special cases, brute force, Theorem 1's guarantee,
the coherent example of Section 4.2)."""

import math

import numpy as np
import pytest
from scipy import stats

import _philox_ref
import oracle
from paper_1902_09465_gb300 import synth

FULL = (1 << 64) - 1


# ------------------------------------------------------------------ Philox

# Known-answer vectors of Philox4x32-10 published with the generator (Salmon
# et al., SC'11, Random123 distribution): counter, key, output words.
KAT = [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
]


@pytest.mark.parametrize("ctr,key,expected", KAT)
def test_philox_known_answers(ctr, key, expected):
    assert [int(v) for v in oracle.philox4x32_10(ctr, key)] == expected


def test_philox_matches_triton_interpreter():
    """Triton's Philox4x32-10 (run on the CPU by its interpreter) on random
    counters and keys: a second, independent implementation."""
    import os
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def blocks(out, seed, c0p, c1p, c2p, c3p, N: tl.constexpr):
        i = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i), 10)
        tl.store(out + i * 4, a)
        tl.store(out + i * 4 + 1, b)
        tl.store(out + i * 4 + 2, c)
        tl.store(out + i * 4 + 3, d)

    g = np.random.default_rng(11)
    for _ in range(3):
        seed = int(g.integers(0, 1 << 63))
        ctr = g.integers(0, 1 << 32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
        cols = [torch.from_numpy(np.ascontiguousarray(ctr[:, j])) for j in range(4)]
        out = torch.zeros(64, dtype=torch.uint32)
        blocks[(1,)](out, seed, *cols, 16)
        got = out.numpy().reshape(16, 4)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for r in range(16):
            np.testing.assert_array_equal(oracle.philox4x32_10(ctr[r], key), got[r])


def test_coordinates_follow_the_documented_stream():
    seed, qid, point, m = 99 + (7 << 40), 3 + (5 << 33), 12345, 784
    for s in range(0, 40):
        assert oracle.coordinate(seed, qid, point, s, m) == _philox_ref.scaled(seed, qid, point, s, m)
    # masks clear the point and query fields of the counter
    for s in range(8):
        w = _philox_ref.word(seed, 0, 0, s)
        assert oracle.coordinate(seed, qid, point, s, m, mask_p=0, mask_q=0) == (w * m) >> 32


def test_coordinates_uniform():
    m = 97
    js = np.array([oracle.coordinate(5, 1, 2, s, m) for s in range(20000)])
    assert js.min() >= 0 and js.max() < m
    counts = np.bincount(js, minlength=m)
    chi2 = ((counts - len(js) / m) ** 2 / (len(js) / m)).sum()
    assert chi2 < stats.chi2.ppf(0.9999, m - 1)


def test_share_mask_makes_coordinates_common():
    a = [oracle.coordinate(1, 0, 10, s, 500, mask_p=0) for s in range(32)]
    b = [oracle.coordinate(1, 0, 77, s, 500, mask_p=0) for s in range(32)]
    c = [oracle.coordinate(1, 0, 77, s, 500) for s in range(32)]
    assert a == b and a != c


# ------------------------------------------------------------------- alpha

def test_alpha_footnote_special_value():
    # delta' = exp(-e): log(1/delta') = e and log log(1/delta') = 1; at u = 1
    # the last term vanishes, so beta = e + 3 and alpha = sqrt(2 (e + 3)).
    d = math.exp(-math.e)
    assert oracle.alpha("footnote", 1, 1, d) == pytest.approx(math.sqrt(2 * (math.e + 3)), rel=1e-12)


def test_alpha_lemma_special_value():
    # 125 log(1.12) / delta' = e^10 gives beta(1) = 20 and alpha(1) = sqrt(40).
    d = 125 * math.log(1.12) / math.exp(10)
    assert oracle.alpha("lemma", 1, 1, d) == pytest.approx(math.sqrt(40.0), rel=1e-12)


def test_alpha_exp_special_value():
    # n / delta = e^5 - 1 gives log(1 + n/delta) = 5 at u = 1.
    d = 1.0 / (math.exp(5) - 1)
    for c in (1.0, 0.01):
        assert oracle.alpha("exp", 1, 1, d, c_alpha=c) == pytest.approx(math.sqrt(5 * c), rel=1e-12)


# alpha at u > 1. Each case fixes delta so the delta-dependent part takes a
# known constant, then compares with decimal values worked out by hand from
# the bound's definition (natural logarithms throughout), so the u-dependent
# terms are pinned: a wrong factor (3 for 1.5), a base-2 logarithm, a dropped
# "1 +", u in place of 1/u, or delta in place of delta' = delta / n fails.
# n = 10 so that the division by n is exercised too.

@pytest.mark.parametrize("u,expected", [
    # delta' = exp(-e): log(1/delta') + 3 log log(1/delta') = e + 3 = 5.718281828...
    # u = 2:     ln 2 = 0.693147181, ln(1.693147181) = 0.526589034, x 1.5 = 0.789883551,
    #            beta = 6.508165380, alpha = sqrt(2 beta / 2) = 2.551110617
    (2, 2.551110617),
    # u = 10:    ln 10 = 2.302585093, ln(3.302585093) = 1.194705523, x 1.5 = 1.792058285,
    #            beta = 7.510340113, alpha = sqrt(2 beta / 10) = 1.225588847
    (10, 1.225588847),
    # u = 12288: ln 12288 = ln 3 + 12 ln 2 = 9.416378455, ln(10.416378455) = 2.343379419,
    #            x 1.5 = 3.515069128, beta = 9.233350957, alpha = sqrt(2 beta / 12288) = 0.03876627463
    (12288, 0.03876627463),
])
def test_alpha_footnote_values_above_one(u, expected):
    n = 10
    d = n * math.exp(-math.e)          # delta' = delta / n = exp(-e)
    assert oracle.alpha("footnote", u, n, d) == pytest.approx(expected, rel=2e-9)


@pytest.mark.parametrize("u,expected", [
    # delta' = 125 ln(1.12) / e^10, so beta(u) = 20 + 2 ln(ln(1.12 u) / ln(1.12)); ln 1.12 = 0.1133286853
    # u = 2:     ln 2.24 = 0.8064758659, ratio 7.116255374, ln = 1.962381656, beta = 23.92476331,
    #            alpha = sqrt(2 beta / 2) = 4.891294646
    (2, 4.891294646),
    # u = 10:    ln 11.2 = 2.415913778, ratio 21.31776056, ln = 3.059540555, beta = 26.11908111,
    #            alpha = sqrt(2 beta / 10) = 2.285566937
    (10, 2.285566937),
    # u = 12288: ln 13762.56 = 9.529707141, ratio 84.08909990, ln = 4.431876950, beta = 28.86375390,
    #            alpha = sqrt(2 beta / 12288) = 0.06854105785
    (12288, 0.06854105785),
])
def test_alpha_lemma_values_above_one(u, expected):
    n = 10
    d = n * 125 * math.log(1.12) / math.exp(10)
    assert oracle.alpha("lemma", u, n, d) == pytest.approx(expected, rel=2e-9)


@pytest.mark.parametrize("u,c,expected", [
    # delta = n (1 + ln u) / (e^5 - 1) makes (1 + ln u) n / delta = e^5 - 1, so the
    # logarithm is exactly 5 and alpha(u) = sqrt(5 C_alpha / u).
    (2, 1.0, 1.581138830),        # sqrt(2.5)
    (2, 1e-3, 0.05),              # sqrt(0.0025)
    (10, 1.0, 0.7071067812),      # sqrt(0.5)
    (12288, 1.0, 0.02017178826),  # sqrt(5 / 12288)
])
def test_alpha_exp_values_above_one(u, c, expected):
    n = 10
    d = n * (1.0 + math.log(u)) / (math.exp(5) - 1)
    assert oracle.alpha("exp", u, n, d, c_alpha=c) == pytest.approx(expected, rel=2e-9)


@pytest.mark.parametrize("form", ["footnote", "lemma", "exp"])
def test_alpha_decreasing_and_lil_rate(form):
    a = np.array([oracle.alpha(form, u, 1000, 0.01) for u in range(1, 5000)])
    assert np.all(np.diff(a) < 0)
    # alpha(u) sqrt(u) grows at most like sqrt(log log u): doubly logarithmic.
    g = a * np.sqrt(np.arange(1, 5000))
    assert g[-1] / g[10] < 1.5


def test_alpha_lemma_coverage():
    """Lemma probound: with prob >= 1 - delta' the running mean of [0,1]
    samples stays within alpha(t) of its mean for every t. Bernoulli arms."""
    rng = np.random.default_rng(0)
    n_arms, horizon, delta = 400, 3000, 0.04
    ts = np.arange(1, horizon + 1)
    for form in ("footnote", "lemma"):
        al = np.array([oracle.alpha(form, t, 1, delta) for t in ts])
        viol = 0
        for p in (0.5, 0.1):
            x = rng.random((n_arms, horizon)) < p
            means = np.cumsum(x, axis=1) / ts
            viol += np.any(np.abs(means - p) > al, axis=1).sum()
        assert viol <= stats.binom.ppf(0.999, 2 * n_arms, delta)


# ------------------------------------------------------------- brute force

def test_exact_knn_matches_numpy_with_ties():
    rng = np.random.default_rng(1)
    for trial in range(20):
        n, m, k = int(rng.integers(5, 17)), int(rng.integers(1, 9)), int(rng.integers(1, 5))
        X = rng.integers(-2, 3, size=(n, m)).astype(np.float32)   # many exact ties
        q = rng.integers(-2, 3, size=(1, m)).astype(np.float32)
        d = ((X.astype(np.float64) - q) ** 2).sum(1)
        order = np.lexsort((np.arange(n), d))[:k]
        idx, dist = oracle.exact_knn(X, q, k)
        np.testing.assert_array_equal(idx[0], order)
        np.testing.assert_allclose(dist[0], d[order], rtol=0, atol=0)


# --------------------------------------------------------------- adaptive

def _params(**kw):
    base = dict(k=5, delta=0.01, bound="exp", c_alpha=1e-4, B0=16, B=16, grow=0, seed=0)
    base.update(kw)
    return oracle.make_params(**base)


def test_all_coordinates_gives_exact_result():
    """T = m means the distance is computed exactly (Algorithm 1)."""
    X, Q, _ = synth.gaussian_planted(300, 24, 4, seed=3)
    p = _params(k=4, B0=24, bound="footnote")
    r = oracle.adaptive(X, Q, p)
    d = ((X.astype(np.float64) - Q[0].astype(np.float64)) ** 2).sum(1)
    st = r["stats"][0]
    assert st["evals"] == 300 * 24 and st["rounds"] == 1
    np.testing.assert_allclose(r["S"][0], d, rtol=1e-12)
    true8 = np.lexsort((np.arange(300), d))[:8]
    assert set(r["idx"][0][: st["count"]]) <= set(true8) | set(r["idx"][0])
    assert set(np.lexsort((np.arange(300), d))[:4]) <= set(r["idx"][0][: st["count"]])


def test_estimates_are_sample_means_of_drawn_coordinates():
    """S is the sum of squared differences at the coordinates the documented
    Philox4x32 stream selects, for T samples (sampled estimator, Section 4)."""
    X, Q, _ = synth.gaussian_planted(40, 64, 3, seed=4)
    p = _params(k=3, B0=8, B=8, c_alpha=1e-3, seed=11)
    r = oracle.adaptive(X, Q, p)
    for i in range(40):
        T = int(r["T"][0, i])
        if T >= 64:
            exp = ((X[i].astype(np.float64) - Q[0]) ** 2).sum()
        else:
            js = []
            for s in range(T):
                js.append(_philox_ref.scaled(11, 0, i, s, 64))
            js = np.array(js)
            exp = ((X[i, js].astype(np.float64) - Q[0, js].astype(np.float64)) ** 2).sum()
        assert r["S"][0, i] == pytest.approx(exp, rel=1e-12, abs=0)


def test_schedule_does_not_change_the_stream():
    X, Q, _ = synth.gaussian_planted(500, 128, 5, seed=5)
    a = oracle.adaptive(X, Q, _params(B0=16, B=16))
    b = oracle.adaptive(X, Q, _params(B0=8, B=8))
    same = a["T"][0] == b["T"][0]
    assert same.sum() > 50
    np.testing.assert_array_equal(a["S"][0][same], b["S"][0][same])


def test_size_and_state_invariants():
    rng = np.random.default_rng(7)
    for trial in range(12):
        n, m, k = int(rng.integers(30, 400)), int(rng.integers(8, 200)), int(rng.integers(1, 6))
        h = int(rng.integers(0, 6))
        X, Q, _ = synth.gaussian_planted(n, m, k, seed=100 + trial)
        p = _params(k=k, h=h, B0=int(rng.integers(1, 20)), B=int(rng.integers(1, 20)), grow=trial % 2,
                    c_alpha=float(10 ** rng.uniform(-5, -2)), seed=trial)
        r = oracle.adaptive(X, Q, p)
        st = r["stats"][0]
        kind = r["code"][0] & 3
        assert st["count"] <= k + h
        out = r["idx"][0][: st["count"]]
        assert len(set(out)) == len(out) and np.all(r["idx"][0][st["count"]:] == -1)
        # candidates are exactly the accepted and still-active points (truncated)
        live = np.flatnonzero(kind != oracle.ELIMINATED)
        assert set(out) <= set(live)
        if len(live) <= k + h:
            assert set(out) == set(live)
        assert (kind == oracle.ACCEPTED).sum() < 2 * k
        # evaluation count = samples drawn + m per exact distance; an exact
        # point also drew every sample of the rounds before its exact round
        T = r["T"][0]
        tb, rr = 0, 0
        while True:
            br = p.B0 if rr == 0 else (max(p.B, tb) if p.grow else p.B)
            if tb + br >= m:
                break
            tb, rr = tb + br, rr + 1
        ex = T == m
        assert st["evals"] == T[~ex].sum() + ex.sum() * (tb + m)


def test_trivial_when_n_le_k_plus_h():
    X, Q, _ = synth.gaussian_planted(9, 16, 4, seed=1)
    r = oracle.adaptive(X, Q, _params(k=4, h=5))
    assert r["stats"][0]["evals"] == 0
    assert list(r["idx"][0]) == list(range(9))


def test_degenerate_identical_points():
    X = np.ones((50, 16), dtype=np.float32)
    q = np.ones((1, 16), dtype=np.float32)
    r = oracle.adaptive(X, q, _params(k=3, h=2, bound="footnote"))
    st = r["stats"][0]
    assert st["term"] == 3 and st["count"] == 5
    assert list(r["idx"][0]) == [0, 1, 2, 3, 4]


def test_coherent_axis_gives_no_savings():
    """Section 4.2: points on one axis need m samples each (theory bound)."""
    X, q = synth.coherent_axis(200, 256, axis=17, seed=2)
    p = _params(k=5, bound="footnote", B0=16, B=16)
    r = oracle.adaptive(X, q, p)
    st = r["stats"][0]
    rounds = r["code"][0] >> 2
    assert st["rounds"] == 16                            # 15 sampled rounds, then the exact one
    assert np.all(rounds == st["rounds"] - 1)          # nothing decided before the exact round
    assert st["evals"] == 200 * (240 + 256)
    ti, _ = oracle.exact_knn(X, q, 5)
    assert set(ti[0]) <= set(r["idx"][0][: st["count"]])


def test_containment_rate_binary_data():
    """Theorem 1: the returned set contains the k nearest neighbours with
    probability >= 1 - delta. Binary +-1/2 data (Theorem 2's model), where a
    sample is an exact Bernoulli draw of the normalised distance."""
    trials, delta, k = 150, 0.05, 3
    fails, saved = 0, 0
    for t in range(trials):
        X, q, near = synth.binary_half(150, 2048, k, 0.05, 0.45, seed=1000 + t)
        p = oracle.make_params(k, delta=delta, bound="footnote", B0=32, B=32, grow=1, seed=t)
        r = oracle.adaptive(X, q, p)
        st = r["stats"][0]
        ti, _ = oracle.exact_knn(X, q, k)
        fails += not set(ti[0]) <= set(r["idx"][0][: st["count"]])
        saved += st["evals"] < 150 * 2048
    assert fails <= stats.binom.ppf(0.999, trials, delta)
    assert saved >= 0.9 * trials    # the bound is not saturated here: adaptivity must pay


def test_easy_instance_recall_and_savings():
    X, Q, planted = synth.gaussian_planted(2000, 256, 5, seed=0)
    ti, _ = oracle.exact_knn(X, Q, 5)
    r = oracle.adaptive(X, Q, _params(k=5, c_alpha=1e-4))
    st = r["stats"][0]
    assert set(ti[0]) <= set(r["idx"][0][: st["count"]])
    assert st["evals"] < 0.15 * 2000 * 256


def test_replay_of_own_log_is_clean_and_detects_a_planted_error():
    X, Q, _ = synth.gaussian_planted(800, 128, 5, seed=9)
    p = _params(c_alpha=3e-4)
    r = oracle.adaptive(X, Q, p)
    rr = oracle.adaptive(X, Q, p, replay=r["code"])
    s = rr["stats"][0]
    assert s["mismatch"] == 0 and s["near_disagree"] == 0 and s["log_inconsistent"] == 0
    np.testing.assert_array_equal(rr["code"], r["code"])
    bad = r["code"].copy()
    i = int(np.flatnonzero((bad[0] & 3) == oracle.ELIMINATED)[0])
    bad[0, i] = (bad[0, i] & ~3) | oracle.ACCEPTED           # flip one logged decision
    rb = oracle.adaptive(X, Q, p, replay=bad)
    assert rb["stats"][0]["mismatch"] + rb["stats"][0]["near_disagree"] >= 1


# ------------------------------------------------------ Algorithm 1 (sequential)

def test_sequential_algorithm_contains_knn():
    fails = 0
    for t in range(20):
        X, q, near = synth.binary_half(60, 256, 3, 0.05, 0.45, seed=t)
        p = oracle.make_params(3, delta=0.05, bound="footnote", seed=t)
        idx, evals, iters = oracle.sequential(X, q, p)
        ti, _ = oracle.exact_knn(X, q, 3)
        assert len(set(idx)) == 6
        fails += not set(ti[0]) <= set(idx)
        assert evals <= 60 * 2 * 256
    assert fails <= 3


def test_sequential_and_batched_same_order_of_cost():
    X, q, _ = synth.binary_half(100, 1024, 3, 0.05, 0.45, seed=77)
    p = oracle.make_params(3, delta=0.05, bound="footnote", B0=8, B=8, grow=1, seed=1)
    _, ev_seq, _ = oracle.sequential(X, q, p)
    r = oracle.adaptive(X, q, p)
    ev_bat = r["stats"][0]["evals"]
    assert 0.1 < ev_bat / ev_seq < 10


# ------------------------------------------------------- stored copies (BF16 / FP8)

def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 10 ** rng.uniform(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, 1e-40])]).astype(np.float32)
    ours = np.array([oracle.lib().orc_round_bf16(float(v)) for v in x], dtype=np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(ours.view(np.uint32), ref.view(np.uint32))


def test_e4m3_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-0.05, 0.05, 5000),
                        np.array([2 ** -10, 3 * 2 ** -11, 2 ** -9, 447.9, 448.0, 15.5, 17.0, -2 ** -10])]
                       ).astype(np.float32)
    ours = np.array([oracle.lib().orc_round_e4m3(float(v)) for v in x], dtype=np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_quantize_rows_and_error():
    X, _ = synth.pixel_mixture(300, 50, 1, seed=2)
    X[7] = 0.0
    for st in ("bf16", "fp8"):
        G, scale, emax = oracle.quantize(X, st)
        assert emax == np.abs(G.astype(np.float64) - X).max()
        if st == "fp8":
            mx = np.abs(X).max(1)
            np.testing.assert_array_equal(scale, np.where(mx > 0, (mx / np.float32(448)).astype(np.float32), 1))
            assert np.all(np.abs(G) <= np.abs(X).max(1, keepdims=True) * (1 + 2 ** -20))
            assert np.all(G[7] == 0)
    assert oracle.quantize(X, "bf16")[2] <= 2 ** -9 * np.abs(X).max()


def test_lossless_bf16_copy_reproduces_the_fp32_run():
    """Integers 0..255 are exact in BF16: the copy equals the data, the
    widening is zero, and every decision must be the FP32 run's."""
    X, Q, _ = synth.gap_planted(3000, 64, 3, 5, [3.0, 1.5, 1.05], seed=6, background="int255")
    a = oracle.adaptive(X, Q, _params(c_alpha=1e-3, storage="f32"))
    b = oracle.adaptive(X, Q, _params(c_alpha=1e-3, storage="bf16"))
    np.testing.assert_array_equal(a["code"], b["code"])
    np.testing.assert_array_equal(a["idx"], b["idx"])


def test_stored_copies_keep_the_guarantee():
    """With the bound widened by the copy's error, Theorem 1's containment
    still holds (binary data: FP8 and BF16 are lossy only through the scale)."""
    X, Q, _ = synth.gaussian_planted(1500, 128, 4, nq=4, seed=8)
    ti, _ = oracle.exact_knn(X, Q, 4)
    for st in ("bf16", "fp8"):
        r = oracle.adaptive(X, Q, _params(k=4, bound="footnote", storage=st))
        for q in range(4):
            c = r["stats"][q]["count"]
            assert c <= 8 and set(ti[q]) <= set(r["idx"][q][:c])


@pytest.mark.parametrize("target,decided", [("between_new_and_old", True), ("below_half_factor", False)])
def test_copy_width_after_round_0_uses_the_active_estimates(target, decided):
    """Closed-form case for the copy term of the width. Query and point 0 at
    0, points 1 and 2 at 257 (their BF16 copy holds 256: error e = 1), point 3
    at 4096 (exact; it fixes span = 4096 and leaves in round 0). In round 1 the
    active points' largest copy estimate is 256^2, so the copy term is
    e (2 * 256 + e) = 513 instead of the span form e (2 * 4096 + e) = 8193.
    Points 1 and 2 (estimate 65536) are eliminated and point 0 accepted in
    round 1 iff the width w1 = span'^2 alpha(4) + 513 is below 32768: alpha(4)
    is set so that this holds, but would fail with the span form (case 1), or
    so that it fails, but would hold with half the copy term (case 2)."""
    n, m, delta, e, span = 4, 32, 0.01, 1.0, 4096.0
    X = np.zeros((n, m), dtype=np.float32)
    X[1:3] = 257.0
    X[3] = 4096.0
    q = np.zeros((1, m), dtype=np.float32)
    _, _, emax = oracle.quantize(X, "bf16")
    assert emax == e
    sp2 = (span + 2 * e) ** 2
    lg = lambda u: math.log(1.0 + (1.0 + math.log(u)) * n / delta)
    if target == "between_new_and_old":
        a4 = (32768 - 0.5 * (513 + 8193)) / sp2          # w1 < 32768 with 513, > with 8193
    else:
        a4 = (32768 - 0.5 * (513 + 257)) / sp2           # w1 > 32768 with 513, < with 257
    c = a4 * a4 * 4 / lg(4)
    a2 = math.sqrt(c * lg(2) / 2)
    assert sp2 * a2 + e * (2 * span + e) > 32768         # round 0 decides points 0-2 neither way
    r = oracle.adaptive(X, q, oracle.make_params(1, h=0, delta=delta, bound="exp", c_alpha=c, B0=2, B=2,
                                                 storage="bf16"))
    rounds = r["code"][0] >> 2
    assert rounds[3] == 0 and (r["code"][0][3] & 3) == oracle.ELIMINATED
    if decided:
        assert r["stats"][0]["rounds"] == 2 and list(r["idx"][0]) == [0]
    else:
        assert np.all(rounds[:3] >= 2)


@pytest.mark.parametrize("target,decided", [("between_new_and_old", True), ("below_half_factor", False)])
def test_copy_width_in_round_0_uses_the_active_estimates(target, decided):
    """Closed-form case for the copy term in round 0. Query and point 0 at 0,
    points 1 and 2 at 257 (BF16 copy 256: e = 1), point 3 alternating -2048
    and +2048: it fixes span = 4096, yet each of its samples is 2048^2, so
    the largest round-0 estimate is 2048^2 and the copy term is
    e (2 * 2048 + e) = 4097 against the span form e (2 * 4096 + e) = 8193.
    Everything is decided in round 0 (point 0 accepted, 1-3 eliminated) iff
    w0 = span'^2 alpha(2) + 4097 is below 32768: alpha(2) is set so that this
    holds but would fail with the span form (case 1), or so that it fails but
    would hold with half the copy term (case 2)."""
    n, m, delta, e, span = 4, 32, 0.01, 1.0, 4096.0
    X = np.zeros((n, m), dtype=np.float32)
    X[1:3] = 257.0
    X[3, 0::2], X[3, 1::2] = -2048.0, 2048.0
    q = np.zeros((1, m), dtype=np.float32)
    _, _, emax = oracle.quantize(X, "bf16")
    assert emax == e
    sp2 = (span + 2 * e) ** 2
    lg = lambda u: math.log(1.0 + (1.0 + math.log(u)) * n / delta)
    if target == "between_new_and_old":
        a2 = (32768 - 0.5 * (4097 + 8193)) / sp2
    else:
        a2 = (32768 - 0.5 * (4097 + 2049)) / sp2
    c = a2 * a2 * 2 / lg(2)
    r = oracle.adaptive(X, q, oracle.make_params(1, h=0, delta=delta, bound="exp", c_alpha=c, B0=2, B=2,
                                                 storage="bf16"))
    rounds = r["code"][0] >> 2
    if decided:
        assert r["stats"][0]["rounds"] == 1 and list(r["idx"][0]) == [0]
        assert np.all(rounds == 0) and np.all((r["code"][0][1:] & 3) == oracle.ELIMINATED)
    else:
        assert r["stats"][0]["rounds"] >= 2 and np.all(rounds[:3] >= 1)


def test_batch_past_m_is_round_0_then_exact_distances():
    """A later-round batch past m (the exact cap T + B >= m): a point is
    decided in round 0 (T = B0) or ends at T = m with its sum the exact
    squared distance and m evaluations more; the planted nearest, kept by
    round 0, are returned."""
    n, m, k = 2000, 96, 5
    X, Q, _ = synth.gaussian_planted(n, m, k, seed=11)
    r = oracle.adaptive(X, Q, _params(k=k, B0=16, B=1 << 20, grow=0, c_alpha=1e-3))
    st = r["stats"][0]
    T = r["T"][0]
    assert st["rounds"] <= 2 and set(np.unique(T).tolist()) <= {16, m}
    full = T == m
    assert 0 < full.sum() < n
    d = ((X.astype(np.float64) - Q[0].astype(np.float64)) ** 2).sum(axis=1)
    np.testing.assert_allclose(r["S"][0][full], d[full], rtol=1e-12)
    assert st["evals"] == n * 16 + int(full.sum()) * m
    ti, _ = oracle.exact_knn(X, Q[:1], k)
    assert set(ti[0].tolist()) <= set(r["idx"][0][: st["count"]].tolist())
