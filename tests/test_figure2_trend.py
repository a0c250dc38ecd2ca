"""The trend of Section 5's experiment (Figure 2) as a test: on the subspace
model x = c Q y, low intrinsic dimension p makes the adaptive method much
cheaper than the naive one while it still returns every true neighbour, and
at p = 1,000 the saving nearly disappears. Same sizes as the paper's
experiment (n = 1,000, m = 12,288, k = h = 10, delta = 0.001, the Section 5
bound), one C_alpha, medians over a few trials.

The CPU test runs the oracle; the GPU test runs the CUDA path through the
C ABI on the same inputs."""

import numpy as np
import pytest

import oracle
from paper_1902_09465_gb300 import synth

N, M, K, H, DELTA, C_ALPHA = 1000, 12288, 10, 10, 0.001, 1e-3
SCHED = dict(B0=16, B=16, grow=0)


def _inputs(p, t):
    return synth.subspace(N, M, p, nq=1, seed=7000 + 31 * p + t)


def _summary(ratios, recalls):
    return float(np.median(ratios)), float(np.median(recalls))


def _check_trend(low, high):
    (r10, rec10), (r1000, rec1000) = low, high
    # Section 5: low intrinsic dimension returns all k nearest at a small
    # fraction of the naive cost; at p = 1,000 the advantage nearly vanishes
    assert rec10 == 1.0, rec10
    assert r10 <= 0.25 * r1000, (r10, r1000)
    assert r1000 >= 0.5, r1000


def test_figure2_trend_oracle():
    out = {}
    for p in (10, 1000):
        ratios, recalls = [], []
        for t in range(4):
            X, Q = _inputs(p, t)
            ti, _ = oracle.exact_knn(X, Q, K)
            prm = oracle.make_params(K, h=H, delta=DELTA, bound="exp", c_alpha=C_ALPHA, seed=t, **SCHED)
            r = oracle.adaptive(X, Q, prm, want_state=False)
            st = r["stats"][0]
            got = set(r["idx"][0][: st["count"]].tolist())
            recalls.append(len(set(ti[0].tolist()) & got) / K)
            ratios.append(st["evals"] / (N * M))
        out[p] = _summary(ratios, recalls)
    _check_trend(out[10], out[1000])


@pytest.mark.gpu
def test_figure2_trend_gpu():
    import torch
    from paper_1902_09465_gb300 import knn

    out = {}
    for p in (10, 1000):
        ratios, recalls = [], []
        for t in range(6):
            X, Q = _inputs(p, t)
            Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
            ti, _ = oracle.exact_knn(X, Q, K)
            r = knn.adaptive(Xd, Qd, K, DELTA, t, h=H, bound="exp", c_alpha=C_ALPHA, **SCHED)
            cnt = int(r["count"][0])
            got = set(r["idx"][0, :cnt].cpu().tolist())
            recalls.append(len(set(ti[0].tolist()) & got) / K)
            ratios.append(int(r["evals"][0]) / (N * M))
        out[p] = _summary(ratios, recalls)
    _check_trend(out[10], out[1000])
