"""Round 0 from the point-major pass drops the points that the tile minima of
the round-0 sums already prove eliminated. The rounds must be exactly those
of the unfiltered path (knn_adaptive draws round 0 in place): same decision
log, sums, evaluation counts and candidates; and they replay in the oracle."""

import numpy as np
import pytest
import torch

from _parity import check
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu


def _same(a, b):
    for key in a:
        assert torch.equal(a[key], b[key]), key


@pytest.mark.parametrize("k,gap", [(1, 20.0), (5, 20.0), (10, 3.0), (10, 1.05), (50, 1.5)])
def test_filtered_round0_equals_in_place_round0(k, gap):
    """Wide gaps leave only the k planted points after the filter (the
    (k+1)-th smallest LCB is then a dropped point's); narrow gaps keep many."""
    X, Q, _ = synth.gap_planted(20000, 96, 12, k, gap, seed=int(gap * 10) + k)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    for opt in (dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1), dict(bound="exp", c_alpha=1e-5, B0=4, B=4),
                dict(bound="footnote", B0=16, B=16, grow=1)):
        with knn.Dataset(Xd, copies=()) as ds:
            a = ds.adaptive(Qd, k, 0.01, 3, trace=True, **opt)
        b = knn.adaptive(Xd, Qd, k, 0.01, 3, trace=True, **opt)
        _same(a, b)


def test_filtered_round0_shared_coordinates():
    X, Q, _ = synth.gap_planted(30000, 128, 16, 10, [4.0, 1.2] * 8, seed=3)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-4, B0=16, B=16, grow=1, share_points=True, share_queries=True)
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        ds.share(5, copies=("f32",))
        a = ds.adaptive(Qd, 10, 0.01, 5, trace=True, **opt)
    b = knn.adaptive(Xd, Qd, 10, 0.01, 5, trace=True, **opt)
    _same(a, b)


def test_fewer_tiles_than_k_keeps_every_point():
    # 200 points in rows of 32 per tile: 7 tiles < k = 20, so no filter
    X, Q, _ = synth.gaussian_planted(200, 64, 20, nq=3, seed=4)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=8, B=8)
    with knn.Dataset(Xd, copies=()) as ds:
        a = ds.adaptive(Qd, 20, 0.01, 1, trace=True, h=5, **opt)
    b = knn.adaptive(Xd, Qd, 20, 0.01, 1, trace=True, h=5, **opt)
    _same(a, b)


def test_filtered_round0_replays_in_the_oracle():
    X, Q, _ = synth.gap_planted(15000, 200, 6, 5, [20.0, 3.0, 1.05, 2.0, 1.2, 8.0], seed=9)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with knn.Dataset(Xd, copies=()) as ds:
        g = ds.adaptive(Qd, 5, 0.01, 2, trace=True, bound="exp", c_alpha=1e-4, B0=8, B=8, grow=1)
    gpu = {key: v.cpu().numpy() for key, v in g.items()}
    summ, _ = check(X, Q, 5, delta=0.01, seed=2, bound="exp", c_alpha=1e-4, B0=8, B=8, grow=1, gpu=gpu)
    assert summ["queries"] == 6


@pytest.mark.parametrize("n,k", [(320, 10), (321, 10), (352, 11), (2048, 64)])
def test_filter_with_as_many_tiles_as_k(n, k):
    """Tiles of 32 rows: n = 320 gives exactly k = 10 tile minima (the k-th
    smallest is the largest of them), 321 one more, 352 with k = 11 again
    exactly k; the rounds must equal the unfiltered path."""
    X, Q, _ = synth.gaussian_planted(n, 64, 2, nq=3, seed=n)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-4, B0=8, B=8, grow=1, h=min(k, n - k))
    with knn.Dataset(Xd, copies=()) as ds:
        a = ds.adaptive(Qd, k, 0.01, 6, trace=True, **opt)
    b = knn.adaptive(Xd, Qd, k, 0.01, 6, trace=True, **opt)
    _same(a, b)
