"""Maximum and empty sizes through the C ABI: k + h = 1024 (the largest
candidate set), m = 16384 (the widest row, with shared coordinates too), no
queries at all, and arguments past the limits refused."""

import numpy as np
import pytest
import torch

from _parity import check
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu


def test_largest_candidate_set():
    X, Q = synth.pixel_mixture(3000, 32, 2, seed=1)
    summ, g = check(X, Q, 600, h=424, delta=0.01, seed=1, bound="exp", c_alpha=1e-3, B0=4, B=4, grow=1)
    assert np.all(g["count"] <= 1024) and np.all(g["count"] >= 600)


@pytest.mark.parametrize("share", [False, True])
def test_widest_rows(share):
    X, Q, _ = synth.gaussian_planted(300, 16384, 3, nq=2, seed=2)
    if not share:
        check(X, Q, 3, delta=0.01, seed=2, bound="exp", c_alpha=1e-3, B0=64, B=64, grow=1)
        return
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=64, B=64, grow=1, share_points=True, share_queries=True)
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        ds.share(2, copies=("f32", "bf16"))
        a = ds.adaptive(Qd, 3, 0.01, 2, trace=True, **opt)
        b = knn.adaptive(Xd, Qd, 3, 0.01, 2, trace=True, **opt)
        for key in a:
            assert torch.equal(a[key], b[key]), key
        ds.adaptive(Qd, 3, 0.01, 2, storage="bf16", **opt)
    torch.cuda.synchronize()


def test_no_queries():
    X, Q, _ = synth.gaussian_planted(500, 16, 2, nq=1, seed=3)
    Xd = torch.from_numpy(X).cuda()
    Q0 = torch.empty((0, 16), dtype=torch.float32, device="cuda")
    r = knn.adaptive(Xd, Q0, 2, 0.01, 0)
    assert r["idx"].shape == (0, 4) and r["count"].numel() == 0
    with knn.Dataset(Xd, copies=("screen",)) as ds:
        r = ds.adaptive(Q0, 2, 0.01, 0)
        assert r["count"].numel() == 0
        gi, gd = ds.exact(Q0, 2)
        assert gi.shape == (0, 2)
    gi, gd = knn.exact(Xd, Q0, 2)
    assert gi.shape == (0, 2)


def test_past_the_limits_refused():
    X = torch.zeros((10, 16385), dtype=torch.float32, device="cuda")
    Q = torch.zeros((1, 16385), dtype=torch.float32, device="cuda")
    with pytest.raises(knn.KnnError):
        knn.adaptive(X, Q, 2, 0.01, 0)                      # m above 16384
    X = torch.zeros((2000, 8), dtype=torch.float32, device="cuda")
    Q = torch.zeros((1, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(knn.KnnError):
        knn.adaptive(X, Q, 600, 0.01, 0, h=425)              # k + h above 1024
    with pytest.raises(knn.KnnError):
        knn.adaptive(X, Q, 2, 1.5, 0)                        # delta outside (0, 1)
