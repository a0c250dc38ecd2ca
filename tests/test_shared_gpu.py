"""Shared coordinates (Philox counter masks zero): the column-permuted copies
must give exactly what the per-pair draws give, and follow the oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

SH = dict(share_points=True, share_queries=True)


@pytest.mark.parametrize("m,B0", [(784, 8), (784, 16), (77, 12), (5, 3), (300, 32), (784, 64), (200, 40), (100, 24)])
def test_shared_copies_equal_per_pair_draws(m, B0):
    X, Q = synth.pixel_mixture(12000, m, 24, seed=m)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=B0, B=8, grow=1, **SH)
    with knn.Dataset(Xd, copies=("bf16", "fp8")) as ds:
        before = {st: ds.adaptive(Qd, 10, 0.01, 42, storage=st, trace=True, **opt) for st in ("f32", "bf16", "fp8")}
        ds.share(42, copies=("f32", "bf16", "fp8"))
        for st in ("f32", "bf16", "fp8"):
            after = ds.adaptive(Qd, 10, 0.01, 42, storage=st, trace=True, **opt)
            for key in after:
                assert torch.equal(after[key], before[st][key]), (st, key)
        raw = knn.adaptive(Xd, Qd, 10, 0.01, 42, trace=True, **opt)
        f32 = ds.adaptive(Qd, 10, 0.01, 42, storage="f32", trace=True, **opt)
        for key in raw:
            assert torch.equal(raw[key], f32[key]), key
        # another seed falls back to drawing per pair, still consistent
        other = ds.adaptive(Qd, 10, 0.01, 7, storage="f32", **opt)
        raw7 = knn.adaptive(Xd, Qd, 10, 0.01, 7, **opt)
        assert torch.equal(other["idx"], raw7["idx"]) and torch.equal(other["evals"], raw7["evals"])


def test_shared_path_replays_in_the_oracle():
    X, Q, _ = synth.gaussian_planted(6000, 128, 5, nq=4, seed=3)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with knn.Dataset(Xd, copies=()) as ds:
        ds.share(9, copies=("f32",))
        g = ds.adaptive(Qd, 5, 0.01, 9, trace=True, bound="exp", c_alpha=1e-3, B0=16, B=16, grow=1, **SH)
        torch.cuda.synchronize()
    code = g["code"].cpu().numpy()
    p = oracle.make_params(5, delta=0.01, bound="exp", c_alpha=1e-3, B0=16, B=16, grow=1, seed=9,
                           share_points=True, share_queries=True)
    o = oracle.adaptive(X, Q, p, replay=code)
    for q, st in enumerate(o["stats"]):
        assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, st
        assert int(g["evals"][q]) == st["evals"]
    np.testing.assert_array_equal(o["code"], code)
