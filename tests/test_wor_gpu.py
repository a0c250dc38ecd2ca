"""Draws without replacement on the GPU (each pair's keyed permutation of
[0, m)): lock-step replay in the oracle through the standalone call (round 0
in place) and a dataset (the point-major round-0 pass and its filter), ragged
and tiny dimensions, both metrics, thread counts; the draws differ from the
with-replacement stream; the option's limits."""

import numpy as np
import pytest
import torch

import oracle
from _parity import check
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("m", [784, 100, 77, 33, 5])
def test_standalone_replay(m):
    X, Q = synth.pixel_mixture(4000, m, 5, seed=m)
    summ, gpu = check(X, Q, 10, delta=0.01, seed=3, bound="exp", c_alpha=1e-3, B0=2, B=2, grow=1, replace=False)
    assert summ["queries"] == 5
    base = check(X, Q, 10, delta=0.01, seed=3, bound="exp", c_alpha=1e-3, B0=2, B=2, grow=1)[1]
    assert not np.array_equal(base["S"], gpu["S"])  # another stream of draws


@pytest.mark.parametrize("B0,B,grow,threads", [(1, 1, 0, 256), (16, 16, 1, 1024), (40, 8, 0, 512)])
def test_standalone_schedules_and_threads(B0, B, grow, threads):
    X, Q, _ = synth.gaussian_planted(3000, 256, 6, nq=3, seed=B0)
    check(X, Q, 6, delta=0.05, seed=7, bound="exp", c_alpha=3e-4, B0=B0, B=B, grow=grow, threads=threads,
          replace=False)


def _replay_ds(X, Q, res, k, metric="l2", **opt):
    g = {key: v.cpu().numpy() for key, v in res.items()}
    for q in range(Q.shape[0]):
        p = oracle.make_params(k, delta=0.01, seed=4, qid=q, tol=TOL, metric=metric, replace=False, **opt)
        o = oracle.adaptive(X, Q[q:q + 1], p, replay=g["code"][q:q + 1])
        st = o["stats"][0]
        assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (q, st)
        np.testing.assert_array_equal(o["code"][0], g["code"][q])
        assert int(g["evals"][q]) == st["evals"] and int(g["count"][q]) == st["count"]
        So, Sg = o["S"][0], g["S"][q].astype(np.float64)
        rel = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-300)
        rel[(So == 0) & (Sg == 0)] = 0
        assert rel.max() <= TOL, (q, rel.max())


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_dataset_round0_pass_and_filter(metric):
    """A dataset runs round 0 point-major (the filter drops the provably
    eliminated points); the same rounds as the standalone call, replayed."""
    X, Q = synth.pixel_mixture(20000, 300, 12, seed=9)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1)
    with knn.Dataset(Xd, copies=()) as ds:
        a = ds.adaptive(Qd, 10, 0.01, 4, trace=True, metric=metric, replace=False, **opt)
    b = knn.adaptive(Xd, Qd, 10, 0.01, 4, trace=True, metric=metric, replace=False, **opt)
    for key in a:
        assert torch.equal(a[key], b[key]), key
    torch.cuda.synchronize()
    _replay_ds(X, Q, a, 10, metric=metric, **opt)


def test_mixed_batch_same_as_alone():
    X, Q = synth.pixel_mixture(8000, 128, 6, seed=2)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1, replace=False)
    ks = np.array([1, 5, 10, 3, 7, 10], dtype=np.int32)
    qids = np.arange(6, dtype=np.int64) * 5 + 3
    with knn.Dataset(Xd, copies=()) as ds:
        mix = ds.adaptive_multi(Qd, torch.from_numpy(ks).cuda(), 10, torch.from_numpy(qids).cuda(), 0.01, 2, **opt)
        for q in range(6):
            solo = ds.adaptive(Qd[q:q + 1], int(ks[q]), 0.01, 2, qid_base=int(qids[q]), **opt)
            c = int(solo["count"][0])
            assert int(mix["count"][q]) == c and int(mix["evals"][q]) == int(solo["evals"][0])
            assert torch.equal(mix["idx"][q, :c], solo["idx"][0, :c])


def test_option_limits():
    X, Q, _ = synth.gaussian_planted(500, 32, 2, nq=1, seed=1)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with pytest.raises(knn.KnnError):
        knn.adaptive(Xd, Qd, 2, 0.01, 0, block=8, replace=False)
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        with pytest.raises(knn.KnnError):
            ds.adaptive(Qd, 2, 0.01, 0, storage="bf16", replace=False)
