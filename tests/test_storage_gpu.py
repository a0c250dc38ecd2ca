"""Mixed-precision storage (BF16, FP8-e4m3 with per-row scale): the GPU's
copies, their error bounds and the adaptive rounds over them, against the
oracle's own quantisers and replay."""

import numpy as np
import pytest
import torch

import oracle
from _parity import check as check_f32
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def replay(X, Q, ds, storage, k, delta=0.01, seed=0, **opt):
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    g = ds.adaptive(Qd, k, delta, seed, storage=storage, trace=True, **opt)
    torch.cuda.synchronize()
    g = {key: v.cpu().numpy() for key, v in g.items()}
    oopt = {kk: v for kk, v in opt.items() if kk in ("h", "bound", "c_alpha", "B0", "B", "grow", "qid_base")}
    qid_base = oopt.pop("qid_base", 0)
    for q in range(Q.shape[0]):
        p = oracle.make_params(k, delta=delta, seed=seed, qid=qid_base + q, tol=TOL, storage=storage, **oopt)
        o = oracle.adaptive(X, Q[q:q + 1], p, replay=g["code"][q:q + 1])
        st = o["stats"][0]
        assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (storage, q, st)
        np.testing.assert_array_equal(o["code"][0], g["code"][q])
        assert int(g["evals"][q]) == st["evals"] and int(g["count"][q]) == st["count"]
        So, Sg = o["S"][0], g["S"][q].astype(np.float64)
        rel = np.abs(Sg - So) / np.maximum(So, 1e-300)
        rel[(So == 0) & (Sg == 0)] = 0
        assert rel.max() <= TOL, (storage, q, rel.max())
    return g


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_copy_error_matches_oracle_quantiser(storage):
    X, _ = synth.pixel_mixture(5000, 300, 1, seed=1)
    X[11] = 0.0
    with knn.Dataset(torch.from_numpy(X).cuda(), copies=(storage,)) as ds:
        _, _, emax = oracle.quantize(X, storage)
        assert ds.error(storage) == np.float32(emax)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_rounds_over_copies_replay(storage):
    X, Q = synth.pixel_mixture(6000, 784, 6, seed=2)
    with knn.Dataset(torch.from_numpy(X).cuda(), copies=(storage,)) as ds:
        replay(X, Q, ds, storage, 10, bound="exp", c_alpha=3e-3, B0=16, B=16, grow=1)
        replay(X, Q, ds, storage, 10, bound="footnote", B0=32, B=32, grow=1)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_copies_gaussian_and_ragged_dims(storage):
    for m in (96, 77, 5):
        X, Q, _ = synth.gaussian_planted(3000, m, 4, nq=3, seed=m)
        with knn.Dataset(torch.from_numpy(X).cuda(), copies=(storage,)) as ds:
            replay(X, Q, ds, storage, 4, bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
@pytest.mark.parametrize("n,k", [(200, 20), (6000, 5)])
def test_round0_copy_width_from_largest_estimate(storage, n, k):
    """N(0,1)-like data, where the largest round-0 estimate sits well below
    the squared span: round 0 takes the copy term from it. n = 200 with k = 20
    has fewer tiles of round-0 minima than k (no round-0 filter: the maximum
    comes from the round's sums); n = 6000 runs the filter (the maximum over
    every round-0 sum, before it drops points)."""
    X, Q, _ = synth.gaussian_planted(n, 256, k, nq=4, seed=n + k)
    with knn.Dataset(torch.from_numpy(X).cuda(), copies=(storage,)) as ds:
        replay(X, Q, ds, storage, k, h=min(k, n - k), bound="exp", c_alpha=1e-3, B0=16, B=16, grow=1)


def test_f32_dataset_equals_knn_adaptive():
    X, Q = synth.pixel_mixture(8000, 256, 8, seed=3)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with knn.Dataset(Xd, copies=()) as ds:
        a = ds.adaptive(Qd, 10, 0.01, 5, bound="exp", c_alpha=1e-3, trace=True)
    b = knn.adaptive(Xd, Qd, 10, 0.01, 5, bound="exp", c_alpha=1e-3, trace=True)
    for key in a:
        assert torch.equal(a[key], b[key]), key


def test_lossless_bf16_copy_reproduces_f32_on_gpu():
    X, Q, _ = synth.gap_planted(5000, 64, 4, 5, [3.0, 1.5, 1.05, 2.0], seed=6, background="int255")
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        assert ds.error("bf16") == 0.0
        a = ds.adaptive(Qd, 5, 0.01, 0, storage="bf16", bound="exp", c_alpha=1e-3, trace=True)
        b = ds.adaptive(Qd, 5, 0.01, 0, storage="f32", bound="exp", c_alpha=1e-3, trace=True)
        for key in a:
            assert torch.equal(a[key], b[key]), key


def test_recall_after_rerank_from_copies():
    X, Q = synth.pixel_mixture(20000, 784, 32, seed=9)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    ti, _ = oracle.exact_knn(X, Q, 10)
    with knn.Dataset(Xd, copies=("bf16", "fp8")) as ds:
        for storage in ("bf16", "fp8"):
            r = ds.adaptive(Qd, 10, 0.01, 0, storage=storage, bound="footnote", B0=16, B=16, grow=1)
            ri, _ = knn.rerank(Xd, Qd, r["idx"], 10)
            np.testing.assert_array_equal(np.sort(ri.cpu().numpy(), 1), np.sort(ti, 1))
