"""Round 0 under shared coordinates as a tcgen05 contraction (knn_opts
r0_tensor): every pair's sum over the shared columns is formed from centred
values split into three BF16 parts, the round-0 filter drops points on those
sums, and the kept points' sums are taken again sample by sample. Replayed
round by round in the oracle (exact FP64 sums): decisions, evaluation counts
and rounds must match outside the near-threshold band and every logged sum --
the dropped points' contraction sums included -- must lie within 1e-5 of the
oracle's."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

SH = dict(share_points=True, share_queries=True)
TOL = 1e-5


def _replay(X, Q, g, k, seed, storage, B0, B, grow, c_alpha, q):
    p = oracle.make_params(k, delta=0.01, bound="exp", c_alpha=c_alpha, B0=B0, B=B, grow=grow, seed=seed, qid=q,
                           share_points=True, share_queries=True, tol=TOL, storage=storage)
    o = oracle.adaptive(X, Q[q:q + 1], p, replay=g["code"][q:q + 1])
    st = o["stats"][0]
    assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (storage, q, st)
    np.testing.assert_array_equal(o["code"][0], g["code"][q])
    assert int(g["evals"][q]) == st["evals"] and int(g["count"][q]) == st["count"], (storage, q, st)
    assert int(g["rounds"][q]) == st["rounds"]
    So, Sg = o["S"][0], g["S"][q].astype(np.float64)
    rel = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-300)
    rel[(So == 0) & (Sg == 0)] = 0
    assert rel.max() <= TOL, (storage, q, rel.max(), int(rel.argmax()))
    return st


@pytest.mark.parametrize("data,B0", [("pixel", 16), ("pixel", 8), ("planted", 16), ("int255", 40), ("pixel", 64)])
def test_tensor_core_round0_replays_in_the_oracle(data, B0):
    if data == "pixel":
        X, Q = synth.pixel_mixture(24000, 200, 20, seed=B0)
        k = 10
    elif data == "planted":
        X, Q, _ = synth.gaussian_planted(20000, 128, 5, nq=20, seed=3)
        k = 5
    else:
        X, Q, _ = synth.gap_planted(16000, 96, 20, 10, 3.0, seed=5, background="int255")
        k = 10
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=B0, B=8, grow=1, **SH)
    with knn.Dataset(Xd, copies=("bf16", "fp8")) as ds:
        ds.share(13, copies=("f32", "bf16", "fp8"))
        for storage in ("f32", "bf16", "fp8"):
            g = ds.adaptive(Qd, k, 0.01, 13, storage=storage, trace=True, r0_tensor=True, **opt)
            plain = ds.adaptive(Qd, k, 0.01, 13, storage=storage, r0_tensor=False, **opt)
            torch.cuda.synchronize()
            assert knn.device_status() == 0
            g = {key: v.cpu().numpy() for key, v in g.items()}
            for q in (0, 7, 19):
                _replay(X, Q, g, k, 13, storage, B0, 8, 1, 1e-3, q)
            # the same candidates as sums taken sample by sample, up to
            # decisions at the threshold
            same = (g["count"] == plain["count"].cpu().numpy()).mean()
            assert same >= 0.9, (storage, same)


def test_tensor_core_round0_in_a_graph_and_mixed_batches():
    X, Q = synth.pixel_mixture(30000, 128, 64, seed=21)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    from paper_1902_09465_gb300 import runtime
    opt = dict(bound="exp", c_alpha=1e-3, B0=16, B=16, grow=1, r0_tensor=True, **SH)
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        ds.share(0, copies=("bf16",))
        eager = ds.adaptive(Qd, 10, 0.01, 0, storage="bf16", **opt)
        step = runtime.GraphStep(ds, 64, 10, 0.01, 0, storage="bf16", rerank=False, **opt)
        res, _, _ = step.run(Qd)
        torch.cuda.synchronize()
        for key in ("idx", "count", "evals", "rounds"):
            assert torch.equal(res[key], eager[key]), key
        ks = torch.full((64,), 10, dtype=torch.int32, device="cuda")
        qids = torch.arange(64, dtype=torch.int64, device="cuda")
        mix = ds.adaptive_multi(Qd, ks, 10, qids, 0.01, 0, storage="bf16", **opt)
        torch.cuda.synchronize()
        assert torch.equal(mix["evals"], eager["evals"]) and torch.equal(mix["count"], eager["count"])
