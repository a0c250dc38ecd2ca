"""Serving: mixed launches (per-query k and Philox query id) and the
continuously batched request loop give every query the same result alone and
in the mix; the loop respects its device-memory budget."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def two_datasets():
    A, PA = synth.mixture_planted(20000, 128, 64, seed=1)
    B, PB = synth.mixture_planted(15000, 96, 64, seed=2)
    dA = knn.Dataset(torch.from_numpy(A).cuda(), copies=("bf16", "screen"))
    dB = knn.Dataset(torch.from_numpy(B).cuda(), copies=("bf16", "screen"))
    yield (dA, dB), (PA, PB), (A, B)
    dA.close()
    dB.close()


def test_mixed_launch_equals_each_query_alone(two_datasets):
    (dA, _), (PA, _), _ = two_datasets
    rng = np.random.default_rng(0)
    nq = 40
    Q = torch.from_numpy(PA[:nq]).cuda()
    ks = rng.integers(1, 30, size=nq).astype(np.int32)
    qids = (1000 + 7 * np.arange(nq)).astype(np.int64)
    opt = dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1)
    mix = dA.adaptive_multi(Q, torch.from_numpy(ks).cuda(), int(ks.max()), torch.from_numpy(qids).cuda(), 0.01, 3,
                            storage="bf16", **opt)
    for q in range(nq):
        k = int(ks[q])
        solo = dA.adaptive(Q[q:q + 1].contiguous(), k, 0.01, 3, storage="bf16", qid_base=int(qids[q]), **opt)
        c = int(solo["count"][0])
        assert int(mix["count"][q]) == c and int(mix["evals"][q]) == int(solo["evals"][0])
        assert torch.equal(mix["idx"][q, :c], solo["idx"][0, :c])
        assert torch.all(mix["idx"][q, c:] == -1)


def test_mixed_launch_replays_in_the_oracle(two_datasets):
    """Per-query k: every query of a mixed launch follows the oracle's rounds
    for its own k and query id. The mixed row must equal the query's solo run
    with its decision log, which is replayed in the oracle (decisions,
    evaluation counts, sums)."""
    (dA, _), (PA, _), (A, _) = two_datasets
    ks = np.array([1, 5, 17, 2, 9, 30], dtype=np.int32)
    qids = np.array([5, 99, 3, 12345, 7, 8], dtype=np.int64)
    Q = PA[10:16].copy()
    Qd = torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=3e-3, B0=16, B=16, grow=0)
    r = dA.adaptive_multi(Qd, torch.from_numpy(ks).cuda(), 30, torch.from_numpy(qids).cuda(), 0.01, 1,
                          storage="f32", **opt)
    for q in range(6):
        solo = dA.adaptive(Qd[q:q + 1], int(ks[q]), 0.01, 1, storage="f32", trace=True, qid_base=int(qids[q]), **opt)
        c = int(solo["count"][0])
        assert int(r["count"][q]) == c and int(r["evals"][q]) == int(solo["evals"][0])
        assert torch.equal(r["idx"][q, :c], solo["idx"][0, :c])
        p = oracle.make_params(int(ks[q]), delta=0.01, seed=1, qid=int(qids[q]), tol=1e-5, **opt)
        code = solo["code"].cpu().numpy()
        o = oracle.adaptive(A, Q[q:q + 1], p, replay=code)
        st = o["stats"][0]
        assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (q, st)
        np.testing.assert_array_equal(o["code"][0], code[0])
        assert int(solo["evals"][0]) == st["evals"] and c == st["count"]


def _requests(pools, n, seed):
    g = np.random.default_rng(seed)
    out, qid = [], 0
    for rid in range(n):
        d = int(g.integers(0, 2))
        nq = int(g.integers(1, 40))
        k = int(g.integers(1, 25))
        rows = g.integers(0, pools[d].shape[0], size=nq)
        Q = torch.from_numpy(np.ascontiguousarray(pools[d][rows])).pin_memory()
        out.append(serve.Request(rid=rid, dataset=d, Q=Q, k=k, qid=qid))
        qid += nq
    return out


def _clone(r):
    return serve.Request(rid=r.rid, dataset=r.dataset, Q=r.Q, k=r.k, qid=r.qid)


def test_each_request_same_alone_and_in_the_mix(two_datasets):
    dss, pools, _ = two_datasets
    cfg = [serve.DatasetConfig(storage="bf16", c_alpha=1e-3), serve.DatasetConfig(storage="f32", c_alpha=1e-3)]
    reqs = _requests(pools, 24, seed=5)
    alone = {}
    for r in reqs:
        s = serve.Server(dss, cfg, slots=1)
        rr = _clone(r)
        s.submit(rr)
        s.drain()
        alone[r.rid] = rr
        assert rr.batch_size == r.Q.shape[0]
    s = serve.Server(dss, cfg, slots=3, max_batch=96)
    # all arrive at once: three take the slots, the rest wait and are packed
    # into shared launches as slots free up (independent of kernel speed)
    arrivals = [(0.0, _clone(r)) for r in reqs]
    done = s.run(arrivals)
    assert len(done) == len(reqs)
    assert any(r.batch_size > r.Q.shape[0] for r in done)       # requests really were batched together
    for r in done:
        a = alone[r.rid]
        assert torch.equal(r.idx, a.idx) and torch.equal(r.dist, a.dist), r.rid


def test_memory_budget_limits_what_is_in_flight(two_datasets):
    dss, pools, _ = two_datasets
    cfg = [serve.DatasetConfig(), serve.DatasetConfig()]
    one = dss[0].multi_workspace_size(40, 25, bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1, threads=512)
    s = serve.Server(dss, cfg, slots=4, mem_budget=int(1.5 * one), max_batch=40)
    done = s.run([(0.0, r) for r in _requests(pools, 12, seed=9)])
    assert len(done) == 12
    assert s.peak_mem <= 1.5 * one or s.launches == len(done)
    st = serve.latency_stats(done)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_shared_coordinate_serving_same_alone_and_in_the_mix(two_datasets):
    dss, pools, _ = two_datasets
    cfg = [serve.DatasetConfig(storage="bf16", c_alpha=1e-3, share=True),
           serve.DatasetConfig(storage="f32", c_alpha=1e-3, share=True)]
    reqs = _requests(pools, 16, seed=13)
    alone = {}
    for r in reqs:
        s = serve.Server(dss, cfg, slots=1, seed=4)
        rr = _clone(r)
        s.submit(rr)
        s.drain()
        alone[r.rid] = rr
    s = serve.Server(dss, cfg, slots=3, max_batch=96, seed=4)
    done = s.run([(0.0003 * i, _clone(r)) for i, r in enumerate(reqs)])
    assert any(r.batch_size > r.Q.shape[0] for r in done)
    for r in done:
        a = alone[r.rid]
        assert torch.equal(r.idx, a.idx) and torch.equal(r.dist, a.dist), r.rid


def test_exact_engine_dataset_in_the_mix(two_datasets):
    """One dataset served by the exact engine, the other by the adaptive
    rounds: every request gets the exact k nearest of its dataset (the oracle's
    brute force) for the exact one, and the same result alone and mixed."""
    dss, pools, raw = two_datasets
    cfg = [serve.DatasetConfig(method="exact"), serve.DatasetConfig(storage="f32", c_alpha=1e-3)]
    reqs = _requests(pools, 14, seed=21)
    alone = {}
    for r in reqs:
        s = serve.Server(dss, cfg, slots=1)
        rr = _clone(r)
        s.submit(rr)
        s.drain()
        alone[r.rid] = rr
    s = serve.Server(dss, cfg, slots=3, max_batch=96)
    done = s.run([(0.0004 * i, _clone(r)) for i, r in enumerate(reqs)])
    assert len(done) == len(reqs)
    for r in done:
        a = alone[r.rid]
        assert torch.equal(r.idx, a.idx) and torch.equal(r.dist, a.dist), r.rid
        if r.dataset == 0:
            oi, _ = oracle.exact_knn(raw[0], r.Q.numpy(), r.k)
            np.testing.assert_array_equal(r.idx.numpy(), oi)
