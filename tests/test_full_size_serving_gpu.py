"""The serving workload at full size: the four resident BF16 datasets
(100,000 x 3,072, 500,000 x 768, 2,000,000 x 128, 1,000,000 x 64; Gaussian
mixtures with planted neighbours), requests of 1-64 queries with k in
[1, 100] served by the continuous-batching loop with each dataset on the
engine the benchmark routes it to. Sampled rows of every request are checked
against the oracle's brute force; two requests are also served alone and
must come out the same as in the mix."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, serve, synth

pytestmark = pytest.mark.gpu

SIZES = [(100_000, 3072), (500_000, 768), (2_000_000, 128), (1_000_000, 64)]


def test_full_size_serving_sampled_rows():
    raw, dss, pools, cfgs = [], [], [], []
    for i, (n, m) in enumerate(SIZES):
        X, P = synth.mixture_planted(n, m, 256, seed=100 + i)
        ds = knn.Dataset(torch.from_numpy(X).cuda(), copies=("bf16", "screen"))
        if i == 0:
            ds.share(0, copies=("bf16",))
            ds._shared_seed, ds._shared = 0, ("bf16",)
            cfgs.append(serve.DatasetConfig(storage="bf16", c_alpha=1e-4, B0=16, B=16, grow=1, threads=1024,
                                            share=True))
        else:
            cfgs.append(serve.DatasetConfig(method="exact"))
        raw.append(X)
        dss.append(ds)
        pools.append(P)
    try:
        g = np.random.default_rng(7)
        reqs, qid = [], 0
        for rid in range(16):
            d = rid % 4
            nq = int(g.integers(1, 65))
            rows = g.integers(0, 256, size=nq)
            Q = torch.from_numpy(np.ascontiguousarray(pools[d][rows])).pin_memory()
            reqs.append(serve.Request(rid=rid, dataset=d, Q=Q, k=int(g.integers(1, 101)), qid=qid))
            qid += nq
        srv = serve.Server(dss, cfgs, slots=4, max_batch=256)
        done = srv.run([(0.0005 * i, r) for i, r in enumerate(reqs)], timeout_s=600)
        assert len(done) == 16
        hit = tot = 0
        for r in done:
            X = raw[r.dataset]
            pick = sorted(set([0, r.Q.shape[0] - 1, r.Q.shape[0] // 2]))
            ti, td = oracle.exact_knn(X, r.Q.numpy()[pick], r.k)
            got = r.idx.numpy()[pick]
            if cfgs[r.dataset].method == "exact":
                np.testing.assert_array_equal(got, ti)
            else:
                for a, b in zip(got, ti):
                    hit += len(set(a.tolist()) & set(b.tolist()))
                    tot += len(b)
        if tot:
            assert hit / tot >= 0.99, hit / tot
        # two requests alone: the same result as in the mix
        for r in done[:2]:
            s = serve.Server(dss, cfgs, slots=1)
            rr = serve.Request(rid=r.rid, dataset=r.dataset, Q=r.Q, k=r.k, qid=r.qid)
            s.submit(rr)
            s.drain()
            assert torch.equal(rr.idx, r.idx) and torch.equal(rr.dist, r.dist)
    finally:
        for ds in dss:
            ds.close()
