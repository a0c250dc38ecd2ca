"""Full-size workloads on the GPU, checked on sampled queries.

* Precision sweep: n = 200,000 points in d = 1,024, 4,096 queries, k = 10,
  planted neighbours at gap ratios 1.05, 1.2, 1.5, 2 and 4 over a N(0,1)
  background; rounds over the FP32 data, the BF16 copy and the FP8-e4m3 copy.
* Uneven batch: n = 1,000,000 points in d = 128 with integer values 0..255,
  16,384 queries (half at gap 3, half at gap 1.05) with k drawn from
  {1, 10, 100}, all in one persistent launch.

Each full batch runs once without a trace. For a few sampled queries the same
query then runs alone with its decision log (its Philox query id unchanged),
must give exactly the row of the full batch, and is replayed in the oracle.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
GAPS = (1.05, 1.2, 1.5, 2.0, 4.0)
OPTS = dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1, threads=1024)


def replay_one(X, q_row, g, k, storage, qid, delta=0.01, seed=0, **opt):
    """Oracle replay of one query's decision log `g` (numpy row dict)."""
    oopt = {kk: v for kk, v in opt.items() if kk in ("h", "bound", "c_alpha", "B0", "B", "grow")}
    p = oracle.make_params(k, delta=delta, seed=seed, qid=qid, tol=TOL, storage=storage, **oopt)
    o = oracle.adaptive(X, q_row[None, :], p, replay=g["code"][None, :])
    st = o["stats"][0]
    assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (storage, qid, st)
    np.testing.assert_array_equal(o["code"][0], g["code"])
    assert int(g["evals"]) == st["evals"] and int(g["count"]) == st["count"], (storage, qid, st)
    assert int(g["rounds"]) == st["rounds"]
    So, Sg = o["S"][0], g["S"].astype(np.float64)
    rel = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-300)
    rel[(So == 0) & (Sg == 0)] = 0
    assert rel.max() <= TOL, (storage, qid, rel.max())
    return st


def solo_traced(ds, Qd, q, k, qid, storage, **opt):
    r = ds.adaptive(Qd[q:q + 1], k, 0.01, 0, storage=storage, trace=True, qid_base=qid, **opt)
    torch.cuda.synchronize()
    return {key: v[0].cpu().numpy() for key, v in r.items()}


@pytest.fixture(scope="module")
def sweep_data():
    gaps = np.array([GAPS[i % len(GAPS)] for i in range(4096)])
    X, Q, planted = synth.gap_planted(200_000, 1024, 4096, 10, gaps, seed=21)
    return X, Q, planted, gaps


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_precision_sweep_full_size(sweep_data, storage):
    X, Q, planted, gaps = sweep_data
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with knn.Dataset(Xd, copies=() if storage == "f32" else (storage,)) as ds:
        full = ds.adaptive(Qd, 10, 0.01, 0, storage=storage, **OPTS)
        torch.cuda.synchronize()
        cnt = full["count"].cpu().numpy()
        assert np.all(cnt >= 10) and np.all(cnt <= 20)
        for q in (0, 1, 2, 3, 4, 4095):        # one query per gap ratio, and the last
            g = solo_traced(ds, Qd, q, 10, q, storage, **OPTS)
            for key in ("count", "evals", "rounds"):
                assert int(g[key]) == int(full[key][q]), (q, key)
            c = int(g["count"])
            assert np.array_equal(g["idx"][:c], full["idx"][q, :c].cpu().numpy())
            replay_one(X, Q[q], g, 10, storage, q, **OPTS)
        del Xd


def test_uneven_batch_full_size():
    g = np.random.Generator(np.random.PCG64(31))
    nq = 16384
    ks = g.choice(np.array([1, 10, 100]), size=nq).astype(np.int32)
    gaps = np.where(np.arange(nq) % 2 == 0, 3.0, 1.05)
    X, Q, planted = synth.gap_planted(1_000_000, 128, nq, ks, gaps, seed=32, background="int255")
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    qids = np.arange(nq, dtype=np.int64) + 7
    with knn.Dataset(Xd, copies=()) as ds:
        mix = ds.adaptive_multi(Qd, torch.from_numpy(ks).cuda(), 100, torch.from_numpy(qids).cuda(), 0.01, 0,
                                storage="f32", **OPTS)
        torch.cuda.synchronize()
        cnt = mix["count"].cpu().numpy()
        assert np.all(cnt >= ks) and np.all(cnt <= 2 * ks)
        picks = []
        for kk in (1, 10, 100):
            for par in (0, 1):
                picks.append(int(np.flatnonzero((ks == kk) & (np.arange(nq) % 2 == par))[0]))
        picks.append(nq - 1)
        for q in picks:
            k = int(ks[q])
            s = solo_traced(ds, Qd, q, k, int(qids[q]), "f32", **OPTS)
            for key in ("count", "evals", "rounds"):
                assert int(s[key]) == int(mix[key][q]), (q, key)
            c = int(s["count"])
            assert np.array_equal(s["idx"][:c], mix["idx"][q, :c].cpu().numpy())
            assert np.all(mix["idx"][q, c:].cpu().numpy() == -1)
            replay_one(X, Q[q], s, k, "f32", int(qids[q]), **OPTS)
