"""Lock-step parity between the CUDA path (through the C ABI) and the CPU
oracle: the oracle replays the GPU's decision log round by round; every
decision must match except those whose bound lies within 1e-5 (relative to
the magnitudes involved) of its threshold, which are flagged and counted."""

import numpy as np
import torch

import oracle
from paper_1902_09465_gb300 import knn

TOL_DECISION = 1e-5   # near-threshold band of the replay
TOL_ESTIMATE = 1e-5   # FP32 sums vs FP64 sums on the same samples


def run_gpu(X, Q, k, delta, seed, **opts):
    """knn.adaptive with the decision log; numpy arrays out."""
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    res = knn.adaptive(Xd, Qd, k, delta, seed, trace=True, **opts)
    torch.cuda.synchronize()
    return {key: v.cpu().numpy() for key, v in res.items()}


def check(X, Q, k, delta=0.01, seed=0, queries=None, h=None, bound="footnote", c_alpha=1.0, B0=16, B=16, grow=0,
          qid_base=0, share_points=False, share_queries=False, gpu=None, block=1, threads=0, replace=True):
    """Runs the GPU (unless `gpu` holds a previous result) and replays the
    chosen queries in the oracle. Returns a summary dict."""
    if gpu is None:
        gpu = run_gpu(X, Q, k, delta, seed, h=h, bound=bound, c_alpha=c_alpha, B0=B0, B=B, grow=grow,
                      qid_base=qid_base, share_points=share_points, share_queries=share_queries, block=block,
                      threads=threads, replace=replace)
    nq, n = Q.shape[0], X.shape[0]
    hh = k if h is None else h
    kh = k + hh
    queries = range(nq) if queries is None else queries
    summ = {"near": 0, "near_disagree": 0, "max_rel_S": 0.0, "queries": 0}
    for q in queries:
        p = oracle.make_params(k, h=hh, delta=delta, bound=bound, c_alpha=c_alpha, B0=B0, B=B, grow=grow, seed=seed,
                               qid=qid_base + q, share_points=share_points, share_queries=share_queries,
                               tol=TOL_DECISION, block=block, replace=replace)
        o = oracle.adaptive(X, Q[q:q + 1], p, replay=gpu["code"][q:q + 1])
        st = o["stats"][0]
        assert st["mismatch"] == 0, (q, st)
        assert st["log_inconsistent"] == 0, (q, st)
        np.testing.assert_array_equal(o["code"][0], gpu["code"][q])
        assert int(gpu["evals"][q]) == st["evals"], (q, int(gpu["evals"][q]), st)
        assert int(gpu["rounds"][q]) == st["rounds"], (q, int(gpu["rounds"][q]), st)
        assert int(gpu["count"][q]) == st["count"], (q, int(gpu["count"][q]), st)
        So = o["S"][0]
        Sg = gpu["S"][q].astype(np.float64)
        rel = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-300)
        rel[(So == 0) & (Sg == 0)] = 0.0
        assert rel.max() <= TOL_ESTIMATE, (q, rel.max(), int(rel.argmax()))
        c = st["count"]
        g_set = set(gpu["idx"][q][:c].tolist())
        o_set = set(o["idx"][0][:c].tolist())
        assert np.all(gpu["idx"][q][c:] == -1)
        kind = o["code"][0] & 3
        live = np.flatnonzero(kind != oracle.ELIMINATED)
        assert g_set <= set(live.tolist())
        if len(live) <= kh:
            assert g_set == o_set == set(live.tolist())
        elif g_set != o_set:
            # truncation by estimate: any difference must be a near-tie
            dh = So / (np.maximum(o["T"][0], 1) * max(block, 1))
            bound_v = max(dh[list(o_set)])
            for i in g_set ^ o_set:
                assert abs(dh[i] - bound_v) <= 1e-5 * max(abs(bound_v), 1e-300), (q, i)
        summ["near"] += st["near"]
        summ["near_disagree"] += st["near_disagree"]
        summ["max_rel_S"] = max(summ["max_rel_S"], float(rel.max()))
        summ["queries"] += 1
    return summ, gpu


def replay_row(X, q_row, g, k, qid, storage="f32", delta=0.01, seed=0, **opt):
    """Oracle replay of one query's decision log; `g` holds that query's
    numpy rows (code, S, evals, count, rounds) from a traced GPU call.
    Returns the oracle's stats and the largest relative error of S."""
    oopt = {kk: v for kk, v in opt.items() if kk in ("h", "bound", "c_alpha", "B0", "B", "grow")}
    p = oracle.make_params(k, delta=delta, seed=seed, qid=qid, tol=TOL_DECISION, storage=storage, **oopt)
    o = oracle.adaptive(X, q_row[None, :], p, replay=g["code"][None, :])
    st = o["stats"][0]
    assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (qid, st)
    np.testing.assert_array_equal(o["code"][0], g["code"])
    assert int(g["evals"]) == st["evals"] and int(g["count"]) == st["count"], (qid, st)
    assert int(g["rounds"]) == st["rounds"], (qid, st)
    So, Sg = o["S"][0], g["S"].astype(np.float64)
    rel = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-300)
    rel[(So == 0) & (Sg == 0)] = 0
    assert rel.max() <= TOL_ESTIMATE, (qid, rel.max())
    return st, float(rel.max()), o
