"""Cost of the batched rounds against Algorithm 1 as printed (the seven-heap
version), both on the CPU oracle: the fraction of the naive method's
coordinate evaluations (n m) each spends, and whether the k nearest are
returned, on the same seeded inputs and the same bound (Section 5's form).

    python oracle/sequential_cost.py

Test infrastructure like the rest of this folder: it runs the oracle only
(inputs from the seeded generators) and prints the table; nothing imports it."""

import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1902_09465_gb300 import synth  # noqa: E402


def run(name, gen, k, h, delta, c_alpha, trials, schedules):
    rows = {"sequential": [], **{f"batched B0={b0} B={b} grow={g}": [] for b0, b, g in schedules}}
    hits = {key: 0 for key in rows}
    for t in range(trials):
        X, Q = gen(t)
        n, m = X.shape
        ti, _ = oracle.exact_knn(X, Q[:1], k)
        true = set(ti[0].tolist())
        p = oracle.make_params(k, h=h, delta=delta, bound="exp", c_alpha=c_alpha, seed=t)
        idx, ev, _ = oracle.sequential(X, Q[0], p, heaps=True)
        rows["sequential"].append(ev / (n * m))
        hits["sequential"] += true <= set(idx.tolist())
        for b0, b, g in schedules:
            pb = oracle.make_params(k, h=h, delta=delta, bound="exp", c_alpha=c_alpha, seed=t, B0=b0, B=b, grow=g)
            r = oracle.adaptive(X, Q[:1], pb, want_state=False)
            st = r["stats"][0]
            key = f"batched B0={b0} B={b} grow={g}"
            rows[key].append(st["evals"] / (n * m))
            hits[key] += true <= set(r["idx"][0][: st["count"]].tolist())
    print(f"{name} (k = {k}, h = {h}, delta = {delta}, C_alpha = {c_alpha}, {trials} trials)")
    for key, v in rows.items():
        print(f"  {key:28s} evaluations / (n m): median {np.median(v):.4f}  "
              f"[{np.percentile(v, 25):.4f}, {np.percentile(v, 75):.4f}]   k nearest returned {hits[key]}/{trials}")


if __name__ == "__main__":
    sched = ((1, 1, 0), (8, 8, 1), (16, 16, 1))
    run("gaussian planted, n = 2,000, m = 256", lambda t: synth.gaussian_planted(2000, 256, 5, seed=t)[:2],
        5, 5, 0.01, 1e-3, 10, sched)
    run("subspace p = 10, n = 1,000, m = 12,288", lambda t: synth.subspace(1000, 12288, 10, nq=1, seed=t),
        10, 10, 0.001, 1e-3, 5, sched)
    run("subspace p = 100, n = 1,000, m = 12,288", lambda t: synth.subspace(1000, 12288, 100, nq=1, seed=t),
        10, 10, 0.001, 1e-4, 5, sched)
