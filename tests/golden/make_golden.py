"""Writes the golden fixtures of this folder from the CPU oracle (and the
seeded input generators); nothing else produces them.

    python tests/golden/make_golden.py

Each fixture records the inputs' recipe and the oracle's results, so a later
change to the oracle or to the GPU path that alters them is caught."""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1902_09465_gb300 import synth  # noqa: E402

CASES = [("footnote", 1.0, 16, 16, 0), ("lemma", 1.0, 16, 16, 0), ("exp", 1e-3, 16, 16, 0), ("exp", 1e-4, 8, 8, 1)]


def single_query():
    X, Q, planted = synth.gaussian_planted(2000, 256, 5, seed=0)
    ti, td = oracle.exact_knn(X, Q, 5)
    runs = []
    for bound, c, B0, B, grow in CASES:
        p = oracle.make_params(5, delta=0.01, bound=bound, c_alpha=c, B0=B0, B=B, grow=grow, seed=0)
        r = oracle.adaptive(X, Q, p)
        st = r["stats"][0]
        runs.append({"bound": bound, "c_alpha": c, "B0": B0, "B": B, "grow": grow,
                     "idx": [int(v) for v in r["idx"][0]], "count": st["count"], "evals": st["evals"],
                     "rounds": st["rounds"], "term": st["term"]})
    return {
        "citation": "Section 3 problem statement and Section 4 sampled estimator, run by the batched rules of "
                    "Algorithm 1 (R0-R5); brute force of Section 3 for the exact neighbours",
        "inputs": "paper_1902_09465_gb300.synth.gaussian_planted(2000, 256, 5, seed=0): n = 2,000 points in "
                  "m = 256, N(0,1) coordinates, 5 planted rows at query + N(0, 0.1^2); k = h = 5, delta = 0.01, "
                  "Philox seed 0, query id 0",
        "planted": [int(v) for v in planted[0]],
        "exact_idx": [int(v) for v in ti[0]],
        "exact_dist": [float(v) for v in td[0]],
        "runs": runs,
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "single_query_gaussian_n2000_m256_k5.json"), "w") as f:
        json.dump(single_query(), f, indent=1)
        f.write("\n")
    print("written")
