"""Batched execution helpers around the C ABI: CUDA-graph replay of a whole
adaptive step, and the autotuner that picks the round schedule, the threads
per query and C_alpha for a dataset.

Everything here is host orchestration: the work itself runs in the library's
kernels (knn_adaptive_ds, knn_rerank); torch supplies device memory, streams
and graph capture.
"""

from __future__ import annotations

import json
import math
import os
import time

import torch

from . import knn


class GraphStep:
    """One adaptive step over a resident dataset for a fixed batch size:
    the rounds (knn_adaptive_ds) and the FP64 rerank (knn_rerank), captured
    once into a CUDA graph and replayed. The static input is copied in, the
    static outputs are returned (they are overwritten by the next run)."""

    def __init__(self, ds: knn.Dataset, nq: int, k: int, delta: float = 0.01, seed: int = 0, storage: str = "f32",
                 rerank: bool = True, **opts):
        dev = ds.X.device
        self.ds, self.nq, self.k = ds, nq, k
        self.kw = dict(delta=delta, seed=seed, storage=storage, **opts)
        o = knn.make_opts(k, **{kk: v for kk, v in opts.items() if kk != "trace"})
        self.Q = torch.zeros((nq, ds.m), dtype=torch.float32, device=dev)
        self.ws = torch.empty(knn.adaptive_workspace_size(ds.n, ds.m, nq, k, o), dtype=torch.uint8, device=dev)
        h = k if o.h < 0 else o.h
        self.out = knn._alloc_out(nq, ds.n, k + h, dev, False)
        self.rerank = rerank
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):  # warm-up outside the capture
            self._body()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.result = self._body()

    def _body(self):
        kw = dict(self.kw)
        delta, seed = kw.pop("delta"), kw.pop("seed")
        res = self.ds.adaptive(self.Q, self.k, delta, seed, workspace=self.ws, out=self.out, **kw)
        if self.rerank:
            ri, rd = knn.rerank(self.ds.X, self.Q, res["idx"], self.k)
            return res, ri, rd
        return res, None, None

    def run(self, Q: torch.Tensor):
        """Copies Q (nq x m, on the device or pinned host) in and replays."""
        self.Q.copy_(Q, non_blocking=True)
        self.graph.replay()
        return self.result


def recall(got_idx, got_dist, true_idx, true_dist, rel: float = 1e-6) -> float:
    """Fraction of the true k nearest returned; a returned point whose exact
    distance ties the k-th true distance within `rel` also counts."""
    gi, gd = got_idx.cpu(), got_dist.cpu()
    ti, td = true_idx.cpu(), true_dist.cpu()
    hit = 0
    for q in range(ti.shape[0]):
        kth = float(td[q, -1])
        ts = set(ti[q].tolist())
        for i, d in zip(gi[q].tolist(), gd[q].tolist()):
            if i in ts or (i >= 0 and abs(d - kth) <= rel * max(abs(kth), 1e-300)):
                hit += 1
    return min(1.0, hit / ti.numel())


# B past any row length: the round after round 0 is the exact distance (the
# exact cap at T + B >= m), so the points round 0 keeps are computed in full
EXACT_NEXT = 1 << 20
DEFAULT_SCHEDULES = ((16, 16, 1), (8, 8, 1), (32, 32, 1), (16, 16, 0), (16, EXACT_NEXT, 0), (32, EXACT_NEXT, 0))
BLOCK_SCHEDULES = ((2, 2, 1), (4, 4, 1), (8, 8, 1))  # in blocks of coordinates
DEFAULT_C_GRID = (1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 3e-5)


def _cache_path(path):
    if path:
        return path
    return os.environ.get("KNN_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "knn_gb300",
                                                           "tune.json"))


def tune_key(ds: knn.Dataset, k: int, storage: str) -> str:
    return f"m={ds.m}|n~2^{round(math.log2(ds.n))}|{storage}|k={k}"


def autotune(ds: knn.Dataset, H: torch.Tensor, k: int, delta: float = 0.01, storage: str = "f32",
             target: float = 0.999, margin: float = 0.0005, schedules=DEFAULT_SCHEDULES, threads=(512, 1024),
             c_grid=DEFAULT_C_GRID, reps: int = 3, cache: str | None = None, use_cache: bool = True,
             seed: int = 0, extra=None, blocks=(1,), block_schedules=BLOCK_SCHEDULES):
    """Picks (block, B0, B, grow, threads, C_alpha) for a dataset: for every
    sampling unit in `blocks` (1: single coordinates, g > 1: blocks of g
    coordinates, tried with `block_schedules`), schedule and thread count,
    the smallest C_alpha of the grid whose recall on the held-out queries H
    (after the FP64 rerank) is at least target + margin, then the fastest of
    those. Returns a dict with the choice and the whole table, and stores it
    in the JSON cache under a key of (d, n bucket, storage, k, delta, the
    recall target and margin, options).
    `extra` adds options to every call (for example the shared-coordinate
    masks); `seed` is the Philox seed used."""
    path = _cache_path(cache)
    extra = dict(extra or {})
    blocks = tuple(int(g) for g in blocks)
    key = tune_key(ds, k, storage) + f"|delta={delta:g}|target={target:g}+{margin:g}"
    key += ("|" + ",".join(f"{a}={b}" for a, b in sorted(extra.items())) if extra else "")
    if blocks != (1,):
        key += "|blocks=" + ",".join(str(g) for g in blocks)
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                got = json.load(f).get(key)
            if got:
                return got
        except (OSError, ValueError):
            pass
    ti, td = ds.exact(H, k, screen="f32")
    table = []
    plan = [(g, sch) for g in blocks for sch in (schedules if g <= 1 else block_schedules)]
    for g, (B0, B, grow) in plan:
        for th in threads:
            opts = dict(bound="exp", B0=B0, B=B, grow=grow, threads=th, qid_base=1 << 41, **extra)
            if g > 1:
                opts["block"] = g
            chosen = None
            for c in c_grid:
                res = ds.adaptive(H, k, delta, seed, storage=storage, c_alpha=c, **opts)
                ri, rd = knn.rerank(ds.X, H, res["idx"], k)
                if recall(ri, rd, ti, td) >= target + margin:
                    chosen = c
                else:
                    break
            if chosen is None:
                continue
            res = ds.adaptive(H, k, delta, seed, storage=storage, c_alpha=chosen, **opts)  # untimed warm-up
            knn.rerank(ds.X, H, res["idx"], k)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                res = ds.adaptive(H, k, delta, seed, storage=storage, c_alpha=chosen, **opts)
                knn.rerank(ds.X, H, res["idx"], k)
            torch.cuda.synchronize()
            qps = reps * H.shape[0] / (time.perf_counter() - t0)
            row = {"B0": B0, "B": B, "grow": grow, "threads": th, "c_alpha": chosen, "queries_per_s": round(qps, 1)}
            if g > 1:
                row["block"] = g
            table.append(row)
    if not table:
        raise knn.KnnError("autotune: no configuration reached the target recall")
    best = max(table, key=lambda r: r["queries_per_s"])
    out = {"key": key, "best": best, "table": table, "target": target}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        data = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
        data[key] = out
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, path)
    except (OSError, ValueError):
        pass
    return out
