"""Batched execution: CUDA-graph replay of the adaptive step, the thread-count
variant of the round-loop kernel, and the autotuner."""

import json
import os

import numpy as np
import pytest
import torch

from paper_1902_09465_gb300 import knn, runtime, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    X, Q = synth.pixel_mixture(30000, 256, 160, seed=21)
    Xd = torch.from_numpy(X).cuda()
    ds = knn.Dataset(Xd, copies=("bf16",))
    yield ds, torch.from_numpy(Q).cuda()
    ds.close()


def test_thread_counts_give_identical_results(data):
    ds, Qd = data
    a = ds.adaptive(Qd, 10, 0.01, 3, bound="exp", c_alpha=1e-3, grow=1, threads=512, trace=True)
    for th in (256, 1024):
        b = ds.adaptive(Qd, 10, 0.01, 3, bound="exp", c_alpha=1e-3, grow=1, threads=th, trace=True)
        for key in a:
            assert torch.equal(a[key], b[key]), (th, key)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_graph_replay_matches_eager(data, storage):
    ds, Qd = data
    step = runtime.GraphStep(ds, 64, 10, 0.01, 5, storage=storage, bound="exp", c_alpha=1e-3, grow=1)
    for part in (Qd[:64], Qd[64:128], Qd[:64]):
        res, ri, rd = step.run(part)
        torch.cuda.synchronize()
        e = ds.adaptive(part.contiguous(), 10, 0.01, 5, storage=storage, bound="exp", c_alpha=1e-3, grow=1)
        ei, ed = knn.rerank(ds.X, part.contiguous(), e["idx"], 10)
        for key in ("idx", "count", "evals", "rounds"):
            assert torch.equal(res[key], e[key]), key
        assert torch.equal(ri, ei) and torch.equal(rd, ed)


def test_autotune_picks_a_configuration_meeting_the_target(data, tmp_path):
    ds, Qd = data
    cache = str(tmp_path / "tune.json")
    H = Qd[96:160].contiguous()
    out = runtime.autotune(ds, H, 10, 0.01, schedules=((16, 16, 1), (8, 8, 0)), threads=(512, 256),
                           c_grid=(1e-2, 1e-3, 1e-4), cache=cache)
    best = out["best"]
    assert best in out["table"] and best["queries_per_s"] == max(r["queries_per_s"] for r in out["table"])
    res = ds.adaptive(H, 10, 0.01, 0, bound="exp", c_alpha=best["c_alpha"], B0=best["B0"], B=best["B"],
                      grow=best["grow"], threads=best["threads"], qid_base=1 << 41)
    ri, rd = knn.rerank(ds.X, H, res["idx"], 10)
    ti, td = ds.exact(H, 10, screen="f32")
    assert runtime.recall(ri, rd, ti, td) >= 0.999
    with open(cache) as f:
        assert out["key"] in json.load(f)
    assert out["key"].startswith(runtime.tune_key(ds, 10, "f32")) and "target=0.999+" in out["key"]
    again = runtime.autotune(ds, H, 10, 0.01, cache=cache)   # served from the cache
    assert again == out


def test_autotune_over_sampling_units(data, tmp_path):
    """Single coordinates and 8-coordinate blocks in one search: the choice
    meets the recall target and names its sampling unit."""
    ds, Qd = data
    H = Qd[96:160].contiguous()
    out = runtime.autotune(ds, H, 10, 0.01, schedules=((8, 8, 1),), threads=(512,), blocks=(1, 8),
                           block_schedules=((2, 2, 1),), c_grid=(1e-2, 1e-3, 1e-4), use_cache=False,
                           cache=str(tmp_path / "t.json"))
    assert {r.get("block", 1) for r in out["table"]} <= {1, 8} and len(out["table"]) >= 1
    best = out["best"]
    res = ds.adaptive(H, 10, 0.01, 0, bound="exp", c_alpha=best["c_alpha"], B0=best["B0"], B=best["B"],
                      grow=best["grow"], threads=best["threads"], block=best.get("block", 1), qid_base=1 << 41)
    ri, rd = knn.rerank(ds.X, H, res["idx"], 10)
    ti, td = ds.exact(H, 10, screen="f32")
    assert runtime.recall(ri, rd, ti, td) >= 0.999


@pytest.mark.parametrize("share", [False, True])
def test_query_locality_order_changes_only_the_schedule(share):
    """Dataset calls take a batch's queries in a locality order (SimHash of
    the query); every output, the decision log included, equals the batch
    order's bit for bit."""
    X, Q = synth.pixel_mixture(30000, 160, 300, seed=17)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=16, B=16, grow=1, threads=512)
    if share:
        opt.update(share_points=True, share_queries=True)
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        if share:
            ds.share(3, copies=("bf16",))
        a = ds.adaptive(Qd, 10, 0.01, 3, storage="bf16", trace=True, query_order=True, **opt)
        b = ds.adaptive(Qd, 10, 0.01, 3, storage="bf16", trace=True, query_order=False, **opt)
        torch.cuda.synchronize()
    for key in a:
        assert torch.equal(a[key], b[key]), key
