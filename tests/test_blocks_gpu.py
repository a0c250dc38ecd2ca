"""Block samples on the GPU (a draw picks one of ceil(m/g) blocks of g
consecutive coordinates): lock-step replay in the oracle over the FP32 data
and the stored copies, ragged rows, the round-0 pass, mixed launches and
thread counts."""

import numpy as np
import pytest
import torch

import oracle
from _parity import check, run_gpu
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def replay_ds(X, Q, res, k, storage, block, qid_base=0, delta=0.01, seed=0, **opt):
    g = {key: v.cpu().numpy() for key, v in res.items()}
    oopt = {kk: v for kk, v in opt.items() if kk in ("h", "bound", "c_alpha", "B0", "B", "grow")}
    for q in range(Q.shape[0]):
        p = oracle.make_params(k, delta=delta, seed=seed, qid=qid_base + q, tol=TOL, storage=storage, block=block,
                               **oopt)
        o = oracle.adaptive(X, Q[q:q + 1], p, replay=g["code"][q:q + 1])
        st = o["stats"][0]
        assert st["mismatch"] == 0 and st["log_inconsistent"] == 0, (storage, block, q, st)
        np.testing.assert_array_equal(o["code"][0], g["code"][q])
        assert int(g["evals"][q]) == st["evals"] and int(g["count"][q]) == st["count"], (storage, q, st)
        assert int(g["rounds"][q]) == st["rounds"]
        So, Sg = o["S"][0], g["S"][q].astype(np.float64)
        rel = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-300)
        rel[(So == 0) & (Sg == 0)] = 0
        assert rel.max() <= TOL, (storage, block, q, rel.max())


@pytest.mark.parametrize("m,g", [(784, 8), (100, 8), (77, 8), (96, 4), (64, 32), (300, 13)])
def test_fp32_blocks_replay(m, g):
    """16-byte aligned rows with full blocks (784, 8), a ragged last block on
    aligned rows (100 = 12 x 8 + 4), unaligned rows (77), blocks that are not
    32 bytes (4, 13) and wider ones (32)."""
    X, Q = synth.pixel_mixture(6000, m, 6, seed=m + g)
    summ, gpu = check(X, Q, 10, delta=0.01, seed=3, bound="exp", c_alpha=1e-3, B0=4, B=2, grow=1, block=g)
    assert summ["queries"] == 6
    assert np.all(gpu["count"] <= 20)


@pytest.mark.parametrize("B0,B,grow", [(1, 1, 0), (3, 5, 1), (40, 40, 0)])
def test_block_schedules(B0, B, grow):
    X, Q, _ = synth.gaussian_planted(3000, 256, 6, nq=3, seed=1)
    check(X, Q, 6, delta=0.05, seed=7, bound="exp", c_alpha=3e-4, B0=B0, B=B, grow=grow, block=8)


@pytest.mark.parametrize("storage,g", [("bf16", 16), ("fp8", 32), ("bf16", 8), ("fp8", 16)])
def test_copies_with_blocks_replay(storage, g):
    for m in (784, 77):
        X, Q = synth.pixel_mixture(5000, m, 4, seed=m)
        Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
        opt = dict(bound="exp", c_alpha=1e-3, B0=4, B=2, grow=1)
        with knn.Dataset(Xd, copies=(storage,)) as ds:
            res = ds.adaptive(Qd, 10, 0.01, 0, storage=storage, trace=True, block=g, **opt)
            torch.cuda.synchronize()
        replay_ds(X, Q, res, 10, storage, g, **opt)


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_round0_pass_equals_in_place_round0(storage):
    """The point-major round-0 pass of a dataset gives the same sums bit for
    bit as the round-loop kernel's own round 0 (a batch too small for it)."""
    X, Q = synth.pixel_mixture(9000, 784, 12, seed=5)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    g = {"f32": 8, "bf16": 16, "fp8": 32}[storage]
    opt = dict(bound="exp", c_alpha=1e-3, B0=6, B=4, grow=1, block=g)
    with knn.Dataset(Xd, copies=() if storage == "f32" else (storage,)) as ds:
        a = ds.adaptive(Qd, 10, 0.01, 4, storage=storage, trace=True, **opt)
        if storage == "f32":
            b = knn.adaptive(Xd, Qd, 10, 0.01, 4, trace=True, **opt)     # no round-0 pass
            for key in a:
                assert torch.equal(a[key], b[key]), key
        # B0 one block short of the exact distance (the round-0 pass draws M - 1 blocks)
        wide = dict(opt, B0=-(-784 // g) - 1)
        c = ds.adaptive(Qd, 10, 0.01, 4, storage=storage, trace=True, **wide)
    torch.cuda.synchronize()
    replay_ds(X, Q, c, 10, storage, g, seed=4, **{kk: v for kk, v in wide.items() if kk != "block"})


def test_threads_and_mixed_launch_with_blocks():
    X, Q = synth.pixel_mixture(8000, 512, 10, seed=8)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=4, B=4, grow=1, block=8)
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        base = ds.adaptive(Qd, 10, 0.01, 2, trace=True, threads=512, **opt)
        for th in (256, 1024):
            other = ds.adaptive(Qd, 10, 0.01, 2, trace=True, threads=th, **opt)
            for key in base:
                assert torch.equal(base[key], other[key]), (th, key)
        ks = np.array([1, 5, 10, 3, 7, 10, 2, 9, 4, 6], dtype=np.int32)
        qids = np.arange(10, dtype=np.int64) * 3 + 11
        mix = ds.adaptive_multi(Qd, torch.from_numpy(ks).cuda(), 10, torch.from_numpy(qids).cuda(), 0.01, 2,
                                storage="bf16", **opt)
        for q in range(10):
            solo = ds.adaptive(Qd[q:q + 1], int(ks[q]), 0.01, 2, storage="bf16", qid_base=int(qids[q]), **opt)
            c = int(solo["count"][0])
            assert int(mix["count"][q]) == c and int(mix["evals"][q]) == int(solo["evals"][0])
            assert torch.equal(mix["idx"][q, :c], solo["idx"][0, :c])


def test_lossless_bf16_copy_with_blocks_reproduces_f32():
    X, Q, _ = synth.gap_planted(5000, 64, 4, 5, [3.0, 1.5, 1.05, 2.0], seed=6, background="int255")
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=2, B=1, grow=1, block=16)
    with knn.Dataset(Xd, copies=("bf16",)) as ds:
        assert ds.error("bf16") == 0.0
        a = ds.adaptive(Qd, 5, 0.01, 0, storage="bf16", trace=True, **opt)
        b = ds.adaptive(Qd, 5, 0.01, 0, storage="f32", trace=True, **opt)
        for key in a:
            assert torch.equal(a[key], b[key]), key


def test_block_argument_checks():
    X, Q, _ = synth.gaussian_planted(300, 16, 2, nq=1, seed=1)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    with pytest.raises(knn.KnnError):
        knn.adaptive(Xd, Qd, 2, 0.01, 0, block=65)
    with pytest.raises(knn.KnnError):
        knn.adaptive(Xd, Qd, 2, 0.01, 0, block=-1)
    # a block wider than the row: one block, every draw is the whole distance
    check(X, Q, 2, bound="exp", c_alpha=1e-3, B0=1, B=1, block=40)


def test_full_size_pixel_workload_with_blocks():
    """The benchmark workload at full size with 8-coordinate blocks; three
    queries replayed."""
    import bench
    X, Q, _ = bench.make_inputs(0)
    summ, gpu = check(X, Q, 10, delta=0.01, seed=0, queries=[0, 511, 1023], bound="exp", c_alpha=1e-4,
                      B0=2, B=2, grow=1, block=8, threads=1024)
    assert summ["queries"] == 3
    assert np.all(gpu["count"] <= 20) and np.all(gpu["count"] >= 10)
