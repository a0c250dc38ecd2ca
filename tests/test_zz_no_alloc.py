"""knn_adaptive_noalloc: the entry point for callers that cannot allocate
device memory (for example inside a host framework that owns all device
memory). It must give exactly what knn_adaptive gives, call after call,
although its scratch is one fixed array that every call reuses.

Kept in a file of its own that pytest collects last."""

import ctypes as C

import numpy as np
import pytest
import torch

from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu


def _noalloc():
    L = knn.lib()
    f = L.knn_adaptive_noalloc
    P = C.c_void_p
    f.restype = C.c_int
    f.argtypes = [P, C.c_int64, C.c_int32, P, C.c_int32, C.c_int32, C.c_double, C.c_uint64, C.POINTER(knn.Opts),
                  P, P, P, P, P, P, P]
    L.knn_adaptive_noalloc_scratch_bytes.restype = C.c_size_t
    return f


def _call(f, Xd, Qd, k, delta, seed, o, trace):
    n, m = Xd.shape
    nq = Qd.shape[0]
    kh = k + (k if o.h < 0 else o.h)
    out = {"idx": torch.full((nq, kh), -7, dtype=torch.int64, device="cuda"),
           "count": torch.full((nq,), -7, dtype=torch.int32, device="cuda"),
           "evals": torch.full((nq,), -7, dtype=torch.int64, device="cuda"),
           "rounds": torch.full((nq,), -7, dtype=torch.int32, device="cuda")}
    if trace:
        out["code"] = torch.full((nq, n), -7, dtype=torch.int32, device="cuda")
        out["S"] = torch.full((nq, n), -7.0, dtype=torch.float32, device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    rc = f(ptr(Xd), n, m, ptr(Qd), nq, k, delta, seed, C.byref(o), ptr(out["idx"]), ptr(out["count"]),
           ptr(out["evals"]), ptr(out["rounds"]), ptr(out["code"]) if trace else None,
           ptr(out["S"]) if trace else None, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


@pytest.mark.parametrize("trace", [False, True])
def test_noalloc_matches_knn_adaptive_on_two_calls_in_a_row(trace):
    f = _noalloc()
    k, delta, seed = 10, 0.01, 4
    X, Q = synth.pixel_mixture(30000, 256, 40, seed=12)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=16, B=16, grow=1)
    o = knn.make_opts(k, **opt)
    ref = knn.adaptive(Xd, Qd, k, delta, seed, trace=trace, **opt)
    for call in range(2):
        rc, got = _call(f, Xd, Qd, k, delta, seed, o, trace)
        assert rc == 0, knn.lib().knn_last_error().decode()
        torch.cuda.synchronize()
        # same kernel, same draws: identical decisions, counts and candidates
        for key in ref:
            assert torch.equal(got[key], ref[key]), (call, key)


def test_noalloc_second_call_with_other_inputs_starts_fresh():
    f = _noalloc()
    X1, Q1 = synth.pixel_mixture(20000, 128, 16, seed=1)
    X2, Q2, _ = synth.gaussian_planted(25000, 96, 5, nq=16, seed=2)
    for X, Q, k in ((X1, Q1, 10), (X2, Q2, 5), (X1, Q1, 10)):
        Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
        o = knn.make_opts(k, bound="exp", c_alpha=3e-3)
        rc, got = _call(f, Xd, Qd, k, 0.01, 0, o, False)
        assert rc == 0
        ref = knn.adaptive(Xd, Qd, k, 0.01, 0, bound="exp", c_alpha=3e-3)
        torch.cuda.synchronize()
        for key in ref:
            assert torch.equal(got[key], ref[key]), key


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    f = _noalloc()
    cap = knn.lib().knn_adaptive_noalloc_scratch_bytes()
    n = cap // 24 + 1024                       # one query's lists no longer fit
    Xd = torch.zeros((n, 1), dtype=torch.float32, device="cuda")
    Qd = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    rc, _ = _call(f, Xd, Qd, 1, 0.01, 0, knn.make_opts(1), False)
    assert rc == 1
    assert "scratch" in knn.lib().knn_last_error().decode()


@pytest.mark.parametrize("threads,max_ctas", [(1024, 0), (256, 7), (512, 3)])
def test_noalloc_matches_for_each_cta_layout(threads, max_ctas):
    """Per-CTA slots of the fixed array follow the launch's grid: 1,024-thread
    CTAs with a grid the array shrinks, and grids capped by max_ctas."""
    f = _noalloc()
    k, delta, seed = 10, 0.01, 9
    X, Q = synth.pixel_mixture(60000, 200, 24, seed=5)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", c_alpha=1e-3, B0=8, B=8, grow=1, threads=threads, max_ctas=max_ctas)
    ref = knn.adaptive(Xd, Qd, k, delta, seed, **opt)
    rc, got = _call(f, Xd, Qd, k, delta, seed, knn.make_opts(k, **opt), False)
    assert rc == 0, knn.lib().knn_last_error().decode()
    torch.cuda.synchronize()
    for key in ref:
        assert torch.equal(got[key], ref[key]), key
