"""Exact method with the tcgen05 tensor-core screens (FP16 scaled, single
BF16, BF16 hi/lo split of the centred data; FP32 accumulation in tensor
memory; selection fused into the GEMM's epilogue) against the oracle's brute
force: the proven margin plus the FP32/FP64 ranking must give the exact k
nearest. Also the candidate-list overflow (full scan) and a bounded wait
that runs out (failure detection without a GPU fault)."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

SCREENS = ("f16", "bf16", "bf16x3")
COPIES = ("screen", "screen_f16", "screen_bf16")
STATUS_TIMEOUT = 0x5C7C


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,m,nq,k", [(1000, 64, 5, 1), (3001, 100, 130, 10), (777, 3, 9, 7),
                                      (5000, 257, 300, 100), (20000, 784, 513, 10), (40000, 128, 1030, 1)])
def test_tc_exact_matches_bruteforce(n, m, nq, k):
    X, Q = synth.pixel_mixture(n, m, nq, seed=n)
    Xd, Qd = _cuda(X), _cuda(Q)
    oi, od = oracle.exact_knn(X, Q, k)
    with knn.Dataset(Xd, copies=COPIES) as ds:
        for screen in SCREENS + ("f32",):
            gi, gd = ds.exact(Qd, k, screen=screen)
            torch.cuda.synchronize()
            assert knn.device_status() == 0
            np.testing.assert_array_equal(gi.cpu().numpy(), oi, err_msg=screen)
            np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=1e-12, err_msg=screen)


def test_tc_exact_gaussian_and_integer_data():
    for X, Q in (synth.gap_planted(9000, 128, 40, 10, 1.05, seed=2, background="int255")[:2],
                 synth.gaussian_planted(4000, 300, 5, nq=70, seed=3)[:2]):
        k = 10 if X.shape[1] == 128 else 5
        oi, od = oracle.exact_knn(X, Q, k)
        with knn.Dataset(_cuda(X), copies=COPIES) as ds:
            for screen in SCREENS:
                gi, gd = ds.exact(_cuda(Q), k, screen=screen)
                np.testing.assert_array_equal(gi.cpu().numpy(), oi, err_msg=screen)
    assert knn.device_status() == 0


def test_clustered_data_far_from_the_origin():
    """Tight clusters far from the centre: the screens' bounds scale with the
    norms, so their windows hold most of a cluster; the candidate lists or
    the full scan must still return the exact k nearest."""
    g = np.random.default_rng(5)
    m, n, nq = 192, 24000, 12
    C = g.normal(0.0, 30.0, size=(3, m))
    X = (C[g.integers(0, 3, size=n)] + 0.05 * g.standard_normal((n, m))).astype(np.float32)
    Q = (C[g.integers(0, 3, size=nq)] + 0.05 * g.standard_normal((nq, m))).astype(np.float32)
    oi, od = oracle.exact_knn(X, Q, 10)
    with knn.Dataset(_cuda(X), copies=COPIES) as ds:
        for screen in SCREENS + ("f32",):
            gi, gd = ds.exact(_cuda(Q), 10, screen=screen)
            np.testing.assert_array_equal(gi.cpu().numpy(), oi, err_msg=screen)
            np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=1e-12)
    assert knn.device_status() == 0


def test_duplicates_overflow_the_candidate_list():
    """Every point at the same distance: every pair passes the cut, the list
    overflows and the query is ranked over every point; among equal
    distances the smallest indices win."""
    g = np.random.default_rng(8)
    row = g.random(96).astype(np.float32)
    X = np.repeat(row[None, :], 6000, axis=0)
    X[::7] += 0.25          # a farther group
    Q = np.stack([row + 0.01, row - 0.02]).astype(np.float32)
    oi, od = oracle.exact_knn(X, Q, 16)
    with knn.Dataset(_cuda(X), copies=COPIES) as ds:
        for screen in SCREENS:
            gi, gd = ds.exact(_cuda(Q), 16, screen=screen)
            np.testing.assert_array_equal(gi.cpu().numpy(), oi, err_msg=screen)
    assert knn.device_status() == 0


def test_bounded_wait_runs_out_and_the_next_call_is_correct():
    """With a wait limit of 0 every pipeline wait of the tensor-core kernel
    gives up before any copy or MMA is issued: the call records the timeout
    code in the status word (read and cleared by knn_device_status) and the
    device stays usable -- the next call, at the default limit, is exact."""
    X, Q = synth.pixel_mixture(5000, 128, 40, seed=4)
    oi, _ = oracle.exact_knn(X, Q, 10)
    with knn.Dataset(_cuda(X), copies=("screen_f16",)) as ds:
        try:
            knn.debug_wait_limit(0)
            ds.exact(_cuda(Q), 10, screen="f16")
            torch.cuda.synchronize()
        finally:
            knn.debug_wait_limit(-1)
        assert knn.device_status() == STATUS_TIMEOUT
        assert knn.device_status() == 0          # read once, cleared
        gi, _ = ds.exact(_cuda(Q), 10, screen="f16")
        torch.cuda.synchronize()
        assert knn.device_status() == 0
        np.testing.assert_array_equal(gi.cpu().numpy(), oi)
