"""Exact method with the tcgen05 tensor-core screen (BF16 hi/lo split of the
centred data, FP32 accumulation in tensor memory) against the oracle's brute
force: the proven margin plus the FP64 rerank must give the exact k nearest."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,m,nq,k", [(1000, 64, 5, 1), (3001, 100, 130, 10), (777, 3, 9, 7),
                                      (5000, 257, 300, 100), (20000, 784, 513, 10)])
def test_tc_exact_matches_bruteforce(n, m, nq, k):
    X, Q = synth.pixel_mixture(n, m, nq, seed=n)
    Xd, Qd = _cuda(X), _cuda(Q)
    with knn.Dataset(Xd, copies=("screen",)) as ds:
        gi, gd = ds.exact(Qd, k, screen="bf16x3")
        fi, fd = ds.exact(Qd, k, screen="f32")
    torch.cuda.synchronize()
    assert knn.device_status() == 0
    oi, od = oracle.exact_knn(X, Q, k)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=1e-12)
    np.testing.assert_array_equal(fi.cpu().numpy(), oi)


def test_tc_exact_gaussian_and_integer_data():
    for X, Q in (synth.gap_planted(9000, 128, 40, 10, 1.05, seed=2, background="int255")[:2],
                 synth.gaussian_planted(4000, 300, 5, nq=70, seed=3)[:2]):
        with knn.Dataset(_cuda(X), copies=("screen",)) as ds:
            gi, gd = ds.exact(_cuda(Q), 10 if X.shape[1] == 128 else 5)
        oi, od = oracle.exact_knn(X, Q, gi.shape[1])
        np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    assert knn.device_status() == 0


def test_clustered_data_far_from_the_origin_takes_the_second_screen():
    """Tight clusters far from the centre: the screen's bound scales with the
    norms, so its window holds most of a cluster (more than the candidate
    list); the direct FP32 second screen must still return the exact k
    nearest (SIMT and tensor-core screens)."""
    g = np.random.default_rng(5)
    m, n, nq = 192, 24000, 12
    C = g.normal(0.0, 30.0, size=(3, m))
    X = (C[g.integers(0, 3, size=n)] + 0.05 * g.standard_normal((n, m))).astype(np.float32)
    Q = (C[g.integers(0, 3, size=nq)] + 0.05 * g.standard_normal((nq, m))).astype(np.float32)
    oi, od = oracle.exact_knn(X, Q, 10)
    with knn.Dataset(_cuda(X), copies=("screen",)) as ds:
        for screen in ("bf16x3", "f32"):
            gi, gd = ds.exact(_cuda(Q), 10, screen=screen)
            np.testing.assert_array_equal(gi.cpu().numpy(), oi)
            np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=1e-12)
    assert knn.device_status() == 0
