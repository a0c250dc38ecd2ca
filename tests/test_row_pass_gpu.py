"""Row passes (knn_opts.row_pass): from a round whose active points nearly
all survived the round before, or that draws at least m/8 coordinates per
point, one read of each active point's row forms the sums of that round and
of up to five later ones, each in the order of its own round's gather. The
results must be the same bit for bit as with every round gathering its own
draws: indices, counts, evaluations, rounds, decision codes and every logged
sum -- whatever rounds the passes cover."""

import pytest
import torch

from paper_1902_09465_gb300 import knn, synth

pytestmark = pytest.mark.gpu

# n, m, nq, k, schedule and bound options
CASES = [
    (20000, 784, 24, 10, dict(B0=16, B=16, grow=1, c_alpha=3e-4)),  # doubling up to the exact round
    (20000, 256, 24, 10, dict(B0=16, B=64, grow=0, c_alpha=1e-3)),  # 8 B >= m: passes from round 1
    (12000, 77, 16, 5, dict(B0=12, B=8, grow=0, c_alpha=1e-3)),  # rows not 16-byte multiples; T off blocks
    (12000, 200, 16, 5, dict(B0=8, B=8, grow=0, c_alpha=1e-2)),  # many rounds: passes of 6 in turn
    (16000, 512, 16, 8, dict(B0=16, B=16, grow=1, c_alpha=1e-3, metric="l1")),
    (16000, 640, 16, 8, dict(B0=40, B=300, grow=0, c_alpha=1e-3)),  # 38 blocks: two per virtual lane
]


def _same(a, b, tag):
    for key in a:
        assert torch.equal(a[key], b[key]), (tag, key)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_row_passes_match_round_by_round_gathers(case):
    n, m, nq, k, opt = CASES[case]
    X, Q = synth.pixel_mixture(n, m, nq, seed=case)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", **opt)
    with knn.Dataset(Xd) as ds:
        a = ds.adaptive(Qd, k, 0.01, 7, trace=True, row_pass=True, **opt)
        b = ds.adaptive(Qd, k, 0.01, 7, trace=True, row_pass=False, **opt)
        torch.cuda.synchronize()
        _same(a, b, ("dataset", case))
        # mixed batch: per-query k and ids
        ks = torch.tensor([k if i % 2 else max(1, k // 2) for i in range(nq)], dtype=torch.int32, device="cuda")
        qids = torch.arange(100, 100 + nq, dtype=torch.int64, device="cuda")
        ma = ds.adaptive_multi(Qd, ks, k, qids, 0.01, 7, row_pass=True, **opt)
        mb = ds.adaptive_multi(Qd, ks, k, qids, 0.01, 7, row_pass=False, **opt)
        torch.cuda.synchronize()
        _same(ma, mb, ("multi", case))
    # the standalone entry point (round 0 in the round loop or point-major)
    sa = knn.adaptive(Xd, Qd, k, 0.01, 7, trace=True, row_pass=True, **opt)
    sb = knn.adaptive(Xd, Qd, k, 0.01, 7, trace=True, row_pass=False, **opt)
    torch.cuda.synchronize()
    _same(sa, sb, ("standalone", case))
    assert knn.device_status() == 0


def test_row_passes_with_every_thread_count():
    X, Q = synth.pixel_mixture(20000, 784, 12, seed=5)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    opt = dict(bound="exp", B0=16, B=16, grow=1, c_alpha=3e-4)
    with knn.Dataset(Xd) as ds:
        ref = ds.adaptive(Qd, 10, 0.01, 1, trace=True, row_pass=False, threads=512, **opt)
        for th in (256, 512, 1024):
            got = ds.adaptive(Qd, 10, 0.01, 1, trace=True, row_pass=True, threads=th, **opt)
            torch.cuda.synchronize()
            _same(got, ref, th)
