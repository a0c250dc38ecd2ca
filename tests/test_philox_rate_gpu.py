"""knn_philox_blocks runs the kernels' own Philox4x32-10 function: with one
block per thread, thread t's word is the XOR of the four words of block
(counter 0, t, 0x9E3779B9, 0x7F4A7C15; key = the two halves of seed
0x243F6A8885A308D3), which the oracle's generator (pinned to the published
known answers) must reproduce; with more blocks the words are their running
sum. A rate measurement that ran another function would be worthless."""

import numpy as np
import pytest
import torch

import oracle
from paper_1902_09465_gb300 import knn

pytestmark = pytest.mark.gpu

SEED = 0x243F6A8885A308D3
KEY = [SEED & 0xFFFFFFFF, SEED >> 32]


def _block_xor(i, t):
    w = oracle.philox4x32_10([i, t, 0x9E3779B9, 0x7F4A7C15], KEY)
    return int(w[0] ^ w[1] ^ w[2] ^ w[3])


def test_generator_rate_kernel_runs_the_kernels_generator():
    out = torch.zeros(2 * 1024, dtype=torch.int32, device="cuda")
    knn.philox_blocks(1, 2, out)
    got = out.cpu().numpy().astype(np.uint32)
    for t in (0, 1, 31, 1023, 1024, 2047):
        assert int(got[t]) == _block_xor(0, t), t
    knn.philox_blocks(3, 1, out)
    got = out.cpu().numpy().astype(np.uint32)
    for t in (0, 7, 1023):
        assert int(got[t]) == sum(_block_xor(i, t) for i in range(3)) % (1 << 32), t


def test_generator_rate_kernel_rejects_bad_arguments():
    out = torch.zeros(1024, dtype=torch.int32, device="cuda")
    with pytest.raises(knn.KnnError):
        knn.philox_blocks(1, 2, out)  # fewer words than threads
    with pytest.raises(knn.KnnError):
        knn.philox_blocks(-1, 1, out)
