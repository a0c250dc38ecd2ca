"""The documented draw stream of a (query, point) pair, built from the
oracle's Philox4x32-10 block function -- itself pinned to the published
known-answer vectors and to triton's CPU interpreter (test_oracle.py) -- so
the oracle's coordinate mapping (counter layout, word choice, scaling to
[0, m)) is checked against the stated reading rather than against itself.

Counter (s / 4, point & mask_p, low and high words of qid & mask_q), key (low
and high words of seed); draw s is word s mod 4, scaled by floor(w m / 2^32)."""

import oracle

M32 = 0xFFFFFFFF
FULL = (1 << 64) - 1


def word(seed, qid, point, s, mask_p=FULL, mask_q=FULL):
    qf = qid & mask_q
    blk = oracle.philox4x32_10([s >> 2, (point & mask_p) & M32, qf & M32, (qf >> 32) & M32],
                               [seed & M32, (seed >> 32) & M32])
    return int(blk[s & 3])


def scaled(seed, qid, point, s, n):
    return (word(seed, qid, point, s) * n) >> 32
