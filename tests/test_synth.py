"""The seeded input generators follow their stated recipes (shapes, value
sets, planted distances), are reproducible, and the recall helper scores
candidate sets as stated (no GPU)."""

import numpy as np
import pytest
import torch

from paper_1902_09465_gb300 import runtime, synth


def test_seeded_and_reproducible():
    a = synth.pixel_mixture(500, 32, 4, seed=3)
    b = synth.pixel_mixture(500, 32, 4, seed=3)
    c = synth.pixel_mixture(500, 32, 4, seed=4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])


def test_pixel_mixture_values():
    X, Q = synth.pixel_mixture(3000, 64, 10, seed=1)
    assert X.shape == (3000, 64) and Q.shape == (10, 64) and X.dtype == np.float32
    for A in (X, Q):
        assert A.min() >= 0.0 and A.max() <= 1.0
        codes = A.astype(np.float64) * 255.0
        assert np.allclose(codes, np.rint(codes), atol=1e-4)   # multiples of 1/255


def test_gaussian_planted_rows_sit_near_their_query():
    X, Q, planted = synth.gaussian_planted(2000, 128, 5, nq=3, sigma=0.1, seed=2)
    assert planted.shape == (3, 5) and len(set(planted.ravel().tolist())) == 15
    for qi in range(3):
        d = np.sqrt(((X[planted[qi]] - Q[qi]) ** 2).sum(axis=1))
        assert np.allclose(d, 0.1 * np.sqrt(128), rtol=0.25)    # ||N(0, 0.1^2 I_128)||
        far = np.sqrt(((np.delete(X, planted.ravel(), axis=0)[:200] - Q[qi]) ** 2).sum(axis=1))
        assert far.min() > 3 * d.max()


@pytest.mark.parametrize("background", ["gaussian", "int255"])
def test_gap_planted_distances_follow_the_gap(background):
    n, m, gaps = 4000, 256, [4.0, 2.0, 1.2]
    X, Q, planted = synth.gap_planted(n, m, 3, 6, gaps, seed=5, background=background)
    others = np.setdiff1d(np.arange(n), np.concatenate(planted))
    for qi, gap in enumerate(gaps):
        q = Q[qi].astype(np.float64)
        d_near = np.sqrt(((X[planted[qi]].astype(np.float64) - q) ** 2).sum(axis=1))
        d_far = np.median(np.sqrt(((X[others[:512]].astype(np.float64) - q) ** 2).sum(axis=1)))
        # planted at D_far / gap (D_far here from other rows than the generator's
        # probe; rounding and clipping to [0, 255] move int255 rows further)
        tol = (0.05 if background == "gaussian" else 0.12) * d_far / gap
        assert np.all(np.abs(d_near - d_far / gap) <= tol), (gap, d_near, d_far)
    if background == "int255":
        assert np.array_equal(X, np.clip(np.rint(X), 0, 255))


def test_binary_half_model():
    X, q, near = synth.binary_half(300, 2000, 4, 0.05, 0.45, seed=6)
    assert set(np.unique(X).tolist()) <= {-0.5, 0.5} and set(np.unique(q).tolist()) <= {-0.5, 0.5}
    flips = (X != q).mean(axis=1)
    assert np.all(np.abs(flips[near] - 0.05) < 0.03)
    assert np.all(np.abs(np.delete(flips, near) - 0.45) < 0.06)


def test_recall_counts_ties_and_padding():
    ti = torch.tensor([[1, 2, 3]])
    td = torch.tensor([[1.0, 2.0, 3.0]], dtype=torch.float64)
    assert runtime.recall(ti, td, ti, td) == 1.0
    # one neighbour missing, replaced by a farther point
    gi = torch.tensor([[1, 2, 9]])
    gd = torch.tensor([[1.0, 2.0, 5.0]], dtype=torch.float64)
    assert runtime.recall(gi, gd, ti, td) == pytest.approx(2 / 3)
    # a point tied with the k-th distance (within 1e-6) counts; -1 padding does not
    gi = torch.tensor([[1, 2, 7]])
    gd = torch.tensor([[1.0, 2.0, 3.0 * (1 + 1e-7)]], dtype=torch.float64)
    assert runtime.recall(gi, gd, ti, td) == 1.0
    gi = torch.tensor([[1, 2, -1]])
    gd = torch.tensor([[1.0, 2.0, 3.0]], dtype=torch.float64)
    assert runtime.recall(gi, gd, ti, td) == pytest.approx(2 / 3)
