"""Seeded synthetic inputs for the adaptive k-NN workloads.

This module draws data only. It holds none of the method's arithmetic (no
distances, no bounds, no sampling of coordinates), so the CPU oracle and the
CUDA path can both be fed from it without sharing any of the computation.

Every generator takes an integer seed and uses numpy's PCG64 generator, so a
(seed, shape) pair always yields the same float32 arrays on every machine.

Workload shapes follow the paper and the benchmark configurations:

* ``gaussian_planted``  i.i.d. N(0,1) points, a N(0,1) query and k planted
  near points at query + N(0, sigma^2) per coordinate.
* ``pixel_mixture``     pixel-like values in [0,1] quantised to 1/255, drawn
  from a mixture of Gaussian centres (stands in for the Tiny ImageNet pixels
  of Section 5, which are not available here).
* ``gap_planted``       a background cloud plus, per query, k planted points
  at distance D_far / gap, D_far being the query's median distance to the
  background; the hardness of a query is set by that gap ratio.
* ``binary_half``       coordinates in {-1/2, +1/2}, the data model of
  Theorem 2 (Section 4.2): a sample of a squared difference is then an exact
  Bernoulli draw of the normalised distance.
* ``subspace``          x = c Q y with Q Gaussian with unit-norm columns, y
  uniform on the unit sphere and c the largest scale with ||x||_inf <= 1/2
  (the synthetic data of Section 5).
* ``coherent_axis``     every point on one standard basis axis (the coherent
  example of Section 4.2, where adaptive sampling cannot save anything).
"""

from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian_planted(n: int, m: int, k: int, nq: int = 1, sigma: float = 0.1, seed: int = 0):
    """N(0,1) points; each query gets k planted rows query + N(0, sigma^2).

    Returns (X [n,m] f32, Q [nq,m] f32, planted [nq,k] int64). Planted rows
    of different queries are distinct rows chosen by the generator.
    """
    if nq * k > n:
        raise ValueError("not enough rows to plant k points per query")
    g = _rng(seed)
    X = g.standard_normal((n, m), dtype=np.float64)
    Q = g.standard_normal((nq, m), dtype=np.float64)
    rows = g.permutation(n)[: nq * k].reshape(nq, k)
    for qi in range(nq):
        X[rows[qi]] = Q[qi][None, :] + sigma * g.standard_normal((k, m))
    return X.astype(np.float32), Q.astype(np.float32), np.sort(rows, axis=1).astype(np.int64)


def pixel_mixture(n: int, m: int, nq: int, n_centres: int = 100, sigma: float = 0.1, seed: int = 0):
    """Pixel-like mixture: centres ~ U[0,1]^m, point = centre + N(0, sigma^2),
    clipped to [0,1] and rounded to a multiple of 1/255. Queries come from the
    same mixture. Returns (X [n,m] f32, Q [nq,m] f32)."""
    g = _rng(seed)
    centres = g.random((n_centres, m))

    def draw(cnt):
        out = np.empty((cnt, m), dtype=np.float32)
        step = 8192
        for s in range(0, cnt, step):
            e = min(cnt, s + step)
            c = g.integers(0, n_centres, size=e - s)
            v = centres[c] + sigma * g.standard_normal((e - s, m))
            v = np.clip(v, 0.0, 1.0)
            out[s:e] = (np.rint(v * 255.0) / 255.0).astype(np.float32)
        return out

    X = draw(n)
    Q = draw(nq)
    return X, Q


def gap_planted(n: int, m: int, nq: int, k, gap, seed: int = 0, background: str = "gaussian",
                dfar_sample: int = 256):
    """Background cloud plus, for each query, k planted rows at distance
    D_far / gap along random directions. D_far is the median distance from
    the query to ``dfar_sample`` background rows drawn by the generator.

    ``k`` and ``gap`` may be scalars or per-query arrays. ``background`` is
    "gaussian" (N(0,1) values) or "int255" (clip(round(N(64, 40^2)), 0, 255)
    values stored as float32; planted rows are rounded and clipped the same way).

    Returns (X [n,m] f32, Q [nq,m] f32, planted list of int64 arrays).
    """
    g = _rng(seed)
    ks = np.broadcast_to(np.asarray(k, dtype=np.int64), (nq,)).copy()
    gaps = np.broadcast_to(np.asarray(gap, dtype=np.float64), (nq,)).copy()
    if int(ks.sum()) > n:
        raise ValueError("not enough rows to plant")

    def bg(shape):
        if background == "gaussian":
            return g.standard_normal(shape, dtype=np.float32)
        if background == "int255":
            v = g.normal(64.0, 40.0, size=shape)
            return np.clip(np.rint(v), 0, 255).astype(np.float32)
        raise ValueError(background)

    X = np.empty((n, m), dtype=np.float32)
    step = 1 << 16
    for s in range(0, n, step):
        X[s:min(n, s + step)] = bg((min(n, s + step) - s, m))
    Q = bg((nq, m)).astype(np.float32)
    perm = g.permutation(n)
    planted = []
    off = 0
    for qi in range(nq):
        kk = int(ks[qi])
        rows = np.sort(perm[off: off + kk])
        off += kk
        probe = X[g.integers(0, n, size=dfar_sample)].astype(np.float64)
        dfar = float(np.median(np.sqrt(((probe - Q[qi].astype(np.float64)) ** 2).sum(axis=1))))
        r = dfar / float(gaps[qi])
        u = g.standard_normal((kk, m))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        P = Q[qi].astype(np.float64)[None, :] + r * u
        if background == "int255":
            P = np.clip(np.rint(P), 0, 255)
        X[rows] = P.astype(np.float32)
        planted.append(rows.astype(np.int64))
    return X, Q, planted


def binary_half(n: int, m: int, k: int, p_near: float, p_far: float, seed: int = 0):
    """Coordinates in {-1/2, +1/2} (Theorem 2 data model). The query is
    uniform; k rows (returned) differ from it in a p_near fraction of
    coordinates, the rest in a p_far fraction (each coordinate flipped
    independently). Returns (X [n,m] f32, q [1,m] f32, near [k] int64)."""
    g = _rng(seed)
    q = np.where(g.random(m) < 0.5, -0.5, 0.5)
    near = np.sort(g.permutation(n)[:k])
    p = np.full(n, p_far)
    p[near] = p_near
    flips = g.random((n, m)) < p[:, None]
    X = np.where(flips, -q[None, :], q[None, :])
    return X.astype(np.float32), q[None, :].astype(np.float32), near.astype(np.int64)


def subspace(n: int, m: int, p: int, nq: int = 1, seed: int = 0):
    """x = c Q y (Section 5): Q in R^{m x p} Gaussian with unit-norm columns,
    y uniform on the unit sphere of R^p, c the largest scalar with
    ||x||_inf <= 1/2 over all generated points and queries.
    Returns (X [n,m] f32, Q [nq,m] f32)."""
    g = _rng(seed)
    B = g.standard_normal((m, p))
    B /= np.linalg.norm(B, axis=0, keepdims=True)
    Y = g.standard_normal((n + nq, p))
    Y /= np.linalg.norm(Y, axis=1, keepdims=True)
    Z = Y @ B.T
    c = 0.5 / np.abs(Z).max()
    Z *= c
    return Z[:n].astype(np.float32), Z[n:].astype(np.float32)


def coherent_axis(n: int, m: int, axis: int = 0, seed: int = 0):
    """Every point and the query on the axis e_axis (Section 4.2 coherent
    example): only one coordinate differs from zero.
    Returns (X [n,m] f32, q [1,m] f32)."""
    g = _rng(seed)
    X = np.zeros((n, m), dtype=np.float32)
    X[:, axis] = (g.random(n) - 0.5).astype(np.float32)
    q = np.zeros((1, m), dtype=np.float32)
    q[0, axis] = np.float32(g.random() - 0.5)
    return X, q


def mixture_planted(n: int, m: int, npool: int, centres: int = 64, sigma_frac: float = 0.1, kplant: int = 10,
                    gap_lo: float = 1.2, gap_hi: float = 4.0, seed: int = 0, dfar_sample: int = 64):
    """Gaussian mixture with planted neighbours (a resident serving dataset):
    `centres` centres ~ N(0, I); a point is a centre plus N(0, s^2) per
    coordinate with s = sigma_frac times the centres' per-coordinate spread
    (1); a pool of `npool` queries is drawn from the mixture and each gets
    `kplant` planted rows at distance D_far / g, g ~ U[gap_lo, gap_hi] and
    D_far the query's median distance to `dfar_sample` rows of its own
    cluster (the points that compete with the planted ones, so g is the ratio
    of the competitors' distance to the planted neighbours' distance).
    Returns (X [n,m] f32, pool [npool,m] f32)."""
    g = _rng(seed)
    C = g.standard_normal((centres, m))
    X = np.empty((n, m), dtype=np.float32)
    lab = np.empty(n, dtype=np.int64)
    step = 1 << 15
    for s in range(0, n, step):
        e = min(n, s + step)
        c = g.integers(0, centres, size=e - s)
        lab[s:e] = c
        X[s:e] = (C[c] + sigma_frac * g.standard_normal((e - s, m))).astype(np.float32)
    c = g.integers(0, centres, size=npool)
    P = (C[c] + sigma_frac * g.standard_normal((npool, m))).astype(np.float32)
    if npool * kplant > n:
        raise ValueError("not enough rows to plant")
    rows = g.permutation(n)[: npool * kplant].reshape(npool, kplant)
    members = [np.flatnonzero(lab == j) for j in range(centres)]
    for qi in range(npool):
        own = members[c[qi]]
        pick = own[g.integers(0, len(own), size=dfar_sample)] if len(own) else g.integers(0, n, size=dfar_sample)
        probe = X[pick].astype(np.float64)
        dfar = float(np.median(np.sqrt(((probe - P[qi].astype(np.float64)) ** 2).sum(axis=1))))
        r = dfar / g.uniform(gap_lo, gap_hi)
        u = g.standard_normal((kplant, m))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        X[rows[qi]] = (P[qi].astype(np.float64)[None, :] + r * u).astype(np.float32)
    return X, P
