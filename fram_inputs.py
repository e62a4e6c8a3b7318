"""Seeded synthetic graph-pair generators for the FRAM workloads.

This module holds only input generation (random graphs, planted
permutations, noise); it contains none of the matching method's arithmetic.
Both the CUDA path's tests/benchmark and the CPU oracle's tests draw their
inputs from here, so the two sides always see identical matrices.

Conventions
-----------
* Every matrix is a dense, row-major, C-contiguous ``float64`` array of shape
  ``(n, n)``, symmetric, nonnegative, with a zero diagonal (undirected graphs
  with nonnegative edge attributes, Sec. 3 "Graph").
* Planted convention: ``B[p[i], p[j]] = A[i, j]`` before noise, so the true
  correspondence of node ``i`` of the first graph is node ``p[i]`` of the
  second; ``truth[i] = p[i]``.
* ``N(0, s)`` is read as a normal law with standard deviation ``s``.
* Noise is added to existing edges only (upper triangle, mirrored) and the
  result is clamped at zero so inputs stay nonnegative.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class GraphPair:
    """One matching problem: two adjacency matrices and the planted truth."""

    A: np.ndarray
    B: np.ndarray
    truth: np.ndarray          # int64[n]; -1 where a node has no true partner
    theta: float               # the paper's setting: 2 dense, 10 sparse (Sec. 7)
    meta: dict = field(default_factory=dict)
    F: np.ndarray | None = None    # n x d node attributes of the first graph
    Ft: np.ndarray | None = None   # n x d node attributes of the second graph

    @property
    def n(self) -> int:
        return int(self.A.shape[0])


def _symmetric_from_upper(U: np.ndarray) -> np.ndarray:
    U = np.triu(U, 1)
    return U + U.T


def _permute(A: np.ndarray, p: np.ndarray) -> np.ndarray:
    """Return B with B[p[i], p[j]] = A[i, j]."""
    n = A.shape[0]
    inv = np.empty(n, dtype=np.int64)
    inv[p] = np.arange(n)
    return np.ascontiguousarray(A[np.ix_(inv, inv)])


def _edge_noise(B: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    if sigma <= 0:
        return B
    n = B.shape[0]
    U = np.triu(B, 1)
    mask = U > 0
    U = U + mask * rng.normal(0.0, sigma, size=(n, n))
    U = np.maximum(U, 0.0)
    return _symmetric_from_upper(U)


def er_graph(n: int, p: float, rng: np.random.Generator) -> np.ndarray:
    """Symmetric Erdos-Renyi graph with U(0,1) edge weights and zero diagonal."""
    mask = rng.random((n, n)) < p
    w = rng.random((n, n))
    return _symmetric_from_upper(np.where(mask, w, 0.0))


def er_pair(n: int, p: float, noise: float = 0.0, flip_frac: float = 0.0,
            seed: int = 0, theta: float = 10.0) -> GraphPair:
    """ER graph and a planted, noisy, relabelled copy.

    ``flip_frac`` deletes that fraction of the copy's edges and adds the same
    number of new edges (U(0,1) weights) between non-adjacent node pairs.
    """
    rng = np.random.default_rng(seed)
    A = er_graph(n, p, rng)
    perm = rng.permutation(n).astype(np.int64)
    B = _permute(A, perm)
    B = _edge_noise(B, noise, rng)
    if flip_frac > 0:
        U = np.triu(B, 1)
        iu = np.triu_indices(n, 1)
        vals = U[iu]
        on = np.flatnonzero(vals > 0)
        off = np.flatnonzero(vals == 0)
        k = int(round(flip_frac * on.size))
        k = min(k, off.size)
        if k > 0:
            dele = rng.choice(on, size=k, replace=False)
            add = rng.choice(off, size=k, replace=False)
            vals = vals.copy()
            vals[dele] = 0.0
            vals[add] = rng.random(k)
            U = np.zeros((n, n))
            U[iu] = vals
        B = _symmetric_from_upper(U)
    return GraphPair(np.ascontiguousarray(A), np.ascontiguousarray(B), perm, theta,
                     dict(kind="er", n=n, p=p, noise=noise, flip_frac=flip_frac, seed=seed))


def _flip_binary_edges(B: np.ndarray, flip_frac: float, rng: np.random.Generator) -> np.ndarray:
    """Delete flip_frac of the edges of a 0/1 graph and add as many new ones."""
    n = B.shape[0]
    iu = np.triu_indices(n, 1)
    vals = B[iu].copy()
    on = np.flatnonzero(vals > 0)
    off = np.flatnonzero(vals == 0)
    k = min(int(round(flip_frac * on.size)), off.size)
    if k > 0:
        vals[rng.choice(on, size=k, replace=False)] = 0.0
        vals[rng.choice(off, size=k, replace=False)] = 1.0
    U = np.zeros((n, n))
    U[iu] = vals
    return _symmetric_from_upper(U)


def social_pair(n: int = 4039, m: int = 88234, flip_frac: float = 0.05, seed: int = 0,
                exponent: float = 3.1, theta: float = 10.0) -> GraphPair:
    """Unweighted social-network-like pair: a Chung-Lu graph whose expected
    degrees follow a power law (exponent 3.1: at the default size the largest
    degree is near 1,200 and the median near 33), scaled so the expected edge
    count is m (n and m default to the size of the Facebook ego graph), a
    planted relabelling, and flip_frac of the copy's edges moved at random."""
    rng = np.random.default_rng(seed)
    w = (np.arange(1, n + 1, dtype=np.float64)) ** (-1.0 / (exponent - 1.0))
    w = w[rng.permutation(n)]
    iu = np.triu_indices(n, 1)
    scale = 1.0
    for _ in range(50):          # fix the scale so that sum_{i<j} p_ij = m
        ws = w * scale
        P = np.minimum(1.0, np.outer(ws, ws) / ws.sum())
        e = P[iu].sum()
        if abs(e - m) <= 1e-6 * m:
            break
        scale *= m / e
    U = np.zeros((n, n))
    U[iu] = (rng.random(iu[0].size) < P[iu]).astype(np.float64)
    A = _symmetric_from_upper(U)
    perm = rng.permutation(n).astype(np.int64)
    B = _flip_binary_edges(_permute(A, perm), flip_frac, rng) if flip_frac > 0 else _permute(A, perm)
    return GraphPair(np.ascontiguousarray(A), np.ascontiguousarray(B), perm, theta,
                     dict(kind="social", n=n, m=m, flip_frac=flip_frac, seed=seed,
                          edges=int(U.sum())))


def _kernel_from_points(P: np.ndarray) -> np.ndarray:
    """Gaussian-kernel adjacency exp(-d^2/sigma^2), sigma = median pairwise distance."""
    sq = np.sum(P * P, axis=1)
    d2 = sq[:, None] + sq[None, :] - 2.0 * (P @ P.T)
    np.maximum(d2, 0.0, out=d2)
    n = P.shape[0]
    iu = np.triu_indices(n, 1)
    sigma = float(np.median(np.sqrt(d2[iu]))) if n > 1 else 1.0
    if sigma <= 0:
        sigma = 1.0
    K = np.exp(-d2 / (sigma * sigma))
    np.fill_diagonal(K, 0.0)
    K = 0.5 * (K + K.T)          # exact symmetry
    return np.ascontiguousarray(K)


def gaussian_pair(n: int, jitter: float = 0.01, seed: int = 0, theta: float = 2.0) -> GraphPair:
    """Dense Gaussian-kernel graph on U[0,1]^2 points and a permuted, jittered copy
    rebuilt with the same sigma rule."""
    rng = np.random.default_rng(seed)
    P = rng.random((n, 2))
    perm = rng.permutation(n).astype(np.int64)
    Q = np.empty_like(P)
    Q[perm] = P
    Q = Q + rng.normal(0.0, jitter, size=Q.shape)
    return GraphPair(_kernel_from_points(P), _kernel_from_points(Q), perm, theta,
                     dict(kind="gaussian", n=n, jitter=jitter, seed=seed))


def _descriptors(rng: np.random.Generator, n: int, d: int) -> np.ndarray:
    """Nonnegative unit-norm rows, like normalised gradient histograms."""
    F = np.abs(rng.normal(0.0, 1.0, size=(n, d)))
    return F / np.linalg.norm(F, axis=1, keepdims=True)


def attributed_pair(n: int, d: int = 128, desc_noise: float = 0.5, jitter: float = 0.01,
                    seed: int = 0, theta: float = 2.0) -> GraphPair:
    """Dense Gaussian-kernel pair (as ``gaussian_pair``) whose nodes also carry
    d-dimensional descriptors.  Node p[i] of the second graph gets node i's
    descriptor plus N(0, desc_noise / sqrt(d)) per component, clamped at zero
    and renormalised, so both sides stay nonnegative with unit norm."""
    g = gaussian_pair(n, jitter=jitter, seed=seed, theta=theta)
    rng = np.random.default_rng(seed + 1_000_003)
    F = _descriptors(rng, n, d)
    Ft = np.empty_like(F)
    noisy = np.maximum(F + rng.normal(0.0, desc_noise / np.sqrt(d), size=F.shape), 0.0)
    Ft[g.truth] = noisy / np.maximum(np.linalg.norm(noisy, axis=1, keepdims=True), 1e-300)
    g.F, g.Ft = F, Ft
    g.meta.update(kind="attributed", d=d, desc_noise=desc_noise)
    return g


def keypoint_pair(rng: np.random.Generator, n_min: int = 10, n_max: int = 64,
                  jitter: float = 0.02, max_outlier_frac: float = 0.2,
                  theta: float = 2.0) -> GraphPair:
    """Small keypoint-like pair with outliers, padded to a square problem.

    ``n`` ~ U{n_min..n_max}.  Each side keeps ``m`` inliers (shared points,
    jittered on the second side) plus its own outliers (0-20% of ``n``);
    the smaller side is padded with isolated dummy nodes so both have ``n``
    nodes.  ``truth`` is -1 for outliers and dummies.
    """
    n = int(rng.integers(n_min, n_max + 1))
    o1 = int(rng.integers(0, int(max_outlier_frac * n) + 1))
    o2 = int(rng.integers(0, int(max_outlier_frac * n) + 1))
    m = n - max(o1, o2)
    inl = rng.random((m, 2))
    P = np.vstack([inl, rng.random((o1, 2))])
    perm_in = rng.permutation(n)[:m]            # slots of the inliers on side 2
    Q = rng.random((n, 2))                      # outlier positions by default
    Q[perm_in] = inl + rng.normal(0.0, jitter, size=inl.shape)
    side2_real = np.zeros(n, dtype=bool)
    side2_real[perm_in] = True
    others = np.flatnonzero(~side2_real)
    side2_real[others[:o2]] = True              # o2 outliers, the rest are dummies
    A = np.zeros((n, n))
    A[: m + o1, : m + o1] = _kernel_from_points(P)
    real = np.flatnonzero(side2_real)
    B = np.zeros((n, n))
    B[np.ix_(real, real)] = _kernel_from_points(Q[real])
    truth = -np.ones(n, dtype=np.int64)
    truth[:m] = perm_in
    return GraphPair(A, B, truth, theta, dict(kind="keypoint", n=n, inliers=m, o1=o1, o2=o2))


def keypoint_batch(count: int, seed: int = 0, **kw) -> list[GraphPair]:
    rng = np.random.default_rng(seed)
    return [keypoint_pair(rng, **kw) for _ in range(count)]


def serving_stream(count: int, seed: int = 0, n_min: int = 20, n_max: int = 2048,
                   p: float = 0.1, noise: float = 0.05, rate: float = 1.0):
    """Poisson arrivals (rate per second) with log-uniform n over [n_min, n_max].

    Returns ``(arrival_times, specs)``; each spec is ``(n, seed)`` for
    :func:`er_pair` so large pairs are only materialised when needed.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    logn = rng.uniform(np.log(n_min), np.log(n_max), size=count)
    ns = np.clip(np.round(np.exp(logn)).astype(int), n_min, n_max)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return t, [(int(n_), int(s_)) for n_, s_ in zip(ns, seeds)]


def serving_pair(n: int, seed: int, p: float = 0.1, noise: float = 0.05) -> GraphPair:
    return er_pair(n, p, noise=noise, seed=seed, theta=10.0)


# The workloads the benchmarks and parity tests use, by name.
def small_er_pair(seed: int = 0) -> GraphPair:
    """n=50, ER p=0.2, U(0,1) weights, N(0,0.02) edge noise; theta=10."""
    return er_pair(50, 0.2, noise=0.02, seed=seed, theta=10.0)


def medium_er_pair(seed: int = 0) -> GraphPair:
    """n=1000, ER p=0.05, N(0,0.05) edge noise, 5% edge flips; theta=10."""
    return er_pair(1000, 0.05, noise=0.05, flip_frac=0.05, seed=seed, theta=10.0)


def attributed_medium_pair(seed: int = 0) -> GraphPair:
    """n=1000 dense Gaussian-kernel pair with d=128 node descriptors, theta=2."""
    return attributed_pair(1000, d=128, seed=seed)


def facebook_like_pair(seed: int = 0) -> GraphPair:
    """n=4039 power-law social pair with about 88,234 edges, 5% edge flips."""
    return social_pair(4039, 88234, 0.05, seed)


def large_gaussian_pair(seed: int = 0, n: int = 8192) -> GraphPair:
    """n=8192 dense Gaussian-kernel pair, N(0,0.01) jitter; theta=2."""
    return gaussian_pair(n, jitter=0.01, seed=seed, theta=2.0)
