"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module draws data only: Gaussian-mixture feature matrices, MNIST-shaped
uint8 images, random kNN-shaped graphs (uniform, or with planted clusters)
and random 2-D positions.  It holds
none of the IVHD arithmetic (no distances, forces, updates or neighbour
sampling), so both implementations can consume the same inputs without
sharing any of the method.

All draws use numpy's PCG64 with an explicit seed.  Feature rows are shuffled
after generation so that vertex order carries no cluster structure, as with
a real dataset stored in arbitrary order.

Workloads (named by content):

* ``gmm2k``    - M=2,000 points in N=50 dims, 10 equal isotropic components,
                 centres ~ N(0, 25 I), unit variance; k=2, r=1, c=0.01,
                 1,000 momentum steps (a=0.9, b=0.01).
* ``mnist70k`` - M=70,000 uint8 images of N=784 pixels: 10 prototypes with
                 i.i.d. U{0..255} pixels, x = clip(rint(p + 40 z), 0, 255),
                 7,000 per class; k=5, r=1, c=0.01, 2,000 steps (b=0.001).  Stands in
                 for MNIST (Sec. 4.2, Table of datasets).
* ``gmm1p4m``  - M=1,400,000 points in N=100 dims, 50 components whose sizes
                 follow a power law with exponent 1.5 (largest-remainder
                 rounding), centres ~ N(0, 25 I), unit variance; k=5, r=1,
                 c=0.01, 2,000 momentum steps (a=0.9, b=0.001).  Stands in for YAHOO (M=1.4e6, N=100,
                 Sec. 5.2 comparison table).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    M: int
    N: int
    k: int
    r: int
    c: float
    n_iter: int
    a: float = 0.9
    b: float = 0.01
    dtype: str = "f32"          # feature dtype: "f32" or "u8"
    seed: int = 0


WORKLOADS = {
    "gmm2k": Workload("gmm2k", M=2000, N=50, k=2, r=1, c=0.01, n_iter=1000, seed=2000),
    # b = 1e-3 for the same stability reason as gmm1p4m (hubs of the 784-D kNN graph)
    "mnist70k": Workload("mnist70k", M=70000, N=784, k=5, r=1, c=0.01, n_iter=2000,
                         b=0.001, dtype="u8", seed=70000),
    # b = 1e-3: momentum is stable only while b * lambda_max < 2 (1 + a), and the exact
    # kNN graph of this mixture has a hub of symmetric degree ~2000 (lambda_max ~ 2000)
    "gmm1p4m": Workload("gmm1p4m", M=1400000, N=100, k=5, r=1, c=0.01, n_iter=2000,
                        b=0.001, seed=1400000),
}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def powerlaw_sizes(M: int, n_comp: int, exponent: float) -> np.ndarray:
    """Component sizes proportional to c^-exponent (c = 1..n_comp), summing to M.

    Largest-remainder rounding keeps the total exact.
    """
    w = np.arange(1, n_comp + 1, dtype=np.float64) ** (-exponent)
    q = w / w.sum() * M
    sizes = np.floor(q).astype(np.int64)
    short = M - int(sizes.sum())
    order = np.argsort(-(q - sizes), kind="stable")
    sizes[order[:short]] += 1
    return sizes


def gaussian_mixture(M: int, N: int, n_comp: int, seed: int, *, centre_std: float = 5.0,
                     sizes: np.ndarray | None = None, shuffle: bool = True):
    """Isotropic Gaussian mixture: centres ~ N(0, centre_std^2 I), unit variance.

    Returns ``(X float32 [M, N], labels int32 [M])``.
    """
    rng = _rng(seed)
    if sizes is None:
        sizes = np.full(n_comp, M // n_comp, dtype=np.int64)
        sizes[: M - int(sizes.sum())] += 1
    sizes = np.asarray(sizes, dtype=np.int64)
    assert int(sizes.sum()) == M
    centres = (rng.standard_normal((n_comp, N)) * centre_std).astype(np.float32)
    labels = np.repeat(np.arange(n_comp, dtype=np.int32), sizes)
    X = rng.standard_normal((M, N), dtype=np.float32)
    X += centres[labels]
    if shuffle:
        perm = rng.permutation(M)
        X = X[perm]
        labels = labels[perm]
    return np.ascontiguousarray(X), np.ascontiguousarray(labels)


def mnist_like(M: int, seed: int, *, N: int = 784, n_proto: int = 10, sigma: float = 40.0,
               shuffle: bool = True, noise_seed: int | None = None):
    """uint8 images: prototypes with i.i.d. U{0..255} pixels plus N(0, sigma^2) noise, clipped.

    The prototypes come from ``seed``; the noise, the labels' order and the
    shuffle from ``noise_seed`` (default: the same stream), so several sets can
    share one distribution (training, held-out and arriving points).
    Returns ``(X uint8 [M, N], labels int32 [M])``.
    """
    rng = _rng(seed)
    protos = rng.integers(0, 256, size=(n_proto, N)).astype(np.float32)
    if noise_seed is not None:
        rng = _rng(noise_seed)
    labels = np.repeat(np.arange(n_proto, dtype=np.int32), -(-M // n_proto))[:M]
    X = np.empty((M, N), dtype=np.uint8)
    chunk = 8192
    for s in range(0, M, chunk):
        e = min(M, s + chunk)
        z = rng.standard_normal((e - s, N), dtype=np.float32)
        X[s:e] = np.clip(np.rint(protos[labels[s:e]] + sigma * z), 0, 255).astype(np.uint8)
    if shuffle:
        perm = rng.permutation(M)
        X = X[perm]
        labels = labels[perm]
    return np.ascontiguousarray(X), np.ascontiguousarray(labels)


def workload_features(w: Workload):
    """Feature matrix and mixture labels of a named workload."""
    if w.name == "gmm2k":
        return gaussian_mixture(w.M, w.N, 10, w.seed)
    if w.name == "mnist70k":
        return mnist_like(w.M, w.seed, N=w.N)
    if w.name == "gmm1p4m":
        return gaussian_mixture(w.M, w.N, 50, w.seed, sizes=powerlaw_sizes(w.M, 50, 1.5))
    raise KeyError(w.name)


def random_knn_graph(M: int, k: int, seed: int, *, hub_frac: float = 0.0,
                     n_hubs: int = 0) -> np.ndarray:
    """A kNN-shaped graph: k distinct neighbours per row, never the row itself.

    ``n_hubs`` vertices (ids 0..n_hubs-1) are drawn with probability
    ``hub_frac`` per slot, producing heavily skewed in-degrees like the hubs of
    high-dimensional kNN graphs.  Rows that come out invalid (self or repeated
    id) are redrawn whole until none is left.  Returns int32 [M, k].
    """
    assert 1 <= k <= M - 1
    if n_hubs > 0:
        assert n_hubs > k, "need more hubs than k so hub-only rows stay possible"
    rng = _rng(seed)

    def draw(n):
        c = rng.integers(0, M, size=(n, k), dtype=np.int64)
        if n_hubs > 0 and hub_frac > 0:
            hub = rng.random((n, k)) < hub_frac
            c[hub] = rng.integers(0, n_hubs, size=int(hub.sum()))
        return c

    out = draw(M)
    todo = np.arange(M)
    while todo.size:
        rows = out[todo]
        srt = np.sort(rows, axis=1)
        bad = (rows == todo[:, None]).any(axis=1) | (srt[:, 1:] == srt[:, :-1]).any(axis=1)
        todo = todo[bad]
        if todo.size:
            out[todo] = draw(todo.size)
    return out.astype(np.int32)


def planted_knn_graph(M: int, k: int, seed: int, *, sizes: np.ndarray, p_out: float = 0.02):
    """A kNN-shaped graph with planted clusters, and its cluster labels.

    Vertex i belongs to cluster labels[i] (cluster c has sizes[c] vertices,
    vertex order shuffled).  Each of its k distinct neighbours is drawn
    uniformly from its own cluster with probability 1 - p_out, otherwise
    uniformly from all vertices; self and repeated ids are redrawn (whole
    rows, as in ``random_knn_graph``).  It has the cluster-local structure of
    the kNN graph of a well-separated Gaussian mixture with these cluster
    sizes, at sizes where the graph of the mixture itself cannot be computed
    exactly on the host.  Returns ``(knn int32 [M, k], labels int32 [M])``.
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    assert int(sizes.sum()) == M and int(sizes.min()) > k
    rng = _rng(seed)
    labels = rng.permutation(np.repeat(np.arange(sizes.size, dtype=np.int64), sizes))
    members = np.argsort(labels, kind="stable")          # vertices grouped by cluster
    start = np.concatenate(([0], np.cumsum(sizes)[:-1]))

    def draw(rows):
        lab = labels[rows][:, None]
        inside = members[start[lab] + (rng.random((rows.size, k)) * sizes[lab]).astype(np.int64)]
        anywhere = rng.integers(0, M, size=(rows.size, k), dtype=np.int64)
        return np.where(rng.random((rows.size, k)) < p_out, anywhere, inside)

    out = draw(np.arange(M))
    todo = np.arange(M)
    while todo.size:
        rows = out[todo]
        srt = np.sort(rows, axis=1)
        bad = (rows == todo[:, None]).any(axis=1) | (srt[:, 1:] == srt[:, :-1]).any(axis=1)
        todo = todo[bad]
        if todo.size:
            out[todo] = draw(todo)
    return out.astype(np.int32), labels.astype(np.int32)


def uniform_positions(M: int, seed: int, *, scale: float = 1.0) -> np.ndarray:
    """Random 2-D positions ~ U(0, scale)^2 as float32 [M, 2]."""
    rng = _rng(seed)
    return (rng.random((M, 2)) * scale).astype(np.float32)


def sample_rows(M: int, n: int, seed: int) -> np.ndarray:
    """A sorted seeded sample of ``min(n, M)`` distinct row ids (int64)."""
    if n >= M:
        return np.arange(M, dtype=np.int64)
    rng = _rng(seed)
    return np.sort(rng.choice(M, size=n, replace=False)).astype(np.int64)


def batch_workload(seed: int = 64, n_emb: int = 64, m_lo: int = 5000, m_hi: int = 200000):
    """Many independent embeddings of uneven size: M log-uniform in [m_lo, m_hi],
    N = 64 Gaussian mixtures with 5-30 equal components, k in {2, 3, 5, 10},
    r in {1, 2}.  Returns a list of dicts with X, labels, k, r, seed."""
    rng = _rng(seed)
    out = []
    for e in range(n_emb):
        M = int(round(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi)))))
        comps = int(rng.integers(5, 31))
        k = int(rng.choice([2, 3, 5, 10]))
        r = int(rng.choice([1, 2]))
        X, labels = gaussian_mixture(M, 64, comps, seed * 1000 + e)
        out.append({"X": X, "labels": labels, "k": k, "r": r, "seed": seed * 1000 + e})
    return out
