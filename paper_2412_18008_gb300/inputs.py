"""Seeded synthetic inputs: graphs in CSR form and s-t query pairs.

This module only produces inputs. It holds none of the contraction-hierarchy
arithmetic (no normalisation, no scoring, no shortest paths): both the CUDA
path and the CPU oracle receive exactly the arrays returned here and process
them independently.

Every graph is returned as a :class:`Graph` with

* ``n``        number of vertices,
* ``offsets``  ``uint64[n + 1]`` out-CSR offsets,
* ``targets``  ``uint32[m]`` edge heads,
* ``weights``  ``uint32[m]`` edge weights, each in ``[1, 0xFFFFFFFE]``.

Raw generators may emit self-loops and parallel edges (the RMAT family and
the ``random_digraph`` family do, on purpose); removing them is the job of the
method's own input normalisation.

The synthetic families stand in for the paper's datasets (Sec. 6.1): road
networks are replaced by a perturbed grid and by geometric k-nearest-neighbour
graphs with road-like travel-time weights; the paper's chain graphs are
reproduced directly (weights 1..32, as in Sec. 6.1).

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64), whose
streams are identical on every platform, and the draw order is fixed in each
function's docstring.
"""
from __future__ import annotations

from typing import NamedTuple

import numpy as np

INF = 0xFFFFFFFF
MAX_WEIGHT = 0xFFFFFFFE


class Graph(NamedTuple):
    n: int
    offsets: np.ndarray  # uint64[n+1]
    targets: np.ndarray  # uint32[m]
    weights: np.ndarray  # uint32[m]

    @property
    def m(self) -> int:
        return int(self.targets.shape[0])

    def edges(self):
        """Return (src, dst, w) arrays of the CSR, in storage order."""
        deg = np.diff(self.offsets.astype(np.int64))
        src = np.repeat(np.arange(self.n, dtype=np.uint32), deg)
        return src, self.targets, self.weights


def csr_from_edges(n: int, src, dst, w) -> Graph:
    """Pack an edge list into an out-CSR, ordered by (src, dst, w).

    Ordering is a storage choice only; duplicates and self-loops are kept.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    if src.size:
        if src.min() < 0 or src.max() >= n or dst.min() < 0 or dst.max() >= n:
            raise ValueError("edge endpoint out of range")
        if w.min() < 1 or w.max() > MAX_WEIGHT:
            raise ValueError("edge weight out of [1, 0xFFFFFFFE]")
    order = np.lexsort((w, dst, src))
    src, dst, w = src[order], dst[order], w[order]
    counts = np.bincount(src, minlength=n) if src.size else np.zeros(n, np.int64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=offsets[1:])
    return Graph(n, offsets, dst.astype(np.uint32), w.astype(np.uint32))


def _both_directions(a, b, w):
    return (np.concatenate([a, b]), np.concatenate([b, a]), np.concatenate([w, w]))


# ---------------------------------------------------------------------------
# Road-like families
# ---------------------------------------------------------------------------

def grid_graph(rows: int = 64, cols: int = 64, delete_frac: float = 0.10,
               wmin: int = 1, wmax: int = 100, seed: int = 1) -> Graph:
    """4-neighbour grid with a random fraction of its undirected edges deleted.

    Draw order: one permutation of the undirected edge list (horizontal edges
    in row-major order, then vertical edges in row-major order); its first
    ``round(delete_frac * E)`` entries are deleted. Then one integer weight in
    ``[wmin, wmax]`` per surviving undirected edge, in edge-list order; both
    directions carry that weight. The largest connected component is kept
    (ties: the one holding the smallest vertex id) and relabelled in ascending
    order of the original ids.
    """
    rng = np.random.default_rng(seed)
    vid = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    ha, hb = vid[:, :-1].ravel(), vid[:, 1:].ravel()
    va, vb = vid[:-1, :].ravel(), vid[1:, :].ravel()
    a = np.concatenate([ha, va])
    b = np.concatenate([hb, vb])
    E = a.size
    k = int(round(delete_frac * E))
    perm = rng.permutation(E)
    keep = np.ones(E, dtype=bool)
    keep[perm[:k]] = False
    a, b = a[keep], b[keep]
    w = rng.integers(wmin, wmax + 1, size=a.size, dtype=np.int64)
    n0 = rows * cols
    comp = _components(n0, a, b)
    sizes = np.bincount(comp, minlength=comp.max() + 1)
    best = sizes.max()
    # smallest vertex id among the largest components
    first_vertex = np.full(sizes.size, n0, dtype=np.int64)
    np.minimum.at(first_vertex, comp, np.arange(n0))
    cand = np.nonzero(sizes == best)[0]
    target = cand[np.argmin(first_vertex[cand])]
    keepv = comp == target
    newid = np.cumsum(keepv) - 1
    m = keepv[a] & keepv[b]
    a, b, w = newid[a[m]], newid[b[m]], w[m]
    n = int(keepv.sum())
    s, d, ww = _both_directions(a, b, w)
    return csr_from_edges(n, s, d, ww)


def _components(n, a, b):
    """Connected-component label per vertex (undirected), by union-find."""
    parent = np.arange(n, dtype=np.int64)

    def find(x):
        root = x
        while parent[root] != root:
            root = parent[root]
        while parent[x] != root:
            parent[x], x = root, parent[x]
        return root

    for x, y in zip(a.tolist(), b.tolist()):
        rx, ry = find(x), find(y)
        if rx != ry:
            if rx < ry:
                parent[ry] = rx
            else:
                parent[rx] = ry
    return np.array([find(i) for i in range(n)], dtype=np.int64)


def geometric_knn_graph(n: int, k: int = 3, oneway_frac: float = 0.05,
                        speeds=(1, 2, 4), weight_scale: float = 1000.0,
                        scale_by_sqrt_n: bool = False, seed: int = 3) -> Graph:
    """Road-like geometric graph: points in the unit square joined to their
    ``k`` nearest neighbours, symmetrised, with a fraction of one-way edges.

    Draw order: ``n`` points ``(x, y)`` uniform in ``[0, 1)^2``; then, over
    the undirected edges sorted by ``(min id, max id)``: one speed-factor
    index per edge, one uniform for the one-way test, one coin for the kept
    direction of a one-way edge.  Weight =
    ``max(1, floor(weight_scale * length * factor + 0.5))`` where ``length`` is
    the Euclidean length (times ``sqrt(n)`` when ``scale_by_sqrt_n``).
    A one-way edge keeps ``min -> max`` when its coin is 0, else ``max -> min``.
    Neighbours come from an exact k-d tree search; equal distances are broken
    by the tree and are measure-zero events for uniform points.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    kk = min(k + 1, n)
    if n <= 1:
        return csr_from_edges(n, [], [], [])
    _, idx = cKDTree(pts).query(pts, k=kk, workers=-1)
    idx = np.asarray(idx, dtype=np.int64).reshape(n, kk)
    rows = np.arange(n, dtype=np.int64)[:, None]
    # drop the point itself (normally column 0); if absent, drop the last column
    is_self = idx == rows
    has_self = is_self.any(axis=1)
    drop_col = np.where(has_self, is_self.argmax(axis=1), kk - 1)
    mask = np.ones_like(idx, dtype=bool)
    mask[np.arange(n), drop_col] = False
    nbr = idx[mask].reshape(n, kk - 1)[:, :k]
    src = np.repeat(np.arange(n, dtype=np.int64), nbr.shape[1])
    dst = nbr.ravel()
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    key = np.sort(lo * n + hi)  # sorted distinct keys (np.unique's result, faster)
    if key.size:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    a, b = key // n, key % n
    E = a.size
    f = np.asarray(speeds, dtype=np.float64)[rng.integers(0, len(speeds), size=E)]
    oneway = rng.random(E) < oneway_frac
    coin = rng.integers(0, 2, size=E)
    d = pts[a] - pts[b]
    length = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1])
    if scale_by_sqrt_n:
        length = length * np.sqrt(n)
    w = np.maximum(1, np.floor(weight_scale * length * f + 0.5)).astype(np.int64)
    w = np.minimum(w, MAX_WEIGHT)
    fwd = ~oneway | (coin == 0)
    bwd = ~oneway | (coin == 1)
    s = np.concatenate([a[fwd], b[bwd]])
    t = np.concatenate([b[fwd], a[bwd]])
    ww = np.concatenate([w[fwd], w[bwd]])
    # (s, t) pairs are distinct here, so ordering by s * n + t is the
    # (src, dst, w) order csr_from_edges would produce
    order = np.argsort(s * n + t, kind="stable")
    s, t, ww = s[order], t[order], ww[order]
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(s, minlength=n), out=offsets[1:])
    return Graph(n, offsets, t.astype(np.uint32), ww.astype(np.uint32))


# ---------------------------------------------------------------------------
# Non-road stress family
# ---------------------------------------------------------------------------

def rmat_graph(scale: int = 21, nsamples: int = 1 << 25, a: float = 0.57,
               b: float = 0.19, c: float = 0.19, wmin: int = 1, wmax: int = 1000,
               seed: int = 8) -> Graph:
    """R-MAT edge sampler (Chakrabarti et al.) on ``2**scale`` vertices.

    Draw order: for each of the ``scale`` bit levels (most significant first)
    one uniform per sample selects the quadrant (a | b | c | d); then one
    integer weight in ``[wmin, wmax]`` per sample. Self-loops and duplicate
    samples are kept; the method's normalisation drops and merges them.
    """
    rng = np.random.default_rng(seed)
    n = 1 << scale
    u = np.zeros(nsamples, dtype=np.int64)
    v = np.zeros(nsamples, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for lvl in range(scale):
        r = rng.random(nsamples)
        bit = np.int64(1) << np.int64(scale - 1 - lvl)
        right = ((r >= a) & (r < ab)) | (r >= abc)
        down = r >= ab
        v += np.where(right, bit, 0)
        u += np.where(down, bit, 0)
    w = rng.integers(wmin, wmax + 1, size=nsamples, dtype=np.int64)
    return csr_from_edges(n, u, v, w)


# ---------------------------------------------------------------------------
# Small structured and random families (tests)
# ---------------------------------------------------------------------------

def chain_graph(n: int, bidirectional: bool = True, wmin: int = 1, wmax: int = 32,
                seed: int = 0) -> Graph:
    """Path 0 - 1 - ... - n-1; one weight per link in ``[wmin, wmax]``, both
    directions equal when ``bidirectional`` (the paper's chain graphs use
    weights 1..32)."""
    rng = np.random.default_rng(seed)
    a = np.arange(max(n - 1, 0), dtype=np.int64)
    b = a + 1
    w = rng.integers(wmin, wmax + 1, size=a.size, dtype=np.int64)
    if bidirectional:
        a, b, w = _both_directions(a, b, w)
    return csr_from_edges(n, a, b, w)


def star_graph(leaves: int, wmin: int = 1, wmax: int = 32, seed: int = 0) -> Graph:
    """Centre 0 joined both ways to ``leaves`` leaves; one weight per link."""
    rng = np.random.default_rng(seed)
    b = np.arange(1, leaves + 1, dtype=np.int64)
    a = np.zeros_like(b)
    w = rng.integers(wmin, wmax + 1, size=b.size, dtype=np.int64)
    s, d, ww = _both_directions(a, b, w)
    return csr_from_edges(leaves + 1, s, d, ww)


def complete_graph(n: int, weight: int = 1) -> Graph:
    """Complete digraph without self-loops, every edge of the same weight."""
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    m = s != d
    return csr_from_edges(n, s[m], d[m], np.full(int(m.sum()), weight))


def random_digraph(n: int, m: int, wmin: int = 1, wmax: int = 32, seed: int = 0,
                   allow_loops: bool = True) -> Graph:
    """``m`` directed edges with endpoints uniform in ``[0, n)`` (so possibly
    self-loops and parallel edges) and weights uniform in ``[wmin, wmax]``.
    Draw order: all sources, all heads, all weights."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, size=m, dtype=np.int64)
    d = rng.integers(0, n, size=m, dtype=np.int64)
    w = rng.integers(wmin, wmax + 1, size=m, dtype=np.int64)
    if not allow_loops:
        keep = s != d
        s, d, w = s[keep], d[keep], w[keep]
    return csr_from_edges(n, s, d, w)


def random_pairs(n: int, k: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """``k`` s-t pairs, sources then targets, each uniform in ``[0, n)``."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, size=k, dtype=np.int64).astype(np.uint32)
    t = rng.integers(0, n, size=k, dtype=np.int64).astype(np.uint32)
    return s, t


# ---------------------------------------------------------------------------
# The workloads the benchmarks and parity tests use, by name
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# Query-server workloads
# ---------------------------------------------------------------------------

def request_mix(n: int, count: int, seed: int, one_to_many: float = 0.2, kmax: int = 1024):
    """Seeded request mix: sources uniform in [0, n); with probability
    1 - one_to_many a single target, else k = floor(2**U[0, log2 kmax])
    targets (log-uniform 1..kmax), all uniform. Returns (src, ks, targets)."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=count, dtype=np.int64).astype(np.uint32)
    many = rng.random(count) < one_to_many
    ks = np.where(many, np.floor(2.0 ** (rng.random(count) * np.log2(kmax))), 1).astype(np.uint32)
    ks = np.maximum(ks, 1)
    targets = rng.integers(0, n, size=int(ks.sum()), dtype=np.int64).astype(np.uint32)
    return src, ks, targets


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (ns) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1e9 / rate_per_s, size=count)
    return np.cumsum(gaps).astype(np.uint64)



def workload(name: str) -> tuple[Graph, dict]:
    """Named workload -> (graph, build parameters)."""
    if name == "grid64":
        return grid_graph(64, 64, 0.10, 1, 100, seed=1), dict(hop_limit=5)
    if name.startswith("geo"):
        # "geo1M", "geo256K", "geo20K", ...
        tag = name[3:]
        scale = {"K": 1000, "M": 1_000_000}
        nn = int(tag[:-1]) * scale[tag[-1]] if tag[-1] in scale else int(tag)
        return geometric_knn_graph(nn, seed=3), dict(hop_limit=5)
    raise KeyError(name)
