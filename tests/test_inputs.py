"""Seeded synthetic inputs: the shapes and distributions the workloads ask
for (no GPU)."""
import numpy as np

from paper_2412_18008_gb300 import inputs as I


def test_request_mix_shape_and_distribution():
    src, ks, tg = I.request_mix(1000, 200_000, seed=1)
    assert src.dtype == np.uint32 and ks.dtype == np.uint32 and tg.dtype == np.uint32
    assert src.max() < 1000 and tg.max() < 1000 and tg.size == int(ks.sum())
    assert ks.min() >= 1 and ks.max() <= 1024
    one = ks == 1
    # 80% single targets, plus the one-to-many requests that drew k = 1
    # (2^U[0,10] < 2 with probability 1/10)
    assert abs(one.mean() - (0.8 + 0.2 * 0.1)) < 0.01
    # log-uniform k: log2(k) of one-to-many requests is uniform on [0, 10),
    # floored; each unit bin holds about 10% of them
    many = ks[~one].astype(np.float64)
    hist = np.bincount(np.floor(np.log2(many)).astype(int), minlength=10)[:10] / (~one).sum()
    assert np.all(np.abs(hist[1:] - 1 / 9) < 0.02)
    # deterministic
    a, b = I.request_mix(1000, 1000, seed=5), I.request_mix(1000, 1000, seed=5)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_poisson_arrivals_rate():
    arr = I.poisson_arrivals(200_000, rate_per_s=50_000, seed=3)
    assert arr.dtype == np.uint64 and np.all(np.diff(arr.astype(np.int64)) >= 0)
    rate = arr.size / (arr[-1] * 1e-9)
    assert abs(rate / 50_000 - 1) < 0.01
    gaps = np.diff(arr.astype(np.float64)) * 1e-9
    # exponential gaps: standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1) < 0.02


def test_geometric_graph_shape():
    g = I.geometric_knn_graph(20_000, seed=3)
    src, dst, w = g.edges()
    assert (w >= 1).all() and (src != dst).all()
    deg = np.diff(g.offsets.astype(np.int64))
    # 3 nearest neighbours symmetrised, 5% one-way: about 3.6 out-edges each
    assert 3.3 < deg.mean() < 3.9
    pairs = set(zip(src.tolist(), dst.tolist()))
    oneway = sum((b, a) not in pairs for a, b in pairs)
    assert 0.02 < oneway / len(pairs) < 0.06


def test_rmat_graph_shape():
    g = I.rmat_graph(scale=10, nsamples=1 << 14, wmax=1000, seed=8)
    src, dst, w = g.edges()
    assert g.n == 1024 and src.size == 1 << 14
    assert w.min() >= 1 and w.max() <= 1000
    # a = 0.57: the low quadrant dominates, so vertex 0 is the heaviest hub
    outdeg = np.bincount(src, minlength=g.n)
    assert outdeg.argmax() == 0 and outdeg[0] > 20 * outdeg.mean()
