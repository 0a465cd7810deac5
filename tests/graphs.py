"""Small helpers shared by the tests (no method arithmetic)."""
import os

import numpy as np

from paper_2412_18008_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INF = 0xFFFFFFFF


def from_edges(n, edges):
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 3)
    return I.csr_from_edges(n, e[:, 0], e[:, 1], e[:, 2])


def load_golden(name):
    """Parse a hand-worked fixture from tests/golden/."""
    spec = {"edges": [], "shortcuts": [], "queries": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "edge":
                spec["edges"].append(tuple(int(v) for v in vals))
            elif key == "shortcut":
                spec["shortcuts"].append(tuple(int(v) for v in vals))
            elif key == "pruned":
                spec.setdefault("pruned", []).append(tuple(int(v) for v in vals))
            elif key == "query":
                s, t, d = vals
                spec["queries"].append((int(s), int(t), INF if d == "inf" else int(d)))
            elif key == "tie_break":
                spec[key] = vals[0]
            elif key.startswith("expect_") and len(vals) != 1:
                spec[key] = [int(v) for v in vals]
            else:
                spec[key] = int(vals[0])
    spec["graph"] = from_edges(spec["n"], spec["edges"])
    return spec


def golden_names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


def small_families():
    """(name, graph) pairs spanning the structures the method meets."""
    out = []
    for seed in range(6):
        out.append((f"digraph{seed}", I.random_digraph(40, 120, 1, 8, seed=seed)))
        out.append((f"sparse{seed}", I.random_digraph(60, 90, 1, 32, seed=100 + seed)))
    out.append(("grid8", I.grid_graph(8, 8, 0.1, 1, 20, seed=3)))
    out.append(("grid10u", I.grid_graph(10, 10, 0.0, 1, 1, seed=4)))
    out.append(("geo150", I.geometric_knn_graph(150, seed=5)))
    out.append(("geo120s", I.geometric_knn_graph(120, seed=6, scale_by_sqrt_n=True)))
    out.append(("chain30", I.chain_graph(30, True, seed=7)))
    out.append(("chain30d", I.chain_graph(30, False, seed=8)))
    out.append(("star9", I.star_graph(9, seed=9)))
    out.append(("complete6", I.complete_graph(6, 1)))
    out.append(("rmat8", I.rmat_graph(scale=7, nsamples=600, wmax=20, seed=10)))
    return out


def all_pairs_truth(g):
    """All-pairs distances from scipy's Dijkstra (INF where unreachable)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import dijkstra

    src, dst, w = g.edges()
    keep = src != dst
    src, dst, w = src[keep], dst[keep], w[keep].astype(np.float64)
    # duplicates: keep the minimum weight per (src, dst)
    if src.size:
        order = np.lexsort((w, dst, src))
        src, dst, w = src[order], dst[order], w[order]
        first = np.ones(src.size, dtype=bool)
        first[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
        src, dst, w = src[first], dst[first], w[first]
    mat = sp.csr_matrix((w, (src, dst)), shape=(g.n, g.n))
    d = dijkstra(mat, directed=True)
    out = np.full(d.shape, INF, dtype=np.uint64)
    fin = np.isfinite(d)
    out[fin] = d[fin].astype(np.uint64)
    return out
