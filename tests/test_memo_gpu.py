"""Memoised witness distances across rounds (witness_memo_limit), the
level-work bound (witness_level_work), the pruning of overlay edges
(witness_prune) and Alg. 3's settled-vertex cap (witness_settle_cap) on the
GPU, against the oracle run with
the same settings: levels, scores, ranks, shortcut logs, E_up, E_down and
every round's counters bit for bit, and exact queries. The oracle modes are
pinned in test_trace_pins.py (the test's own map, bound, clearing rule,
frontier and work sums, deletion log) and test_witness_modes.py."""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import all_pairs_truth, small_families
from tests.test_gpu_parity import assert_same_hierarchy

pytestmark = pytest.mark.gpu


def _ch():
    from paper_2412_18008_gb300 import ch
    return ch


FAMILIES = small_families()


@pytest.mark.parametrize("H,limit,cmax,ball", [(5, 1 << 30, None, None), (2, 1 << 30, None, None),
                                               (5, 40, None, None), (3, 1 << 30, 6, None),
                                               (4, 25, None, 3), (0, 1 << 30, None, None)])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_small_families(name, g, H, limit, cmax, ball):
    och = O.build_ch(g, H, cmax=O.CMAX_ALL if cmax is None else cmax,
                     ball=O.CMAX_ALL if ball is None else ball, memo=limit)
    gch = _ch().CH.build(g, hop_limit=H, max_candidates_per_vertex=cmax, witness_ball_limit=ball,
                         witness_memo_limit=limit)
    assert_same_hierarchy(gch, och)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = gch.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


@pytest.mark.parametrize("limit", [1 << 30, 200_000, 5_000])
def test_geometric(limit):
    g = I.geometric_knn_graph(20_000, seed=151)
    och = O.build_ch(g, 5, memo=limit)
    gch = _ch().CH.build(g, hop_limit=5, witness_memo_limit=limit)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 5000, seed=152)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


def test_dense_graph_tiers_and_rmat_core():
    # balls that outgrow both shared-memory tiers, and hubs in a core
    for g, kw in ((I.random_digraph(1500, 9000, 1, 1000, seed=97, allow_loops=False), dict(H=4)),
                  (I.rmat_graph(scale=12, nsamples=1 << 15, wmax=1000, seed=91), dict(H=3, cmax=64))):
        cmax = kw.get("cmax")
        och = O.build_ch(g, kw["H"], cmax=O.CMAX_ALL if cmax is None else cmax, memo=1 << 30)
        gch = _ch().CH.build(g, hop_limit=kw["H"], max_candidates_per_vertex=cmax,
                             witness_memo_limit=1 << 30)
        assert_same_hierarchy(gch, och)
        s, t = I.random_pairs(g.n, 3000, seed=153)
        assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


# ---------------------------------------------------------------------------
# Level-work bound (witness_level_work), alone and with memoised distances
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("H,lw,limit,ball", [(3, 4, None, None), (5, 12, None, None),
                                             (5, 40, 1 << 30, None), (4, 12, None, 5),
                                             (5, 20, 30, 6)])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_level_work_small_families(name, g, H, lw, limit, ball):
    och = O.build_ch(g, H, ball=O.CMAX_ALL if ball is None else ball, memo=limit or 0,
                     level_work=lw)
    gch = _ch().CH.build(g, hop_limit=H, witness_ball_limit=ball, witness_memo_limit=limit,
                         witness_level_work=lw)
    assert_same_hierarchy(gch, och)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = gch.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


@pytest.mark.parametrize("lw,limit", [(1024, None), (256, 1 << 30)])
def test_level_work_on_rmat_with_a_core(lw, limit):
    g = I.rmat_graph(scale=12, nsamples=1 << 16, wmax=1000, seed=154)
    och = O.build_ch(g, 2, cmax=256, ball=256, memo=limit or 0, level_work=lw)
    gch = _ch().CH.build(g, hop_limit=2, max_candidates_per_vertex=256, witness_ball_limit=256,
                         witness_memo_limit=limit, witness_level_work=lw)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 3000, seed=155)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


# ---------------------------------------------------------------------------
# Pruning of overlay edges (witness_prune), with and without memoisation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("H,limit,ball,cmax", [(5, None, None, None), (2, None, None, None),
                                               (5, 1 << 30, None, None), (4, 30, None, None),
                                               (4, None, 3, None), (5, 1 << 30, None, 6)])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_prune_small_families(name, g, H, limit, ball, cmax):
    och = O.build_ch(g, H, ball=O.CMAX_ALL if ball is None else ball,
                     cmax=O.CMAX_ALL if cmax is None else cmax, memo=limit or 0, prune=True)
    gch = _ch().CH.build(g, hop_limit=H, witness_ball_limit=ball, max_candidates_per_vertex=cmax,
                         witness_memo_limit=limit, witness_prune=True)
    assert_same_hierarchy(gch, och)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = gch.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


@pytest.mark.parametrize("H,limit,lw", [(2, None, None), (5, 1 << 30, None), (5, 1 << 30, 64)])
def test_prune_geometric(H, limit, lw):
    g = I.geometric_knn_graph(20_000, seed=156)
    och = O.build_ch(g, H, memo=limit or 0, prune=True,
                     level_work=O.CMAX_ALL if lw is None else lw)
    assert och.pruned.shape[0] > 0
    gch = _ch().CH.build(g, hop_limit=H, witness_memo_limit=limit, witness_prune=True,
                         witness_level_work=lw)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 5000, seed=157)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


# ---------------------------------------------------------------------------
# Alg. 3's settled-vertex cap (witness_settle_cap), alone and with memo and
# pruning
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("theta,limit,prune,cmax", [(1, None, False, None), (3, None, False, None),
                                                    (20, None, False, None), (10**6, None, False, None),
                                                    (8, 1 << 30, False, None), (8, 30, True, None),
                                                    (6, 1 << 30, False, 6)])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_settled_cap_small_families(name, g, theta, limit, prune, cmax):
    och = O.build_ch(g, 5, theta=theta, memo=limit or 0, prune=prune,
                     cmax=O.CMAX_ALL if cmax is None else cmax)
    gch = _ch().CH.build(g, hop_limit=5, witness_settle_cap=theta, witness_memo_limit=limit,
                         witness_prune=prune, max_candidates_per_vertex=cmax)
    assert_same_hierarchy(gch, och)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = gch.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


def _settle_cap_cases():
    geo = lambda: I.geometric_knn_graph(20_000, seed=158)
    # 400 settled vertices outgrow a warp's 256-slot table: the global-memory
    # tier. (A small cap on this dense digraph lets the overlay fill in: at
    # theta = 50 the oracle alone needs a minute for 600 vertices.)
    dense = lambda: I.random_digraph(600, 3600, 1, 1000, seed=159, allow_loops=False)
    return [("geo20K", geo, 50), ("geo20K", geo, 400), ("dense600", dense, 400)]


@pytest.mark.parametrize("name,make,theta", _settle_cap_cases(), ids=lambda v: str(v) if not callable(v) else "")
def test_settled_cap_geometric_and_dense(name, make, theta):
    g = make()
    och = O.build_ch(g, 5, theta=theta)
    gch = _ch().CH.build(g, hop_limit=5, witness_settle_cap=theta)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 3000, seed=160)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))

