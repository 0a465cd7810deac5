"""Oracle pins for Alg. 3 as the paper writes it (no GPU): the witness search
capped at theta settled vertices, the pruning of overlay edges heavier than
their pair's witness distance, the memoised distance map kept across rounds,
and the one-to-all query (PHAST, which the paper cites for SSSP on a CH).

Pins, none of which goes through the oracle's own search code:
  * theta = 1 settles only the source, so every candidate pair is kept: the
    hierarchy equals the one of hop limit 0 (every d_0(v1, v2) is INF).
  * theta >= n settles every reachable vertex, and a hop limit >= n - 1
    admits every simple path: both give exact distances, so the two
    hierarchies are identical.
  * every pruned edge (s, v, w) has w > dist(s, v) in the input graph
    (scipy's Dijkstra), so pruning never deletes a needed edge.
  * one-to-all rows equal scipy's all-pairs Dijkstra, with or without a core,
    a ball bound, a settled cap or pruning.
  * with hop limit 0 or theta = 1 every recorded value is INF, so
    memoisation cannot change a decision: the same hierarchy.
  * a level-work bound of 0 leaves level 1 alone: the hierarchy of hop
    limit 1.
  * every query is exact in every mode.
Round-by-round re-derivations of both modes are in test_trace_pins.py."""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import INF, all_pairs_truth, small_families

FAMILIES = small_families()


def _same(a, b):
    assert a.level.tolist() == b.level.tolist()
    assert a.priority.tolist() == b.priority.tolist()
    assert a.rank.tolist() == b.rank.tolist()
    assert a.shortcuts.tolist() == b.shortcuts.tolist()
    assert a.stats.tolist() == b.stats.tolist()
    assert sorted(map(tuple, a.up.tolist())) == sorted(map(tuple, b.up.tolist()))
    assert sorted(map(tuple, a.down.tolist())) == sorted(map(tuple, b.down.tolist()))


def _all_pairs(ch, n):
    s, t = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return ch.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32)).reshape(n, n)


@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_theta_one_equals_hop_limit_zero(name, g):
    for tie in (O.TIE_HASHED, O.TIE_ID):
        _same(O.build_ch(g, 5, tie, theta=1), O.build_ch(g, 0, tie))


@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_theta_unbounded_equals_exact_hop_limit(name, g):
    H = max(g.n, 1)
    _same(O.build_ch(g, 3, theta=g.n + 5), O.build_ch(g, H))
    _same(O.build_ch(g, 3, theta=g.n, cmax=6), O.build_ch(g, H, cmax=6))


@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_memo_changes_nothing_where_every_value_is_inf(name, g):
    # hop limit 0 and theta = 1 record INF for every pair, so reusing a value
    # decides exactly as a fresh search would: the same hierarchy, and never
    # more searches
    for kw in (dict(hop_limit=0), dict(hop_limit=5, theta=1)):
        a = O.build_ch(g, **kw)
        b = O.build_ch(g, memo=1 << 40, **kw)
        _same(a, b)
        assert b.searches <= a.searches


def test_memo_halves_the_searches_on_a_geometric_graph():
    g = I.geometric_knn_graph(5000, seed=21)
    a = O.build_ch(g, 5)
    b = O.build_ch(g, 5, memo=1 << 40)
    assert b.searches < 0.7 * a.searches
    s, t = I.random_pairs(g.n, 3000, seed=22)
    assert np.array_equal(b.query(s, t), O.dijkstra_pairs(g, s, t))


@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_level_work_zero_equals_hop_limit_one(name, g):
    # with no out-edge allowed past the first level a search runs level 1
    # alone (a second level whose frontier has no out-edge lowers nothing)
    _same(O.build_ch(g, 5, level_work=0), O.build_ch(g, 1))
    _same(O.build_ch(g, 4, level_work=0, cmax=6), O.build_ch(g, 1, cmax=6))


def test_level_work_bound_cuts_the_work_on_rmat():
    g = I.rmat_graph(scale=10, nsamples=16 << 10, wmax=1000, seed=8)
    a = O.build_ch(g, 2, cmax=256, ball=256)
    b = O.build_ch(g, 2, cmax=256, ball=256, level_work=1024)
    assert b.witness_work * 5 < a.witness_work
    s, t = I.random_pairs(g.n, 2000, seed=9)
    want = O.dijkstra_pairs(g, s, t)
    assert np.array_equal(a.query(s, t), want)
    assert np.array_equal(b.query(s, t), want)


def test_theta_and_ball_are_exclusive():
    g = I.random_digraph(10, 30, 1, 5, seed=1)
    with pytest.raises(ValueError):
        O.build_ch(g, 5, theta=4, ball=3)


MODES = [dict(), dict(prune=True), dict(theta=3), dict(theta=3, prune=True),
         dict(ball=2, prune=True), dict(cmax=4, prune=True), dict(cmax=4, theta=8),
         dict(memo=1 << 40), dict(memo=30, prune=True), dict(memo=1 << 40, theta=4, cmax=4),
         dict(level_work=6), dict(level_work=10, prune=True, memo=1 << 40, cmax=4)]


@pytest.mark.parametrize("mode", MODES, ids=[",".join(f"{k}={v}" for k, v in m.items()) or "plain"
                                            for m in MODES])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_queries_and_one_to_all_are_exact(name, g, mode):
    och = O.build_ch(g, 4, **mode)
    truth = all_pairs_truth(g)
    assert np.array_equal(_all_pairs(och, g.n).astype(np.uint64), truth)
    assert np.array_equal(och.one_to_all(np.arange(g.n)).astype(np.uint64), truth)
    for r, s, v, w in och.pruned.tolist():
        assert truth[s, v] < w, (r, s, v, w)


@pytest.mark.parametrize("seed", range(4))
def test_pruning_deletes_edges_on_geometric_graphs(seed):
    # 3-NN graphs with a hop limit of 2: a witness beyond two hops is missed,
    # the shortcut is kept, and a later round finds the lighter walk
    g = I.geometric_knn_graph(400, seed=70 + seed)
    plain = O.build_ch(g, 2)
    pr = O.build_ch(g, 2, prune=True)
    assert pr.pruned.shape[0] > 0
    assert plain.pruned.shape[0] == 0
    s, t = I.random_pairs(g.n, 2000, seed=80 + seed)
    want = O.dijkstra_pairs(g, s, t)
    assert np.array_equal(pr.query(s, t), want)
    assert np.array_equal(plain.query(s, t), want)


def test_one_to_all_edge_cases():
    one = O.build_ch(I.Graph(1, np.zeros(2, np.uint64), np.zeros(0, np.uint32),
                             np.zeros(0, np.uint32)), 5)
    assert one.one_to_all([0]).tolist() == [[0]]
    g = I.chain_graph(12, False, seed=3)
    och = O.build_ch(g, 5)
    d = och.one_to_all([0, 11, 5])
    assert d.shape == (3, 12)
    truth = all_pairs_truth(g)
    assert np.array_equal(d.astype(np.uint64), truth[[0, 11, 5]])
    assert d[1, 0] == INF  # a directed chain runs one way
    assert och.one_to_all([]).shape == (0, 12)
    with pytest.raises(ValueError):
        och.one_to_all([12])


def test_one_to_all_on_larger_graphs():
    for g in (I.geometric_knn_graph(3000, seed=11), I.rmat_graph(scale=10, nsamples=6000,
                                                                 wmax=100, seed=12)):
        och = O.build_ch(g, 5, cmax=64)
        src = np.array([0, 17, g.n - 1, g.n // 2], np.uint32)
        d = och.one_to_all(src)
        for i, s in enumerate(src.tolist()):
            assert np.array_equal(d[i], O.dijkstra(g, s))
