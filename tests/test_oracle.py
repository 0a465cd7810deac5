"""Pins for the CPU oracle: each test checks it against something other than
itself (hand-worked examples, brute force, min-plus algebra, scipy's
Dijkstra, closed forms and invariants the paper states)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import (INF, all_pairs_truth, from_edges, golden_names, load_golden,
                          small_families)


def _adj(g):
    """Normalised adjacency as dict of dict, built independently in Python."""
    a = {u: {} for u in range(g.n)}
    s, d, w = g.edges()
    for u, v, x in zip(s.tolist(), d.tolist(), w.tolist()):
        if u != v and x < a[u].get(v, INF):
            a[u][v] = x
    return a


def _walk_bruteforce(adj, src, H):
    """Least weight over all walks of at most H edges, by enumeration."""
    best = {src: 0}

    def rec(v, dist, hops):
        if hops == H:
            return
        for y, w in adj[v].items():
            nd = dist + w
            if nd < best.get(y, INF):
                best[y] = nd
            rec(y, nd, hops + 1)

    rec(src, 0, 0)
    return best


# ---------------------------------------------------------------------------
# Hand-worked examples (tests/golden/)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", golden_names())
def test_golden_examples(name):
    spec = load_golden(name)
    tie = O.TIE_ID if spec.get("tie_break") == "id" else O.TIE_HASHED
    ch = O.build_ch(spec["graph"], spec["hop_limit"], tie, cmax=spec.get("cmax", O.CMAX_ALL),
                    ball=spec.get("ball", O.CMAX_ALL), theta=spec.get("theta", 0),
                    prune=bool(spec.get("prune", 0)), level_work=spec.get("level_work", O.CMAX_ALL),
                    composite=bool(spec.get("composite", 0)))
    assert sorted(map(tuple, ch.pruned.tolist())) == sorted(spec.get("pruned", []))
    if "expect_searches" in spec:
        assert ch.searches == spec["expect_searches"]
    if "expect_witness_work" in spec:
        assert ch.witness_work == spec["expect_witness_work"]
    assert ch.rounds == spec["expect_rounds"]
    if "expect_stats" in spec:  # every round's counters, row after row
        assert ch.stats.ravel().tolist() == spec["expect_stats"]
    assert ch.level.tolist() == spec["expect_level"]
    assert ch.priority.tolist() == spec["expect_priority"]
    assert ch.rank.tolist() == spec["expect_rank"]
    assert len(ch.shortcuts) == spec["expect_shortcuts"]
    assert sorted(map(tuple, ch.shortcuts.tolist())) == sorted(spec["shortcuts"])
    for s, t, d in spec["queries"]:
        assert int(ch.query([s], [t])[0]) == d


# ---------------------------------------------------------------------------
# Hop-limited distance d_H
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("H", [0, 1, 2, 3, 4])
def test_hop_limited_vs_walk_enumeration(seed, H):
    g = I.random_digraph(7, 16, 1, 9, seed=seed)
    adj = _adj(g)
    for src in range(g.n):
        best = _walk_bruteforce(adj, src, H)
        got = O.hop_limited(g, H, src)
        want = np.array([best.get(v, INF) for v in range(g.n)], dtype=np.uint32)
        assert np.array_equal(got, want), (src, got, want)


@pytest.mark.parametrize("seed", range(4))
def test_hop_limited_vs_min_plus_power(seed):
    g = I.random_digraph(50, 160, 1, 40, seed=200 + seed)
    adj = _adj(g)
    W = np.full((g.n, g.n), np.inf)
    np.fill_diagonal(W, 0)
    for u in adj:
        for v, w in adj[u].items():
            W[u, v] = w
    D = np.full_like(W, np.inf)
    np.fill_diagonal(D, 0)
    for H in range(0, 7):
        if H > 0:
            D = np.min(D[:, :, None] + W[None, :, :], axis=1)  # (D (+) W) in min-plus
        for src in (0, 7, 31):
            got = O.hop_limited(g, H, src).astype(np.float64)
            got[got == INF] = np.inf
            assert np.array_equal(got, D[src]), (H, src)


def test_hop_limited_long_equals_dijkstra():
    g = I.geometric_knn_graph(80, seed=11)
    truth = all_pairs_truth(g)
    for src in (0, 13, 79):
        assert np.array_equal(O.hop_limited(g, g.n, src).astype(np.uint64), truth[src])


# ---------------------------------------------------------------------------
# Plain routines
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,g", small_families())
def test_dijkstra_vs_scipy(name, g):
    truth = all_pairs_truth(g)
    for src in range(0, g.n, max(1, g.n // 7)):
        assert np.array_equal(O.dijkstra(g, src).astype(np.uint64), truth[src]), src


def test_normalize_drops_loops_and_merges_min():
    g = from_edges(4, [(0, 0, 5), (0, 1, 7), (0, 1, 3), (0, 1, 9), (1, 2, 4),
                       (2, 1, 4), (3, 3, 1), (2, 0, 8), (2, 0, 8)])
    off, tgt, w = O.normalize(g)
    assert off.tolist() == [0, 1, 2, 4, 4]
    assert tgt.tolist() == [1, 2, 0, 1]
    assert w.tolist() == [3, 4, 8, 4]


# ---------------------------------------------------------------------------
# Scores (Alg. 4) against a brute-force recount
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("H", [0, 1, 2, 5])
def test_round0_scores_bruteforce(seed, H):
    g = I.random_digraph(8, 22, 1, 6, seed=300 + seed)
    adj = _adj(g)
    radj = {u: {} for u in range(g.n)}
    for u in adj:
        for v, w in adj[u].items():
            radj[v][u] = w
    dh = {s: _walk_bruteforce(adj, s, H) for s in range(g.n)}
    want = []
    for u in range(g.n):
        cnt = 0
        for v1, w1 in radj[u].items():
            for v2, w2 in adj[u].items():
                if v1 != v2 and w1 + w2 <= dh[v1].get(v2, INF):
                    cnt += 1
        want.append(cnt - len(radj[u]) - len(adj[u]))
    assert O.round0_scores(g, H).tolist() == want


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("H,ball", [(3, 2), (4, 4), (5, 6), (2, 1), (5, 100)])
def test_round0_scores_with_ball_bound_bruteforce(seed, H, ball):
    # The bounded witness search, written out: labels below the source's
    # heaviest candidate weight, levels 1..H, stopping after the first level
    # at which more than `ball` vertices hold such a label.
    g = I.random_digraph(9, 26, 1, 6, seed=320 + seed)
    adj = _adj(g)
    radj = {u: {} for u in range(g.n)}
    for u in adj:
        for v, w in adj[u].items():
            radj[v][u] = w
    dist = {}
    for s in range(g.n):
        bound = max([w1 + w2 for u, w1 in adj[s].items() for v, w2 in adj[u].items() if v != s],
                    default=0)
        if bound == 0:
            continue
        for h in range(1, H + 1):
            lab = {v: d for v, d in _walk_bruteforce(adj, s, h).items() if d < bound}
            if len(lab) > ball:
                break
        dist[s] = lab
    want = []
    for u in range(g.n):
        cnt = 0
        for v1, w1 in radj[u].items():
            for v2, w2 in adj[u].items():
                if v1 != v2 and w1 + w2 <= dist.get(v1, {}).get(v2, INF):
                    cnt += 1
        want.append(cnt - len(radj[u]) - len(adj[u]))
    assert O.round0_scores(g, H, ball=ball).tolist() == want


@pytest.mark.parametrize("ball", [0, 1, 3, 10])
@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph1", "sparse2", "grid8", "geo150", "rmat8",
                                             "chain30")],
                         ids=lambda x: x if isinstance(x, str) else "")
def test_ball_bound_keeps_distances(name, g, ball):
    ch = O.build_ch(g, 5, ball=ball)
    ss, tt = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = ch.query(ss.ravel().astype(np.uint32), tt.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))
    # a bound at least the graph's size never stops a search
    full, big = O.build_ch(g, 5), O.build_ch(g, 5, ball=g.n)
    assert np.array_equal(full.shortcuts, big.shortcuts) and np.array_equal(full.rank, big.rank)


# ---------------------------------------------------------------------------
# The CH invariant: every upward-upward query equals the true distance
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,g", small_families())
@pytest.mark.parametrize("H,tie", [(5, O.TIE_HASHED), (0, O.TIE_HASHED), (1, O.TIE_ID),
                                   (2, O.TIE_HASHED), (3, O.TIE_ID)])
def test_all_pairs_query_equals_truth(name, g, H, tie):
    ch = O.build_ch(g, H, tie, tie_seed=17)
    truth = all_pairs_truth(g)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    got = ch.query(s.ravel(), t.ravel()).astype(np.uint64).reshape(g.n, g.n)
    assert np.array_equal(got, truth)


@pytest.mark.parametrize("name,g", small_families())
def test_structure_invariants(name, g):
    ch = O.build_ch(g, 5)
    n = g.n
    assert (ch.level != INF).all()
    assert sorted(ch.rank.tolist()) == list(range(n))
    # rank follows (level, score, id)
    order = sorted(range(n), key=lambda u: (int(ch.level[u]), int(ch.priority[u]), u))
    assert [int(ch.rank[u]) for u in order] == list(range(n))
    # every CH edge joins a lower level to a strictly higher level
    # (so V_F of each round is independent) and points upward in rank
    for u, x, w in ch.up.tolist():
        assert ch.level[x] > ch.level[u] and ch.rank[x] > ch.rank[u]
    for x, u, w in ch.down.tolist():
        assert ch.level[x] > ch.level[u] and ch.rank[x] > ch.rank[u]
    # each shortcut is the sum of the two CH edges of its contracted vertex
    upw = {(u, x): w for u, x, w in ch.up.tolist()}
    dnw = {(x, u): w for x, u, w in ch.down.tolist()}
    for r, v1, v2, w, via in ch.shortcuts.tolist():
        assert ch.level[via] == r
        assert ch.level[v1] > r and ch.level[v2] > r
        assert w == dnw[(v1, via)] + upw[(via, v2)]
    # per-round bookkeeping adds up
    st = ch.stats
    assert st[:, 2].sum() == n
    assert np.all(st[:, 2] >= 1)
    assert np.all(st[:, 5] <= st[:, 4]) and np.all(st[:, 6] <= st[:, 5])
    assert np.all(st[:, 7] <= st[:, 6])
    assert st[:, 7].sum() == len(ch.shortcuts)
    assert st[-1, 8] == 0 and st[-1, 9] == 0
    # round 0 rescoring covers every vertex
    assert st[0, 0] == n


# ---------------------------------------------------------------------------
# Special cases with closed forms
# ---------------------------------------------------------------------------

def test_hop_zero_keeps_every_candidate():
    for g in (I.random_digraph(40, 150, 1, 9, seed=5), I.geometric_knn_graph(200, seed=6)):
        ch = O.build_ch(g, 0)
        assert np.array_equal(ch.stats[:, 5], ch.stats[:, 4])


def test_complete_unit_digraph_needs_no_shortcut():
    for n in (3, 5, 8):
        ch = O.build_ch(I.complete_graph(n, 1), 5)
        assert len(ch.shortcuts) == 0
        assert len(ch.up) + len(ch.down) == n * (n - 1)


def test_star_contracts_leaves_first_without_shortcuts():
    for k in (3, 6, 11):
        ch = O.build_ch(I.star_graph(k, seed=k), 5)
        assert len(ch.shortcuts) == 0
        assert ch.level[0] == 1 and (ch.level[1:] == 0).all()


@pytest.mark.parametrize("bidirectional", [False, True])
@pytest.mark.parametrize("tie", [O.TIE_HASHED, O.TIE_ID])
def test_chain_one_shortcut_per_interior_contraction(bidirectional, tie):
    # Sec. 6.1: on a chain every contraction of an inner vertex adds exactly
    # one shortcut (per direction). A vertex was inner iff it still had a
    # neighbour on both sides, i.e. two upward CH edges (one per direction of
    # travel along each side) when stored both ways, one in and one out when
    # directed.
    g = I.chain_graph(200, bidirectional, seed=3)
    ch = O.build_ch(g, 5, tie)
    ups = np.bincount(ch.up[:, 0], minlength=g.n) if len(ch.up) else np.zeros(g.n, int)
    dns = np.bincount(ch.down[:, 1], minlength=g.n) if len(ch.down) else np.zeros(g.n, int)
    if bidirectional:
        inner = (ups == 2) & (dns == 2)
        assert len(ch.shortcuts) == 2 * int(inner.sum())
    else:
        inner = (ups == 1) & (dns == 1)
        assert len(ch.shortcuts) == int(inner.sum())
    # hashed tie-break contracts a constant fraction per round (Sec. 6.4)
    if tie == O.TIE_HASHED:
        assert ch.rounds < 60


def test_empty_and_isolated():
    ch = O.build_ch(I.csr_from_edges(0, [], [], []), 5)
    assert ch.rounds == 0 and ch.level.size == 0
    ch = O.build_ch(I.csr_from_edges(5, [], [], []), 5)
    assert ch.rounds == 1 and (ch.level == 0).all()
    assert ch.query([0, 1], [0, 2]).tolist() == [0, INF]


def test_saturation_drops_unrepresentable_candidates():
    big = 0xFFFFFFFE
    g = from_edges(3, [(0, 1, big), (1, 2, big), (1, 0, big), (2, 1, big)])
    ch = O.build_ch(g, 5, O.TIE_ID)
    assert len(ch.shortcuts) == 0
    assert ch.query([0, 1, 0], [1, 2, 2]).tolist() == [big, big, INF]


def test_rejects_invalid_input():
    with pytest.raises(ValueError):
        O.build_ch(I.Graph(2, np.array([0, 1, 1], np.uint64), np.array([1], np.uint32),
                           np.array([0], np.uint32)))
    with pytest.raises(ValueError):
        O.build_ch(I.Graph(2, np.array([0, 1, 1], np.uint64), np.array([2], np.uint32),
                           np.array([1], np.uint32)))
    with pytest.raises(ValueError):
        O.build_ch(I.Graph(2, np.array([0, 2, 1], np.uint64), np.array([1, 0], np.uint32),
                           np.array([1, 1], np.uint32)))


def test_deterministic():
    g = I.geometric_knn_graph(500, seed=9)
    a, b = O.build_ch(g, 5), O.build_ch(g, 5)
    assert np.array_equal(a.shortcuts, b.shortcuts)
    assert np.array_equal(a.level, b.level) and np.array_equal(a.rank, b.rank)


def test_sampled_queries_on_grid_workload():
    g, params = I.workload("grid64")
    ch = O.build_ch(g, params["hop_limit"])
    s, t = I.random_pairs(g.n, 1000, seed=2)
    assert np.array_equal(ch.query(s, t), O.dijkstra_pairs(g, s, t))
    # the grid keeps the largest component: everything is reachable
    assert (ch.query(s, t) != INF).all()
    # >99% of the vertices go in the first rounds on road-like inputs (Sec. 3.3)
    frac = np.cumsum(ch.stats[:, 2]) / g.n
    assert frac[min(40, len(frac) - 1)] > 0.99


# ---------------------------------------------------------------------------
# Candidate bound Cmax and the core (partial hierarchy)
# ---------------------------------------------------------------------------

P_INELIGIBLE = 2**31 - 2


@pytest.mark.parametrize("cmax", [0, 1, 4, 12, 40])
@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph0", "digraph3", "sparse1", "grid8", "geo150",
                                             "rmat8", "star9", "chain30d")],
                         ids=lambda x: x if isinstance(x, str) else "")
def test_core_queries_equal_truth(name, g, cmax):
    ch = O.build_ch(g, 5, cmax=cmax)
    ss, tt = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = ch.query(ss.ravel().astype(np.uint32), tt.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


@pytest.mark.parametrize("seed", range(4))
def test_core_invariants(seed):
    g = I.random_digraph(80, 320, 1, 20, seed=40 + seed)
    ch = O.build_ch(g, 5, cmax=9)
    core = ch.level == ch.rounds
    assert core.any() and (ch.level <= ch.rounds).all()
    assert (ch.priority[core] == P_INELIGIBLE).all()
    # the core takes the top ranks, in id order (equal level and score)
    top = np.sort(ch.rank[core])
    assert np.array_equal(top, np.arange(g.n - core.sum(), g.n))
    assert np.array_equal(np.argsort(ch.rank)[g.n - core.sum():], np.flatnonzero(core))
    # no shortcut after the last contraction round; core edges stay in the core
    assert (ch.shortcuts[:, 0] < ch.rounds).all() if len(ch.shortcuts) else True
    for u, x, _ in ch.up:
        if core[u]:
            assert core[x]
    for x, u, _ in ch.down:
        if core[u]:
            assert core[x]
    # contracted vertices were eligible when selected: |N_in| * |N_out| <= Cmax,
    # which bounds the candidates they emitted
    per_round = ch.stats[:, 4]
    assert (per_round <= 9 * ch.stats[:, 2]).all()


def test_core_closed_forms():
    # complete digraph: (n - 1)^2 candidates exceed the bound, nothing is
    # eligible, everything is core at level 0
    g = I.complete_graph(6, 1)
    ch = O.build_ch(g, 5, cmax=24)
    assert ch.rounds == 0 and (ch.level == 0).all() and len(ch.shortcuts) == 0
    assert len(ch.up) == 30 and len(ch.down) == 30
    assert (ch.priority == P_INELIGIBLE).all()
    # one bound higher the whole graph is contracted
    assert (O.build_ch(g, 5, cmax=25).level < 2**32 - 1).all()
    # star: the hub (k^2 candidates) waits for its leaves, then goes alone
    g = I.star_graph(9, seed=9)
    ch = O.build_ch(g, 5, cmax=1)
    assert ch.rounds == 2 and ch.level[0] == 1 and (ch.level[1:] == 0).all()
    assert len(ch.shortcuts) == 0
    # bidirectional chain under Cmax = 1: only ends are eligible, so it is
    # peeled from both ends without a single shortcut
    for n in (5, 6, 9):
        g = I.chain_graph(n, True, seed=n)
        ch = O.build_ch(g, 5, cmax=1)
        assert len(ch.shortcuts) == 0
        assert ch.rounds == (n + 1) // 2 + (1 - n % 2)
        assert (ch.level < ch.rounds).all()
        lv = ch.level.astype(np.int64)
        assert (lv[: n // 2] == np.arange(n // 2)).all() or n % 2 == 0


# ---------------------------------------------------------------------------
# The threaded oracle build (-DORACLE_THREADS) gives the same hierarchy
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph2", "grid8", "geo150", "rmat8", "star9")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("cmax,ball", [(O.CMAX_ALL, O.CMAX_ALL), (6, O.CMAX_ALL), (O.CMAX_ALL, 4)])
def test_threaded_build_is_identical(name, g, cmax, ball):
    a = O.build_ch(g, 5, cmax=cmax, ball=ball, trace=True)
    b = O.build_ch(g, 5, cmax=cmax, ball=ball, trace=True, threads=True)
    for f in ("level", "priority", "rank", "shortcuts", "up", "down", "stats", "trace", "labels"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    s, t = s.ravel(), t.ravel()
    da, sa = a.query(s, t, want_settled=True)
    db, sb = b.query(s, t, want_settled=True)  # pairs split over host threads
    assert np.array_equal(da, db) and np.array_equal(sa, sb)


# ---------------------------------------------------------------------------
# Bidirectional trees: every shortest path is the unique tree path
# ---------------------------------------------------------------------------

def _random_tree(n, seed, wmax=30):
    rng = np.random.default_rng(seed)
    label = rng.permutation(n)
    parent = [int(rng.integers(0, i)) for i in range(1, n)]
    w = rng.integers(1, wmax + 1, n - 1)
    edges = []
    for i, (p, c) in enumerate(zip(parent, range(1, n))):
        edges += [(label[p], label[c], int(w[i])), (label[c], label[p], int(w[i]))]
    return from_edges(n, edges)


@pytest.mark.parametrize("seed", range(6))
def test_tree_shortcuts_follow_tree_paths(seed):
    """With exact witnesses (H >= n) on a bidirectional tree, contracting x
    keeps (a, x, b) exactly when x lies on the tree path from a to b, with
    weight dist(a, b); it is inserted when (a, b) is not yet an overlay edge.
    Replaying the oracle's contraction order with that rule alone (no witness
    search) must give its shortcut log."""
    n = 40
    g = _random_tree(n, seed)
    truth = all_pairs_truth(g).astype(np.int64)
    och = O.build_ch(g, n)
    adj = {(a, b) for a, bs in _adj(g).items() for b in bs}
    alive = np.ones(n, bool)
    want = set()
    for r in range(och.rounds):
        F = np.flatnonzero(och.level == r).tolist()
        new = set()
        for x in F:
            nb = {b for (a, b) in adj if a == x and alive[b]}
            for a in nb:
                for b in nb:
                    if a != b and truth[a, x] + truth[x, b] == truth[a, b] and (a, b) not in adj:
                        new.add((r, a, b, int(truth[a, b]), x))
        want |= new
        adj |= {(a, b) for _, a, b, _, _ in new}
        alive[F] = False
        adj = {(a, b) for (a, b) in adj if alive[a] and alive[b]}
    assert set(map(tuple, och.shortcuts.tolist())) == want
    assert np.array_equal(och.one_to_all(np.arange(n)).astype(np.int64), truth)
