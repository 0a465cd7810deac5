"""Finite candidate bound (Cmax) and the core it leaves: the GPU hierarchy
equals the oracle's bit for bit (levels, scores, ranks, shortcuts, E_up and
E_down with the core's edges, per-round counters), and queries, which then
also search the core, stay exact."""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import all_pairs_truth, small_families
from tests.test_gpu_parity import assert_same_hierarchy, assert_same_queries

pytestmark = pytest.mark.gpu


def _ch():
    from paper_2412_18008_gb300 import ch
    return ch


FAMILIES = [(n, g) for n, g in small_families()
            if n in ("digraph0", "digraph3", "sparse1", "grid8", "geo150", "rmat8", "star9",
                     "complete6", "chain30")]


@pytest.mark.parametrize("cmax", [0, 1, 4, 12, 40])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_small_families_with_a_core(name, g, cmax):
    och = O.build_ch(g, 5, cmax=cmax)
    gch = _ch().CH.build(g, hop_limit=5, max_candidates_per_vertex=cmax)
    assert_same_hierarchy(gch, och)
    assert gch.stats()["core_vertices"] == int((och.level == och.rounds).sum())
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    s, t = s.ravel().astype(np.uint32), t.ravel().astype(np.uint32)
    d = assert_same_queries(gch, och, s, t)
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))
    assert np.array_equal(gch.query(s, t), d)  # pruned searches too


@pytest.mark.parametrize("cmax", [16, 256])
def test_rmat_with_a_core(cmax):
    # an RMAT graph of the stress family (a = 0.57, b = c = 0.19), scaled
    # down so the oracle finishes in seconds; its hubs stay in the core
    g = I.rmat_graph(scale=12, nsamples=1 << 15, wmax=1000, seed=91)
    och = O.build_ch(g, 5, cmax=cmax)
    gch = _ch().CH.build(g, hop_limit=5, max_candidates_per_vertex=cmax)
    assert_same_hierarchy(gch, och)
    core = int((och.level == och.rounds).sum())
    assert core > 0 and gch.stats()["core_vertices"] == core
    assert gch.query_config()[4] == 0  # no delta-stepping levels by default with a core
    s, t = I.random_pairs(g.n, 3000, seed=92)
    d = assert_same_queries(gch, och, s, t)
    assert np.array_equal(d, O.dijkstra_pairs(g, s, t))
    for cfg in _ch().QUERY_CONFIGS:
        gch.set_query_config(*cfg)
        assert np.array_equal(gch.query(s, t), d), cfg


def test_learned_priority_with_a_core():
    g = I.random_digraph(400, 2000, 1, 30, seed=93)
    w = _ch().mlp_init(5)
    gch = _ch().CH.build(g, hop_limit=5, mlp_weights=w, trace=True, max_candidates_per_vertex=16)
    tr = gch.export_trace()
    assert tr["rows"].shape[0] == gch.stats()["trace_rows"]
    och = O.build_ch(g, 5, replay=(tr["rows"][:, 0], tr["rows"][:, 1], tr["prio"]), cmax=16)
    assert_same_hierarchy(gch, och)
    # trace rows are those of eligible rescorings only
    ot = O.build_ch(g, 5, trace=True, cmax=16)
    plain = _ch().CH.build(g, hop_limit=5, trace=True, max_candidates_per_vertex=16)
    assert np.array_equal(plain.export_trace()["rows"], ot.trace)
    s, t = I.random_pairs(g.n, 3000, seed=94)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


def test_build_autotune_keeps_an_oracle_equal_hierarchy():
    """The build autotuner picks a hop limit and a witness routing threshold;
    the hierarchy it keeps equals the oracle's at the chosen hop limit, and
    the routing threshold changes no result."""
    g = I.geometric_knn_graph(20_000, seed=95)
    gch, rows, k = _ch().CH.build_autotune(g, hop_limits=(2, 5), route_degs=(16, 64, 256),
                                           sample=4096, queries_per_build=1e5)
    assert len(rows) == 6 and 0 <= k < 6
    assert all(r["build_ms"] > 0 and r["query_ms"] > 0 for r in rows)
    assert rows[k]["cost"] == min(r["cost"] for r in rows)
    for i in (0, 3):  # same hop limit, other thresholds: the same hierarchy
        assert rows[i]["shortcuts"] == rows[i + 1]["shortcuts"] == rows[i + 2]["shortcuts"]
    och = O.build_ch(g, rows[k]["hop_limit"])
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 2000, seed=96)
    assert np.array_equal(gch.query(s, t), och.query(s, t))


def test_build_autotune_on_rmat_with_a_core():
    g = I.rmat_graph(scale=12, nsamples=1 << 15, wmax=1000, seed=91)
    gch, rows, k = _ch().CH.build_autotune(g, hop_limits=(1, 3, 5), route_degs=(64,), sample=2048,
                                           queries_per_build=1e5, max_candidates_per_vertex=16)
    och = O.build_ch(g, rows[k]["hop_limit"], cmax=16)
    assert_same_hierarchy(gch, och)
    assert rows[k]["core_vertices"] == int((och.level == och.rounds).sum())


# ---------------------------------------------------------------------------
# Witness ball bound (θ)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ball", [1, 3, 10, 200])
@pytest.mark.parametrize("name,g", FAMILIES[:6], ids=[n for n, _ in FAMILIES[:6]])
def test_ball_bound_matches_oracle(name, g, ball):
    och = O.build_ch(g, 5, ball=ball)
    gch = _ch().CH.build(g, hop_limit=5, witness_ball_limit=ball)
    assert_same_hierarchy(gch, och)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    s, t = s.ravel().astype(np.uint32), t.ravel().astype(np.uint32)
    d = assert_same_queries(gch, och, s, t)
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


@pytest.mark.parametrize("ball", [600])
def test_ball_bound_on_the_global_memory_tiers(ball):
    # dense random digraph: balls outgrow both shared-memory tiers
    g = I.random_digraph(1500, 9000, 1, 1000, seed=97, allow_loops=False)
    och = O.build_ch(g, 4, ball=ball)
    gch = _ch().CH.build(g, hop_limit=4, witness_ball_limit=ball)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 3000, seed=98)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


def _hub_graph():
    # two hubs of out-degree 1500 (above the shared-memory tiers' source
    # bound) on a sparse random digraph: their searches go straight to the
    # global-memory tier and use its direct-edge table
    base = I.random_digraph(3000, 9000, 1, 50, seed=99)
    src, dst, w = base.edges()
    rng = np.random.default_rng(100)
    hs, hd, hw = [], [], []
    for hub in (0, 1):
        nb = rng.choice(np.arange(2, 3000), 1500, replace=False)
        hs += [hub] * 1500 + list(nb)
        hd += list(nb) + [hub] * 1500
        hw += list(rng.integers(1, 50, 3000))
    return I.csr_from_edges(3000, np.concatenate([src, hs]), np.concatenate([dst, hd]),
                            np.concatenate([w, hw]))


@pytest.mark.parametrize("cmax,ball", [(64, None), (64, 300)])
def test_hub_sources_use_the_global_memory_tier(cmax, ball):
    g = _hub_graph()
    och = O.build_ch(g, 3, cmax=O.CMAX_ALL if cmax is None else cmax,
                     ball=O.CMAX_ALL if ball is None else ball)
    gch = _ch().CH.build(g, hop_limit=3, max_candidates_per_vertex=cmax, witness_ball_limit=ball)
    assert gch.stats()["witness_dense"] > 0
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 3000, seed=101)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


# ---------------------------------------------------------------------------
# Core distance table (ch_core_table): queries join their upward searches
# through the core's all-pairs distances instead of searching inside it
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("cmax", [0, 4, 12])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_core_table_answers_every_pair(name, g, cmax):
    gch = _ch().CH.build(g, hop_limit=5, max_candidates_per_vertex=cmax)
    gch.core_table()
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    s, t = s.ravel().astype(np.uint32), t.ravel().astype(np.uint32)
    truth = all_pairs_truth(g)
    d = gch.query(s, t)
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), truth)
    for cfg in _ch().QUERY_CONFIGS:
        gch.set_query_config(*cfg)
        assert np.array_equal(gch.query(s, t).astype(np.uint64).reshape(g.n, g.n), truth), cfg


@pytest.mark.parametrize("cmax", [16, 256])
def test_core_table_on_rmat(cmax):
    g = I.rmat_graph(scale=12, nsamples=1 << 15, wmax=1000, seed=91)
    och = O.build_ch(g, 5, cmax=cmax)
    core = np.nonzero(och.level == och.rounds)[0].astype(np.uint32)
    gch = _ch().CH.build(g, hop_limit=5, max_candidates_per_vertex=cmax)
    s, t = I.random_pairs(g.n, 3000, seed=92)
    _, full = gch.query(s, t, want_settled=True)
    gch.core_table()
    # between core vertices a query reads the table itself
    rng = np.random.default_rng(93)
    cs = core[rng.integers(0, core.size, 2000)]
    ct = core[rng.integers(0, core.size, 2000)]
    assert np.array_equal(gch.query(cs, ct), O.dijkstra_pairs(g, cs, ct))
    d, joined = gch.query(s, t, want_settled=True)
    assert np.array_equal(d, O.dijkstra_pairs(g, s, t))
    for cfg in _ch().QUERY_CONFIGS:
        gch.set_query_config(*cfg)
        assert np.array_equal(gch.query(s, t), d), cfg
    # the searches stop at the core: fewer labels than the search inside it
    assert joined.mean() < full.mean()


def test_core_table_byte_limit():
    g = I.rmat_graph(scale=10, nsamples=1 << 13, wmax=100, seed=94)
    gch = _ch().CH.build(g, hop_limit=3, max_candidates_per_vertex=16)
    core = gch.stats()["core_vertices"]
    assert core > 10
    with pytest.raises(_ch().CHError) as ei:
        gch.core_table(max_bytes=4 * core * core - 1)
    assert ei.value.code == _ch().CH_ERANGE
    s, t = I.random_pairs(g.n, 2000, seed=95)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))  # no table: the full search
    gch.core_table(max_bytes=4 * core * core)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))
