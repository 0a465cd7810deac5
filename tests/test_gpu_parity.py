"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work, so the bar is bit-exact: levels, scores, ranks, the sorted
shortcut set, both CH edge sets, the per-round counters, every query
distance and every search-space size.
"""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import INF, all_pairs_truth, from_edges, golden_names, load_golden, small_families

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def ch_mod():
    from paper_2412_18008_gb300 import ch
    return ch


def gpu_build(g, H=5, tie=0, seed=0):
    return ch_mod().CH.build(g, hop_limit=H, tie_break=tie, tie_seed=seed)


def _sorted_rows(a, cols):
    a = np.asarray(a, dtype=np.uint64).reshape(-1, a.shape[1] if a.ndim == 2 else 1)
    if a.size == 0:
        return a
    return a[np.lexsort(tuple(a[:, c] for c in reversed(cols)))]


def assert_same_hierarchy(gch, och):
    ex = gch.export()
    assert np.array_equal(ex["level"], och.level), "levels differ"
    assert np.array_equal(ex["priority"], och.priority), "scores differ"
    assert np.array_equal(ex["rank"], och.rank), "ranks differ"
    assert np.array_equal(ex["shortcuts"].astype(np.uint64),
                          _sorted_rows(och.shortcuts, [0, 1, 2])), "shortcut sets differ"
    assert np.array_equal(ex["up"].astype(np.uint64), _sorted_rows(och.up, [0, 1])), "E_up differs"
    assert np.array_equal(ex["down"].astype(np.uint64), _sorted_rows(och.down, [1, 0])), "E_down differs"
    assert np.array_equal(gch.round_stats(), och.stats), "per-round counters differ"


def assert_same_queries(gch, och, s, t):
    d, st = gch.query(s, t, want_settled=True)
    od, ost = och.query(s, t, want_settled=True)
    assert np.array_equal(d, od)
    assert np.array_equal(st.astype(np.uint64), ost)
    return d


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", golden_names())
def test_golden_examples(name):
    spec = load_golden(name)
    tie = 1 if spec.get("tie_break") == "id" else 0
    g = ch_mod().CH.build(spec["graph"], hop_limit=spec["hop_limit"], tie_break=tie,
                          max_candidates_per_vertex=spec.get("cmax"),
                          witness_ball_limit=spec.get("ball"),
                          witness_memo_limit=spec.get("memo"),
                          witness_level_work=spec.get("level_work"),
                          witness_prune=bool(spec.get("prune")),
                          witness_settle_cap=spec.get("theta"),
                          composite=bool(spec.get("composite")))
    ex = g.export()
    assert ex["level"].tolist() == spec["expect_level"]
    assert ex["priority"].tolist() == spec["expect_priority"]
    assert ex["rank"].tolist() == spec["expect_rank"]
    assert sorted(map(tuple, ex["shortcuts"].tolist())) == sorted(spec["shortcuts"])
    for s, t, d in spec["queries"]:
        assert int(g.query(np.array([s]), np.array([t]))[0]) == d


@pytest.mark.parametrize("name,graph", small_families())
@pytest.mark.parametrize("H,tie", [(5, 0), (0, 0), (1, 1), (2, 0), (3, 1)])
def test_small_families(name, graph, H, tie):
    och = O.build_ch(graph, H, tie, tie_seed=17)
    gch = gpu_build(graph, H, tie, 17)
    assert_same_hierarchy(gch, och)
    s, t = np.meshgrid(np.arange(graph.n), np.arange(graph.n), indexing="ij")
    s, t = s.ravel().astype(np.uint32), t.ravel().astype(np.uint32)
    d = assert_same_queries(gch, och, s, t)
    assert np.array_equal(d.astype(np.uint64).reshape(graph.n, graph.n), all_pairs_truth(graph))


def test_grid_workload_full_parity():
    g, params = I.workload("grid64")
    och = O.build_ch(g, params["hop_limit"])
    gch = gpu_build(g, params["hop_limit"])
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 1000, seed=2)
    d = assert_same_queries(gch, och, s, t)
    assert np.array_equal(d, O.dijkstra_pairs(g, s, t))


@pytest.mark.parametrize("n,seed", [(20_000, 21), (150_000, 22)])
def test_geometric_full_parity(n, seed):
    g = I.geometric_knn_graph(n, seed=seed)
    och = O.build_ch(g, 5)
    gch = gpu_build(g, 5)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(n, 5000, seed=seed + 1)
    d = assert_same_queries(gch, och, s, t)
    assert np.array_equal(d[:300], O.dijkstra_pairs(g, s[:300], t[:300]))


def test_full_size_road_like_graph():
    """The 1M-vertex geometric workload, built in the configuration the
    benchmark times: the whole hierarchy is compared with the oracle's, and
    every answer of the 1M-query batch with the oracle's CH query (its
    threaded build, whose output equals the sequential one), sampled
    answers and search-space sizes also with Dijkstra and the sequential
    query."""
    g = I.geometric_knn_graph(1_000_000, seed=3)
    gch = gpu_build(g, 5)
    och = O.build_ch(g, 5, threads=True)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 1_000_000, seed=4)
    ds = torch.from_numpy(s.view(np.int32)).cuda()
    dt = torch.from_numpy(t.view(np.int32)).cuda()
    out, settled = gch.query(ds, dt, want_settled=True)
    torch.cuda.synchronize()
    gch.query_status()
    d = out.cpu().numpy().view(np.uint32)
    st = settled.cpu().numpy().view(np.uint32)
    assert np.array_equal(d, och.query(s, t)), "answers differ from the oracle's"
    idx = np.random.default_rng(0).choice(g.n, 4000, replace=False)
    od, ost = och.query(s[idx], t[idx], want_settled=True)
    assert np.array_equal(d[idx], od)
    assert np.array_equal(st[idx].astype(np.uint64), ost)
    assert np.array_equal(d[idx[:100]], O.dijkstra_pairs(g, s[idx[:100]], t[idx[:100]]))
    # properties that hold for every pair of the batch
    same = s == t
    assert (d[same] == 0).all()
    assert (st >= 2 - same).all()
    # the pruned searches the benchmark times, in both table tiers and both
    # layouts, answer every pair of the batch as the exhaustive ones do
    default = gch.query_config()
    assert default[:4] == (1, 256, 1, 1) and default[4] > 0
    for cfg in ((1, 256, 0, 0, 0), (1, 256, 1, 0, 0), (0, 256, 1, 0, 0), (1, 256, 1, 1, 0), default):
        gch.set_query_config(*cfg)
        dp = gch.query(ds, dt)
        torch.cuda.synchronize()
        gch.query_status()
        assert np.array_equal(dp.cpu().numpy().view(np.uint32), d), cfg


def test_dense_graph_exercises_global_memory_paths():
    # a random digraph of average out-degree 6 with weights up to 1000: its
    # 4-hop witness balls and its query search spaces outgrow the
    # shared-memory tables, so the global-memory kernels run too
    g = I.random_digraph(1500, 9000, 1, 1000, seed=5, allow_loops=False)
    och = O.build_ch(g, 4)
    gch = gpu_build(g, 4)
    assert gch.stats()["witness_fallback"] > 0
    assert_same_hierarchy(gch, och)
    qs, qt = I.random_pairs(g.n, 3000, seed=6)
    dd = assert_same_queries(gch, och, qs, qt)
    truth = all_pairs_truth(g)
    assert np.array_equal(dd.astype(np.uint64), truth[qs, qt])


def test_device_input_matches_host_input():
    g = I.geometric_knn_graph(30_000, seed=9)
    a = gpu_build(g, 5)
    off = torch.from_numpy(g.offsets.view(np.int64)).cuda()
    tgt = torch.from_numpy(g.targets.view(np.int32)).cuda()
    w = torch.from_numpy(g.weights.view(np.int32)).cuda()
    b = ch_mod().CH.build(n=g.n, offsets=off, targets=tgt, weights=w, hop_limit=5)
    ea, eb = a.export(), b.export()
    for k in ea:
        assert np.array_equal(ea[k], eb[k]), k


def test_deterministic_builds():
    g = I.geometric_knn_graph(50_000, seed=10)
    ea, eb = gpu_build(g).export(), gpu_build(g).export()
    for k in ea:
        assert np.array_equal(ea[k], eb[k]), k


def test_device_queries_match_host_queries():
    g = I.geometric_knn_graph(40_000, seed=11)
    gch = gpu_build(g)
    s, t = I.random_pairs(g.n, 100_000, seed=12)
    host = gch.query(s, t)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ds = torch.from_numpy(s.view(np.int32)).cuda()
        dt = torch.from_numpy(t.view(np.int32)).cuda()
        out = gch.query(ds, dt, stream=stream)
    stream.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), host)


def test_normalisation_of_loops_and_duplicates():
    g = I.random_digraph(300, 2000, 1, 5, seed=13)  # many parallel edges and loops
    och = O.build_ch(g, 5)
    gch = gpu_build(g, 5)
    assert gch.stats()["m_input"] == O.normalize(g)[1].size
    assert_same_hierarchy(gch, och)


def test_empty_isolated_and_trivial():
    ch = ch_mod()
    g0 = I.csr_from_edges(0, [], [], [])
    e = ch.CH.build(g0)
    assert e.stats()["rounds"] == 0
    g5 = I.csr_from_edges(5, [], [], [])
    c5 = ch.CH.build(g5)
    assert c5.export()["level"].tolist() == [0] * 5
    assert c5.query(np.array([0, 1], np.uint32), np.array([0, 2], np.uint32)).tolist() == [0, INF]
    g1 = from_edges(2, [(0, 1, 7)])
    c1 = ch.CH.build(g1)
    assert c1.query(np.array([0, 1]), np.array([1, 0])).tolist() == [7, INF]


def test_rejects_malformed_input():
    ch = ch_mod()
    bad_w = I.Graph(2, np.array([0, 1, 1], np.uint64), np.array([1], np.uint32),
                    np.array([0], np.uint32))
    bad_t = I.Graph(2, np.array([0, 1, 1], np.uint64), np.array([5], np.uint32),
                    np.array([1], np.uint32))
    bad_o = I.Graph(2, np.array([0, 2, 1], np.uint64), np.array([1, 0], np.uint32),
                    np.array([1, 1], np.uint32))
    inf_w = I.Graph(2, np.array([0, 1, 1], np.uint64), np.array([1], np.uint32),
                    np.array([0xFFFFFFFF], np.uint32))
    for g in (bad_w, bad_t, bad_o, inf_w):
        with pytest.raises(ch.CHError) as ei:
            ch.CH.build(g)
        assert ei.value.code == ch.CH_EINVAL
    good = ch.CH.build(from_edges(3, [(0, 1, 1), (1, 2, 1)]))
    with pytest.raises(ch.CHError) as ei:
        good.query(np.array([0, 7], np.uint32), np.array([1, 1], np.uint32))
    assert ei.value.code == ch.CH_EINVAL
    # the handle stays usable after a rejected batch
    assert good.query(np.array([0]), np.array([2])).tolist() == [2]


@pytest.mark.parametrize("H", [0, 1, 2, 4])
def test_hop_limits_on_road_like_graph(H):
    g = I.geometric_knn_graph(8_000, seed=14)
    och = O.build_ch(g, H)
    gch = gpu_build(g, H)
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 2000, seed=15)
    assert_same_queries(gch, och, s, t)


def test_id_tie_break_on_long_chain():
    g = I.chain_graph(3000, True, seed=16)
    och = O.build_ch(g, 5, O.TIE_ID)
    gch = gpu_build(g, 5, 1)
    assert_same_hierarchy(gch, och)


@pytest.mark.parametrize("which", ["geo", "grid", "digraph"])
def test_pruned_queries_match_exhaustive_and_oracle(which):
    # without search-space counts the query prunes relaxations that cannot
    # beat the best meeting sum so far; the answers must not change
    if which == "geo":
        g = I.geometric_knn_graph(60_000, seed=31)
    elif which == "grid":
        g, _ = I.workload("grid64")
    else:
        g = I.random_digraph(1200, 7000, 1, 1000, seed=32, allow_loops=False)
    gch = gpu_build(g, 5)
    s, t = I.random_pairs(g.n, 20_000, seed=33)
    pruned = gch.query(s, t)
    full, settled = gch.query(s, t, want_settled=True)
    assert np.array_equal(pruned, full)
    och = O.build_ch(g, 5)
    idx = np.arange(0, s.size, 7)
    assert np.array_equal(pruned[idx], och.query(s[idx], t[idx]))
