"""Composite priority (CH_PRIO_COMPOSITE: 4 * edge difference + (|N_in| +
|N_out|) + 8 * hierarchy depth, clamped to +-2^30; the hop-distance term of
the paper's list is not kept). The oracle's priorities are pinned to the
definition through its trace features (themselves pinned in
test_trace_pins.py); the GPU hierarchy equals the oracle's bit for bit and
answers exactly."""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import all_pairs_truth, small_families


def composite_of_row(row):
    """The composite score from a trace row (round, u, S, |N_in|, |N_out|, |N|,
    ED, cn, depth, ...)."""
    p = 4 * int(row[2 + 4]) + int(row[2 + 1]) + int(row[2 + 2]) + 8 * int(row[2 + 6])
    return max(-(1 << 30), min(1 << 30, p))


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph0", "grid8", "geo150", "rmat8", "chain30")])
def test_oracle_priorities_follow_the_definition(name, g):
    och = O.build_ch(g, 5, composite=True, trace=True)
    # the priority a vertex is contracted with is the composite of its last
    # rescoring (trace rows are in round order)
    last = {}
    for row in och.trace:
        last[int(row[1])] = row
    for u, row in last.items():
        assert och.priority[u] == composite_of_row(row), (name, u)
    # any order yields exact distances
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = och.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


def test_composite_differs_from_edge_difference_and_is_shallower():
    g = I.geometric_knn_graph(8_000, seed=61)
    a, b = O.build_ch(g, 5), O.build_ch(g, 5, composite=True)
    assert not np.array_equal(a.level, b.level)
    assert b.stats.shape[0] < a.stats.shape[0]  # fewer rounds: the depth term flattens
    s, t = I.random_pairs(g.n, 2000, seed=62)
    da, sa = a.query(s, t, want_settled=True)
    db, sb = b.query(s, t, want_settled=True)
    assert np.array_equal(da, db)
    assert sb.mean() < sa.mean()


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

@pytest.mark.gpu
@pytest.mark.parametrize("name,g", small_families())
def test_gpu_equals_oracle_on_small_families(name, g):
    from paper_2412_18008_gb300 import ch
    from tests.test_gpu_parity import assert_same_hierarchy
    och = O.build_ch(g, 5, composite=True)
    gch = ch.CH.build(g, hop_limit=5, composite=True)
    assert_same_hierarchy(gch, och)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = gch.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


@pytest.mark.gpu
def test_gpu_equals_oracle_on_a_geometric_graph_with_trace():
    from paper_2412_18008_gb300 import ch
    from tests.test_gpu_parity import assert_same_hierarchy
    g = I.geometric_knn_graph(30_000, seed=63)
    och = O.build_ch(g, 5, composite=True, trace=True)
    gch = ch.CH.build(g, hop_limit=5, composite=True, trace=True)
    assert_same_hierarchy(gch, och)
    tr = gch.export_trace()
    assert np.array_equal(tr["rows"], och.trace)
    assert [composite_of_row(r) for r in tr["rows"]] == tr["prio"].tolist()
    s, t = I.random_pairs(g.n, 4000, seed=64)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))


def test_binding_marshals_the_priority_modes():
    from paper_2412_18008_gb300 import ch
    g = I.grid_graph(4, 4, 0.0, 1, 5, seed=1)
    args = (g, None, None, None, None, 5, ch.CH_TIE_HASHED, 0, None)
    _, p, _ = ch.CH._marshal(*args, None, False, None, 0, composite=True)
    assert p.priority == ch.CH_PRIO_COMPOSITE and not p.mlp_weights
    _, p, keep = ch.CH._marshal(*args, ch.mlp_init(1), False, None, 0)
    assert p.priority == ch.CH_PRIO_LEARNED and p.mlp_weights
    _, p, _ = ch.CH._marshal(*args, None, False, None, 0)
    assert p.priority == ch.CH_PRIO_EDGE_DIFF
    with pytest.raises(ValueError):
        ch.CH._marshal(*args, ch.mlp_init(1), False, None, 0, composite=True)
