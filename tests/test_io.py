"""Saving and loading a built hierarchy, and one-to-many queries: a loaded
hierarchy exports and answers exactly as the saved one; malformed files are
rejected; one-to-many answers equal the batch query's for the same pairs."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ch():
    from paper_2412_18008_gb300 import ch
    return ch


def _torch():
    return pytest.importorskip("torch")


@pytest.mark.parametrize("cmax", [None, 8])
def test_save_load_roundtrip(tmp_path, cmax):
    g = I.geometric_knn_graph(20_000, seed=111) if cmax is None else I.random_digraph(400, 2000, 1, 30, seed=112)
    a = _ch().CH.build(g, hop_limit=5, max_candidates_per_vertex=cmax)
    path = str(tmp_path / "h.gbch")
    a.save(path)
    b = _ch().CH.load(path)
    ea, eb = a.export(), b.export()
    for key in ea:
        assert np.array_equal(ea[key], eb[key]), key
    assert np.array_equal(a.round_stats(), b.round_stats())
    sa, sb = a.stats(), b.stats()
    for key in ("n", "m_input", "rounds", "shortcuts", "up_edges", "down_edges", "core_vertices"):
        assert sa[key] == sb[key], key
    s, t = I.random_pairs(g.n, 5000, seed=113)
    da = a.query(s, t)
    assert np.array_equal(b.query(s, t), da)
    assert np.array_equal(da, O.dijkstra_pairs(g, s, t))


def test_load_rejects_malformed_files(tmp_path):
    ch = _ch()
    bad = tmp_path / "bad.gbch"
    bad.write_bytes(b"not a hierarchy at all")
    with pytest.raises(ch.CHError) as ei:
        ch.CH.load(str(bad))
    assert ei.value.code == ch.CH_EINVAL
    g = I.grid_graph(8, 8, 0.1, 1, 20, seed=3)
    good = tmp_path / "good.gbch"
    ch.CH.build(g, hop_limit=5).save(str(good))
    data = good.read_bytes()
    cut = tmp_path / "cut.gbch"
    cut.write_bytes(data[: len(data) // 2])
    with pytest.raises(ch.CHError) as ei:
        ch.CH.load(str(cut))
    assert ei.value.code == ch.CH_EINVAL
    with pytest.raises(ch.CHError):
        ch.CH.load(str(tmp_path / "missing.gbch"))


def test_save_load_empty_graph(tmp_path):
    ch = _ch()
    g = I.Graph(0, np.zeros(1, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    path = str(tmp_path / "empty.gbch")
    ch.CH.build(g, hop_limit=5).save(path)
    h = ch.CH.load(path)
    assert h.stats()["n"] == 0


def test_one_to_many_equals_batch():
    torch = _torch()
    ch = _ch()
    g = I.geometric_knn_graph(20_000, seed=114)
    h = ch.CH.build(g, hop_limit=5)
    rng = np.random.default_rng(115)
    for s, k in ((0, 1), (17, 1000), (g.n - 1, 4096)):
        t = rng.integers(0, g.n, k).astype(np.uint32)
        dt = torch.from_numpy(t.view(np.int32)).cuda()
        got = h.query_one_to_many(s, dt)
        torch.cuda.synchronize()
        h.query_status()
        want = h.query(np.full(k, s, np.uint32), t)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want)
    with pytest.raises(ch.CHError) as ei:
        h.query_one_to_many(g.n, torch.zeros(4, dtype=torch.int32, device="cuda"))
    assert ei.value.code == ch.CH_EINVAL
