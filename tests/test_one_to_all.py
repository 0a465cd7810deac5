"""One-to-all distances on the GPU (ch_one_to_all, the PHAST sweeps) against
the oracle's one-to-all, which is pinned to scipy's all-pairs Dijkstra in
test_witness_modes.py: every row bit for bit, with and without a core, for
ragged source batches (the kernel runs 64 sources at a time), on a loaded
hierarchy, and with an out-of-range source."""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import all_pairs_truth, small_families

pytestmark = pytest.mark.gpu


def _ch():
    from paper_2412_18008_gb300 import ch
    return ch


def _run(h, src):
    import torch
    s = torch.from_numpy(np.ascontiguousarray(src, np.uint32).view(np.int32)).cuda()
    out = h.one_to_all(s)
    torch.cuda.synchronize()
    h.query_status()
    return out.cpu().numpy().view(np.uint32)


FAMILIES = small_families()


@pytest.mark.parametrize("cmax", [None, 4, 0])
@pytest.mark.parametrize("name,g", FAMILIES, ids=[n for n, _ in FAMILIES])
def test_small_families_all_sources(name, g, cmax):
    h = _ch().CH.build(g, hop_limit=5, max_candidates_per_vertex=cmax)
    got = _run(h, np.arange(g.n))
    assert np.array_equal(got.astype(np.uint64), all_pairs_truth(g))
    och = O.build_ch(g, 5, cmax=O.CMAX_ALL if cmax is None else cmax)
    assert np.array_equal(got, och.one_to_all(np.arange(g.n)))


@pytest.mark.parametrize("k", [1, 15, 16, 17, 63, 64, 65, 150])
def test_geometric_ragged_batches(k):
    g = I.geometric_knn_graph(20_000, seed=131)
    h = _ch().CH.build(g, hop_limit=5)
    src = np.random.default_rng(k).integers(0, g.n, k).astype(np.uint32)
    got = _run(h, src)
    assert got.shape == (k, g.n)
    och = O.build_ch(g, 5)
    assert np.array_equal(got, och.one_to_all(src))


def test_rmat_with_a_core_and_a_loaded_hierarchy(tmp_path):
    g = I.rmat_graph(scale=12, nsamples=1 << 15, wmax=1000, seed=91)
    h = _ch().CH.build(g, hop_limit=5, max_candidates_per_vertex=16)
    assert h.stats()["core_vertices"] > 0
    src = np.array([0, 1, 17, g.n - 1, g.n // 2], np.uint32)
    got = _run(h, src)
    for i, s in enumerate(src.tolist()):
        assert np.array_equal(got[i], O.dijkstra(g, s))
    path = str(tmp_path / "h.gbch")
    h.save(path)
    assert np.array_equal(_run(_ch().CH.load(path), src), got)


def test_out_of_range_source_and_empty_batch():
    import torch
    ch = _ch()
    g = I.grid_graph(8, 8, 0.1, 1, 20, seed=3)
    h = ch.CH.build(g, hop_limit=5)
    s = torch.tensor([0, g.n], dtype=torch.int32, device="cuda")
    out = h.one_to_all(s)
    torch.cuda.synchronize()
    with pytest.raises(ch.CHError) as ei:
        h.query_status()
    assert ei.value.code == ch.CH_EINVAL
    assert np.array_equal(out[0].cpu().numpy().view(np.uint32), O.dijkstra(g, 0))
    assert (out[1].cpu().numpy().view(np.uint32) == 0xFFFFFFFF).all()
    assert h.one_to_all(torch.zeros(0, dtype=torch.int32, device="cuda")).shape == (0, g.n)
