"""Query kernel configurations, the autotuner, the work counters and CUDA
graph replay: each is performance-only, so every answer must equal the
oracle's (and Dijkstra's) and the exhaustive search-space sizes must not
depend on the configuration."""
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


@pytest.fixture(scope="module")
def geo():
    g = I.geometric_knn_graph(40_000, seed=81)
    return g, _ch().CH.build(g, hop_limit=5), O.build_ch(g, 5)


# every fixed configuration, then delta-stepping from a bucket width of one
# weight unit (nearly one label value per level: the most deferral) to one
# far above the labels (no deferral), in both table tiers and block sizes
DELTA_CASES = [(1, 256, 1, 1, d) for d in (1, 3, 64, 1000, 1 << 30)] + [(1, 128, 0, 1, d) for d in (1, 50)]


@pytest.mark.parametrize("cfg", [(lay, thr, sf, 0, 0) for sf in (0, 1) for lay in (0, 1) for thr in (128, 256)]
                         + [(1, thr, sf, 1, 0) for sf in (0, 1) for thr in (128, 256)] + DELTA_CASES)
def test_every_configuration_gives_the_oracle_answers(geo, cfg):
    g, gch, och = geo
    gch.set_query_config(*cfg)
    assert gch.query_config() == cfg
    s, t = I.random_pairs(g.n, 20_000, seed=82)
    d, st = gch.query(s, t, want_settled=True)
    od, ost = och.query(s, t, want_settled=True)
    assert np.array_equal(d, od)
    assert np.array_equal(st.astype(np.uint64), ost)  # exhaustive: same labelled set
    assert np.array_equal(gch.query(s, t), od)  # pruned
    idx = np.arange(0, s.size, 50)
    assert np.array_equal(d[idx], O.dijkstra_pairs(g, s[idx], t[idx]))


def test_configurations_on_a_dense_random_digraph():
    g = I.random_digraph(1500, 9000, 1, 1000, seed=83)
    gch = _ch().CH.build(g, hop_limit=4)
    och = O.build_ch(g, 4)
    s, t = I.random_pairs(g.n, 5000, seed=84)
    want = och.query(s, t)
    for cfg in _ch().QUERY_CONFIGS + tuple(DELTA_CASES):
        gch.set_query_config(*cfg)
        assert np.array_equal(gch.query(s, t), want), cfg


def test_invalid_configuration_is_rejected(geo):
    ch = _ch()
    _, gch, _ = geo
    before = gch.query_config()
    for cfg in ((2, 256, 0, 0, 0), (0, 64, 0, 0, 0), (1, 512, 0, 0, 0), (1, 256, 2, 0, 0), (0, 256, 0, 1, 0),
                (1, 256, 0, 2, 0), (0, 256, 0, 0, 5), (1, 256, 1, 0, 5), (1, 256, 1, 1, 0xFFFFFFFF)):
        with pytest.raises(ch.CHError) as ei:
            gch.set_query_config(*cfg)
        assert ei.value.code == ch.CH_EINVAL
    assert gch.query_config() == before


def test_autotune_keeps_a_configuration_and_the_answers(geo):
    g, gch, och = geo
    cfg, ms = gch.autotune_queries(sample=8192, seed=3)
    assert ms.size == len(_ch().QUERY_CONFIGS) and (ms > 0).all()
    assert gch.query_config() == cfg
    # the fastest candidate was kept; its delta is its multiple of the
    # hierarchy's weight scale
    best = _ch().QUERY_CONFIGS[int(ms.argmin())]
    assert cfg[:4] == best[:4] and (cfg[4] == 0) == (best[4] == 0)
    if best[4]:
        assert cfg[4] % best[4] == 0
    s, t = I.random_pairs(g.n, 5000, seed=85)
    assert np.array_equal(gch.query(s, t), och.query(s, t))


def test_work_counters(geo):
    torch = _torch()
    g, gch, och = geo
    gch.query_work()  # clear
    s, t = I.random_pairs(g.n, 4000, seed=86)
    ds = torch.from_numpy(s.view(np.int32)).cuda()
    dt = torch.from_numpy(t.view(np.int32)).cuda()
    gch.query(ds, dt, want_settled=True)
    exp, edges = gch.query_work()
    # exhaustive searches: every labelled vertex is expanded at least once,
    # except the labelled vertices with no upward edge in that direction
    _, st = och.query(s, t, want_settled=True)
    assert 0 < exp and edges >= exp // 2
    assert exp <= 64 * int(st.sum())
    assert gch.query_work() == (0, 0)  # cleared by the read


@pytest.mark.parametrize("cfg", [(1, 256, 0, 0, 0), (1, 256, 1, 0, 0), (1, 256, 1, 1, 0), (1, 256, 1, 1, 40)])
def test_graph_replay_matches_batch_calls(geo, cfg):
    torch = _torch()
    g, gch, och = geo
    gch.set_query_config(*cfg)
    k = 3000
    s1, t1 = I.random_pairs(g.n, k, seed=87)
    s2, t2 = I.random_pairs(g.n, k, seed=88)
    ds = torch.from_numpy(s1.view(np.int32)).cuda()
    dt = torch.from_numpy(t1.view(np.int32)).cuda()
    out = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with gch.query_graph(ds, dt, out) as qg:
        qg.launch(stream)
        stream.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), och.query(s1, t1))
        # new inputs in the same buffers: the replay answers them
        ds.copy_(torch.from_numpy(s2.view(np.int32)))
        dt.copy_(torch.from_numpy(t2.view(np.int32)))
        torch.cuda.synchronize()
        for _ in range(3):
            qg.launch(stream)
        stream.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), och.query(s2, t2))
    gch.query_status()


def test_empty_graph_capture(geo):
    torch = _torch()
    _, gch, _ = geo
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    with gch.query_graph(e, e, e) as qg:
        qg.launch()
    torch.cuda.synchronize()
