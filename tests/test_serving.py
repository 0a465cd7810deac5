"""Query server (continuous batching): every answer equals the batch
query's answer for the same pair, alone or in a mix of overlapping
requests; admission by memory; bounded idle wait."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ch():
    from paper_2412_18008_gb300 import ch
    return ch


@pytest.fixture(scope="module")
def built():
    g = I.geometric_knn_graph(30_000, seed=71)
    return g, _ch().CH.build(g, hop_limit=5)


def _expected(gch, src, ks, targets):
    return gch.query(np.repeat(src, ks), targets)


def test_mixed_stream_answers_equal_batch_answers(built):
    g, gch = built
    ch = _ch()
    src, ks, targets = I.request_mix(g.n, 3000, seed=72)
    arr = I.poisson_arrivals(src.size, rate_per_s=200_000, seed=73)
    with ch.Server(gch, blocks=96, ring=2048, pool=1 << 20, idle_ms=5000) as sv:
        ans, lat, svc = sv.replay(src, ks, targets, arr)
    assert np.array_equal(ans, _expected(gch, src, ks, targets))
    assert (lat > 0).all() and (svc > 0).all()
    # against Dijkstra on a sample of the pairs
    flat_s = np.repeat(src, ks)
    idx = np.arange(0, targets.size, 97)
    assert np.array_equal(ans[idx], O.dijkstra_pairs(g, flat_s[idx], targets[idx]))


def test_same_answer_alone_and_in_the_mix(built):
    g, gch = built
    ch = _ch()
    src, ks, targets = I.request_mix(g.n, 400, seed=74)
    toff = np.concatenate([[0], np.cumsum(ks.astype(np.int64))[:-1]]).astype(np.int64)
    with ch.Server(gch, blocks=32, ring=1024, pool=1 << 18) as sv:
        mix, _, _ = sv.replay(src, ks, targets, np.zeros(src.size, np.uint64))  # all at once
        for i in range(0, src.size, 37):  # alone: one request on an idle server
            a, b = int(toff[i]), int(toff[i]) + int(ks[i])
            tk = sv.submit(int(src[i]), targets[a:b])
            res = None
            t0 = time.time()
            while res is None and time.time() - t0 < 30:
                res = sv.poll(tk, int(ks[i]))
            if res is None:  # report the device loop's state with the failure
                try:
                    sv.stop()
                    why = "the loop then stopped cleanly"
                except ch.CHError as e:
                    why = f"stopping the loop failed: {e}"
                raise AssertionError(f"request {i} (k = {ks[i]}) not served in 30 s; {why}")
            assert np.array_equal(res, mix[a:b])


def test_admission_by_memory_and_ring(built):
    g, gch = built
    ch = _ch()
    src, ks, targets = I.request_mix(g.n, 600, seed=75, one_to_many=0.5)
    # a pool smaller than the sum of all targets and a short ring: requests
    # are admitted as earlier ones complete
    with ch.Server(gch, blocks=16, ring=64, pool=4096) as sv:
        ans, _, _ = sv.replay(src, ks, targets, np.zeros(src.size, np.uint64))
    assert np.array_equal(ans, _expected(gch, src, ks, targets))


def test_idle_limit_ends_the_loop(built):
    g, gch = built
    ch = _ch()
    sv = ch.Server(gch, blocks=8, ring=64, pool=4096, idle_ms=200)
    time.sleep(1.0)
    with pytest.raises(ch.CHError) as ei:
        for _ in range(200):  # the ring fills only if the loop were still serving
            sv.submit(0, [1])
    assert ei.value.code == ch.CH_ETIMEOUT
    sv.stop()
