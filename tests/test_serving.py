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


def test_idle_limit_ends_the_loop_and_a_request_resumes_it(built):
    g, gch = built
    ch = _ch()
    sv = ch.Server(gch, blocks=8, ring=64, pool=4096, idle_ms=200)
    time.sleep(1.0)
    assert not sv.running()  # ended at the idle limit, holding no work
    tk = sv.submit(5, [1, 2, 3])
    res = None
    t0 = time.time()
    while res is None and time.time() - t0 < 30:
        res = sv.poll(tk, 3)
    assert res is not None
    assert np.array_equal(res, gch.query(np.full(3, 5, np.uint32), np.array([1, 2, 3], np.uint32)))
    sv.stop()


def test_device_wide_synchronisation_during_serving(built):
    """A device-wide synchronisation (cudaDeviceSynchronize, or the cudaFree
    of another hierarchy) waits for the running loop, which ends at its idle
    limit; requests submitted afterwards are served by a new launch, and
    every answer equals the batch query's."""
    torch = pytest.importorskip("torch")
    g, gch = built
    ch = _ch()
    other = ch.CH.build(I.grid_graph(8, 8, 0.0, 1, 5, seed=3), hop_limit=5)
    src, ks, targets = I.request_mix(g.n, 60, seed=76, one_to_many=0.5)
    cut = int(ks[:30].sum())
    zeros = np.zeros(30, np.uint64)
    with ch.Server(gch, blocks=16, ring=64, pool=4096, idle_ms=300) as sv:
        first, _, _ = sv.replay(src[:30], ks[:30], targets[:cut], zeros)
        torch.cuda.synchronize()  # returns once the loop has ended
        assert not sv.running()
        other.close()
        rest, _, _ = sv.replay(src[30:], ks[30:], targets[cut:], zeros)
    assert np.array_equal(np.concatenate([first, rest]), _expected(gch, src, ks, targets))
