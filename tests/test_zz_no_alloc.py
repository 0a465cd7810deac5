"""ch_query_batch_static: the query entry point that allocates nothing.

It serves callers that must not allocate device memory (a serving thread
that may not block on an allocation's implicit device synchronisation, or a
process whose device memory another allocator has reserved). Its scratch is
a static device array shared by every call, so this file checks that it
gives exactly the answers of the regular entry point, on two calls in a row
(the second call must not be affected by what the first left in the
scratch), and that it refuses batches above its stated maximum. A second
case leaves a core larger than the shared-memory table, so that every query
that reaches it overflows into the scratch's overflow list and is finished by
the global-memory kernel. Collected last on purpose; it runs alone or after
the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CH_STATIC_QUERY_MAX = 1 << 18


def _entry_point(lib):
    fn = lib.ch_query_batch_static
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return fn


def _two_calls(h, static_query, lib, g, sizes, seed):
    """Runs both entry points on the same batches, two calls in a row, and
    yields each call's pairs and static-scratch answers."""
    from paper_2412_18008_gb300 import inputs as I

    stream = torch.cuda.Stream()
    for call, k in enumerate(sizes):
        s, t = I.random_pairs(g.n, k, seed=seed + call)
        with torch.cuda.stream(stream):
            ds = torch.from_numpy(s.view(np.int32)).cuda()
            dt = torch.from_numpy(t.view(np.int32)).cuda()
            ref = h.query(ds, dt, stream=stream)
            out = torch.full((k,), -7, dtype=torch.int32, device="cuda")
            rc = static_query(h._h, ds.data_ptr(), dt.data_ptr(), k, out.data_ptr(),
                              stream.cuda_stream)
        assert rc == 0, lib.ch_last_error()
        stream.synchronize()
        h.query_status(stream)
        assert torch.equal(out, ref), f"call {call}: answers differ from ch_query_batch"
        yield s, t, out.cpu().numpy().view(np.uint32)


def test_overflowing_queries_match_regular_entry_point():
    """A core of more than 4096 vertices: the searches outgrow the block
    tables, so the answers come through the overflow list."""
    import oracle as O
    from paper_2412_18008_gb300 import ch, inputs as I

    lib = ch.load()
    static_query = _entry_point(lib)
    g = I.geometric_knn_graph(12_000, seed=43)
    # Cmax = 1 keeps every vertex with |N_in| * |N_out| > 1 in the core
    h = ch.CH.build(g, hop_limit=5, max_candidates_per_vertex=1)
    assert h.stats()["core_vertices"] > 4096
    for s, t, got in _two_calls(h, static_query, lib, g, (3000, 2001), seed=44):
        idx = np.arange(0, s.size, 29)
        assert np.array_equal(got[idx], O.dijkstra_pairs(g, s[idx], t[idx]))
    h.close()


def test_static_scratch_queries_match_regular_entry_point():
    from paper_2412_18008_gb300 import ch, inputs as I

    lib = ch.load()
    static_query = _entry_point(lib)
    g = I.geometric_knn_graph(80_000, seed=41)
    h = ch.CH.build(g, hop_limit=5)
    for _ in _two_calls(h, static_query, lib, g, (CH_STATIC_QUERY_MAX, 70_001), seed=42):
        pass
    # a batch above the stated maximum is refused, and nothing is written
    big = CH_STATIC_QUERY_MAX + 1
    ds = torch.zeros(big, dtype=torch.int32, device="cuda")
    out = torch.full((big,), -7, dtype=torch.int32, device="cuda")
    rc = static_query(h._h, ds.data_ptr(), ds.data_ptr(), big, out.data_ptr(), None)
    assert rc == ch.CH_ERANGE
    torch.cuda.synchronize()
    assert bool((out == -7).all())
    h.close()
