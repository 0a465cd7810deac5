"""Host-side logic of the Python binding (no GPU): closing a hierarchy first
stops its servers and frees its captured query graphs, whose device work
reads the hierarchy's memory, and a server that fails to stop leaves the
hierarchy's memory allocated; the build autotuner keeps the cheapest build
over its level-work values and frees the others. The library is replaced by
recorders."""
import pytest

from paper_2412_18008_gb300 import ch


class _Recorder:
    def __init__(self, stop_rc=0):
        self.calls = []
        self.stop_rc = stop_rc

    def ch_free(self, h):
        self.calls.append(("free", h))

    def ch_server_stop(self, h):
        self.calls.append(("server_stop", h))
        return self.stop_rc

    def ch_query_graph_free(self, h):
        self.calls.append(("graph_free", h))

    def ch_last_error(self):
        return b"server kernel did not finish within its bounded wait"


def _fixture(monkeypatch, stop_rc=0):
    rec = _Recorder(stop_rc)
    monkeypatch.setattr(ch, "load", lambda *a, **k: rec)
    monkeypatch.setattr(ch, "_lib", rec)
    h = ch.CH("hier")
    sv = ch.Server.__new__(ch.Server)
    sv._ch, sv._h = h, "server"
    h._deps.add(sv)
    g = ch.QueryGraph("graph", (), h)
    h._deps.add(g)
    return rec, h, sv, g


def test_close_ends_dependents_before_freeing(monkeypatch):
    rec, h, sv, g = _fixture(monkeypatch)
    h.close()
    assert rec.calls[-1] == ("free", "hier")
    assert set(rec.calls[:-1]) == {("server_stop", "server"), ("graph_free", "graph")}
    h.close()  # idempotent
    sv.stop()
    g.close()
    assert len(rec.calls) == 3


def test_server_that_does_not_stop_leaves_the_hierarchy_allocated(monkeypatch):
    rec, h, sv, g = _fixture(monkeypatch, stop_rc=ch.CH_ETIMEOUT)
    with pytest.raises(ch.CHError):
        h.close()
    h.close()
    del h
    assert ("free", "hier") not in rec.calls


class _TuneRecorder:
    """Stands in for ch_build_autotune: each call fills its rows with the
    next costs and names the cheapest row as chosen."""

    def __init__(self, costs_per_call):
        self.costs = list(costs_per_call)
        self.params = []
        self.freed = []
        self.calls = 0

    def ch_default_params(self, p):
        pass

    def ch_build_autotune(self, g, p, hl, nhl, rd, nrd, sample, qpb, h_out, rows, chosen):
        import ctypes as C
        prm = C.cast(p, C.POINTER(ch.ParamsT)).contents
        self.params.append(prm.witness_level_work)
        costs = self.costs[self.calls]
        self.calls += 1
        for i, c in enumerate(costs):
            rows[i].cost = c
            rows[i].hop_limit = i
        chosen._obj.value = min(range(len(costs)), key=lambda i: costs[i])
        C.cast(h_out, C.POINTER(C.c_void_p)).contents.value = 1000 + self.calls
        return 0

    def ch_free(self, h):
        self.freed.append(h)

    def ch_last_error(self):
        return b""


def test_build_autotune_keeps_the_cheapest_over_level_work_values(monkeypatch):
    from paper_2412_18008_gb300 import inputs as I
    rec = _TuneRecorder([[5.0, 4.0], [3.0, 6.0], [7.0, 8.0]])
    monkeypatch.setattr(ch, "load", lambda *a, **k: rec)
    monkeypatch.setattr(ch, "_lib", rec)
    g = I.grid_graph(4, 4, 0.0, 1, 5, seed=1)
    h, rows, k = ch.CH.build_autotune(g, hop_limits=(2, 5), route_degs=(64,), level_works=(None, 512, 64))
    assert rec.params == [0, 512, 64]
    assert len(rows) == 6 and [r["level_work"] for r in rows] == [None, None, 512, 512, 64, 64]
    assert k == 2 and rows[k]["cost"] == 3.0  # the second call's first row
    assert h._h.value == 1002
    assert sorted(x.value for x in rec.freed) == [1001, 1003]  # the others were freed
    h.close()  # while the stand-in is installed: the handle is not a real one
    # one value (the default) is one call, as before
    rec2 = _TuneRecorder([[2.0, 1.0]])
    monkeypatch.setattr(ch, "load", lambda *a, **k: rec2)
    monkeypatch.setattr(ch, "_lib", rec2)
    h2, rows2, k2 = ch.CH.build_autotune(g, hop_limits=(2, 5), route_degs=(64,))
    assert rec2.calls == 1 and k2 == 1 and rows2[1]["level_work"] is None and h2._h.value == 1001
    h2.close()


def test_device_entry_points_reject_host_arrays():
    import numpy as np
    h = ch.CH.__new__(ch.CH)
    h._h = None
    with pytest.raises(ValueError):
        h.one_to_all(np.zeros(3, np.uint32))
    with pytest.raises(ValueError):
        h.query_one_to_many(0, np.zeros(3, np.uint32))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        h.one_to_all(torch.zeros(3, dtype=torch.int32))  # a CPU tensor
    with pytest.raises(ValueError):
        h.one_to_all(torch.zeros(3, dtype=torch.int64))
