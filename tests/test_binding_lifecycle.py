"""Host-side lifetime rules of the Python binding (no GPU): closing a
hierarchy first stops its servers and frees its captured query graphs, whose
device work reads the hierarchy's memory, and a server that fails to stop
leaves the hierarchy's memory allocated. The library is replaced by a
recorder."""
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
