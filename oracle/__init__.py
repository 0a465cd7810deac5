"""CPU oracle for CH construction and CH s-t queries (test infrastructure).

The oracle is the reference the CUDA path is checked against: a plain,
sequential C++ implementation of the round algorithm (Alg. 2-6 of arXiv
2412.18008), of its postprocessing and of the bidirectional upward query
(Sec. 5), plus the plain definitions it is pinned with (hop-limited distance,
Dijkstra). Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library itself never
does, and there is no CPU fallback through it.

Functions here only marshal arguments; the arithmetic is in ``oracle.cpp``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_LIB_MT = os.path.join(_LIB_DIR, "liboracle_mt.so")  # -DORACLE_THREADS
INF = 0xFFFFFFFF

STAT_FIELDS = ("affected", "score_sources", "selected", "contract_sources",
               "candidates", "kept", "merged", "inserted", "vo_after", "eo_after")

TIE_HASHED = 0
TIE_ID = 1


def build(force: bool = False, threads: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``_build/liboracle.so`` (portable flags),
    or, with ``threads``, the -DORACLE_THREADS build ``liboracle_mt.so``."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    lib = _LIB_MT if threads else _LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    extra = ["-DORACLE_THREADS", "-pthread"] if threads else []
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", *extra,
                           "-o", tmp, _SRC])
    os.replace(tmp, lib)
    return lib


_libs = {}


def _load(threads: bool = False):
    """The sequential oracle library, or (threads) its -DORACLE_THREADS build."""
    if threads not in _libs:
        lib = C.CDLL(build(threads=threads))
        P = C.c_void_p
        u32, u64, i32 = C.c_uint32, C.c_uint64, C.c_int32
        lib.orc_build.argtypes = [u32, u64, P, P, P, u32, u32, u32, C.POINTER(P)]
        lib.orc_build.restype = C.c_int
        lib.orc_free.argtypes = [P]
        lib.orc_build2.argtypes = [u32, u64, P, P, P, u32, u32, u32, C.c_int, u64, P, P, P,
                                   u64, u64, u64, C.c_int, u64, u64, C.c_int, C.POINTER(P)]
        lib.orc_searches.argtypes = [P]
        lib.orc_searches.restype = u64
        lib.orc_witness_work.argtypes = [P]
        lib.orc_witness_work.restype = u64
        lib.orc_num_pruned.argtypes = [P]
        lib.orc_num_pruned.restype = u64
        lib.orc_get_pruned.argtypes = [P, P]
        lib.orc_get_pruned.restype = None
        lib.orc_one_to_all.argtypes = [P, u64, P, P]
        lib.orc_one_to_all.restype = C.c_int
        lib.orc_build2.restype = C.c_int
        lib.orc_num_trace.argtypes = [P]
        lib.orc_num_trace.restype = u64
        lib.orc_get_trace.argtypes = [P, P]
        lib.orc_get_trace.restype = None
        lib.orc_get_labels.argtypes = [P, P]
        lib.orc_get_labels.restype = None
        for name in ("orc_rounds",):
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = u32
        lib.orc_nstat.restype = u32
        for name in ("orc_num_shortcuts", "orc_num_up", "orc_num_down"):
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = u64
        for name in ("orc_get_stats", "orc_get_level", "orc_get_priority", "orc_get_rank",
                     "orc_get_shortcuts", "orc_get_up", "orc_get_down"):
            getattr(lib, name).argtypes = [P, P]
            getattr(lib, name).restype = None
        lib.orc_query_batch.argtypes = [P, u64, P, P, P, P]
        lib.orc_query_batch.restype = None
        lib.orc_round0_scores.argtypes = [u32, u64, P, P, P, u32, u64, P]
        lib.orc_normalize.argtypes = [u32, u64, P, P, P, P, P, P, P]
        lib.orc_hop_limited.argtypes = [u32, u64, P, P, P, u32, u32, P]
        lib.orc_dijkstra.argtypes = [u32, u64, P, P, P, u32, P]
        lib.orc_dijkstra_pairs.argtypes = [u32, u64, P, P, P, u64, P, P, P]
        for name in ("orc_round0_scores", "orc_normalize", "orc_hop_limited",
                     "orc_dijkstra", "orc_dijkstra_pairs"):
            getattr(lib, name).restype = C.c_int
        del i32
        _libs[threads] = lib
    return _libs[threads]


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def _graph_args(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.uint64)
    tgt = np.ascontiguousarray(g.targets, dtype=np.uint32)
    w = np.ascontiguousarray(g.weights, dtype=np.uint32)
    keep = (off, tgt, w)
    return (g.n, int(tgt.size), _p(off), _p(tgt), _p(w)), keep


@dataclass
class OracleCH:
    """Everything the oracle's build produces, as numpy arrays."""
    n: int
    hop_limit: int
    level: np.ndarray          # uint32[n]: round in which the vertex was contracted
    priority: np.ndarray       # int32[n]: score at contraction
    rank: np.ndarray           # uint32[n]: position in (level, score, id) order
    shortcuts: np.ndarray      # uint32[k, 5]: (round, v1, v2, w, via), inserted order
    up: np.ndarray             # uint32[a, 3]: (u, x, w) upward edges
    down: np.ndarray           # uint32[b, 3]: (x, u, w) downward edges
    stats: np.ndarray          # uint64[rounds, len(STAT_FIELDS)]
    _handle: C.c_void_p = field(default=None, repr=False)
    _threads: bool = field(default=False, repr=False)  # which library owns the handle

    @property
    def rounds(self) -> int:
        return int(self.stats.shape[0])

    def query(self, s, t, want_settled: bool = False):
        """Bidirectional upward queries for arrays of sources and targets."""
        s = np.ascontiguousarray(s, dtype=np.uint32)
        t = np.ascontiguousarray(t, dtype=np.uint32)
        if s.shape != t.shape:
            raise ValueError("sources and targets differ in length")
        if s.size and (s.max() >= self.n or t.max() >= self.n):
            raise ValueError("query vertex out of range")
        out = np.empty(s.size, dtype=np.uint32)
        settled = np.empty(s.size, dtype=np.uint64)
        if s.size:
            _load(self._threads).orc_query_batch(self._handle, s.size, _p(s), _p(t), _p(out),
                                                 _p(settled))
        return (out, settled) if want_settled else out

    def one_to_all(self, sources) -> np.ndarray:
        """Distances from each source to every vertex (upward search, then a
        downward sweep in descending rank), uint32[len(sources), n]."""
        s = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.uint32)
        out = np.empty((s.size, self.n), dtype=np.uint32)
        if s.size and self.n:
            if _load(self._threads).orc_one_to_all(self._handle, s.size, _p(s), _p(out)) != 0:
                raise ValueError("source vertex out of range")
        elif s.size:
            raise ValueError("source vertex out of range")
        return out

    def close(self):
        if self._handle:
            _load(self._threads).orc_free(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CMAX_ALL = (1 << 64) - 1


def build_ch(g, hop_limit: int = 5, tie_break: int = TIE_HASHED, tie_seed: int = 0,
             trace: bool = False, replay=None, cmax: int = CMAX_ALL,
             ball: int = CMAX_ALL, threads: bool = False, theta: int = 0,
             prune: bool = False, memo: int = 0, level_work: int = CMAX_ALL,
             composite: bool = False) -> OracleCH:
    """Run the oracle's round algorithm on graph ``g`` (see ``oracle.cpp``).

    ``trace`` records the learned-priority features of every rescoring
    (``OracleCH.trace``: rows of round, vertex, 12 features; ``labels``).
    ``replay`` = (rounds, vertices, priorities) arrays replaces the edge
    difference by the given int32 priorities of each (round, vertex).
    ``cmax`` bounds |N_in| * |N_out| of a contractible vertex; the vertices
    left when none is eligible form the core. ``ball`` bounds each witness
    search: it stops after the first hop level at which more than ``ball``
    vertices hold a label (see ``oracle.cpp``). ``theta`` > 0 replaces the
    hop-limited search by Alg. 3's Dijkstra capped at ``theta`` settled
    vertices (``ball`` must then stay unbounded). ``prune`` deletes, after
    each LocalSearch, the overlay edges heavier than the witness distance of
    their pair (``OracleCH.pruned``: rows of round, s, v, w). ``memo`` > 0
    keeps the witness distances across phases and rounds (pairs already
    recorded are not searched again) and clears them at the end of a round
    that leaves more than ``memo`` of them; ``OracleCH.searches`` counts the
    witness searches run. ``level_work`` bounds a hop-limited search's work:
    a level from the second on whose frontier has more out-edges in total is
    not run (``OracleCH.witness_work`` sums the frontier out-edges of the
    levels run). ``composite`` scores by 4 * edge difference + (|N_in| +
    |N_out|) + 8 * hierarchy depth (clamped to +-2^30) instead of the edge
    difference. ``threads`` runs
    the -DORACLE_THREADS build (witness searches on all host threads; the
    same result).
    """
    lib = _load(threads)
    args, keep = _graph_args(g)
    h = C.c_void_p()
    if replay is None:
        rr = ru = rpv = np.zeros(0, np.uint32)
        rpv = np.zeros(0, np.int32)
    else:
        rr = np.ascontiguousarray(replay[0], np.uint32)
        ru = np.ascontiguousarray(replay[1], np.uint32)
        rpv = np.ascontiguousarray(replay[2], np.int32)
    rc = lib.orc_build2(*args, hop_limit, tie_break, tie_seed & 0xFFFFFFFF, int(trace),
                        rr.size, _p(rr), _p(ru), _p(rpv), int(cmax), int(ball), int(theta),
                        int(bool(prune)), int(memo), int(level_work), int(bool(composite)),
                        C.byref(h))
    if rc != 0:
        raise ValueError(f"oracle rejected the graph or parameters (status {rc})")
    n = g.n
    level = np.empty(n, np.uint32)
    prio = np.empty(n, np.int32)
    rank = np.empty(n, np.uint32)
    if n:
        lib.orc_get_level(h, _p(level))
        lib.orc_get_priority(h, _p(prio))
        lib.orc_get_rank(h, _p(rank))
    ns = lib.orc_num_shortcuts(h)
    sc = np.empty((ns, 5), np.uint32)
    if ns:
        lib.orc_get_shortcuts(h, _p(sc))
    nu, nd = lib.orc_num_up(h), lib.orc_num_down(h)
    up = np.empty((nu, 3), np.uint32)
    down = np.empty((nd, 3), np.uint32)
    if nu:
        lib.orc_get_up(h, _p(up))
    if nd:
        lib.orc_get_down(h, _p(down))
    rounds = lib.orc_rounds(h)
    stats = np.empty((rounds, lib.orc_nstat()), np.uint64)
    if rounds:
        lib.orc_get_stats(h, _p(stats))
    nt = lib.orc_num_trace(h)
    tr = np.empty((nt, 14), np.int64)
    if nt:
        lib.orc_get_trace(h, _p(tr))
    labels = np.empty(n, np.int32)
    if n:
        lib.orc_get_labels(h, _p(labels))
    del keep
    och = OracleCH(n, hop_limit, level, prio, rank, sc, up, down, stats, h, threads)
    npr = lib.orc_num_pruned(h)
    pruned = np.empty((npr, 4), np.uint32)
    if npr:
        lib.orc_get_pruned(h, _p(pruned))
    och.trace = tr
    och.labels = labels
    och.pruned = pruned
    och.searches = int(lib.orc_searches(h))
    och.witness_work = int(lib.orc_witness_work(h))
    return och


def round0_scores(g, hop_limit: int = 5, ball: int = None) -> np.ndarray:
    """Scores P[u] of every vertex as round 0 computes them (Alg. 3 + 4),
    with an optional witness ball bound."""
    args, keep = _graph_args(g)
    P = np.empty(g.n, np.int32)
    rc = _load().orc_round0_scores(*args, hop_limit, CMAX_ALL if ball is None else int(ball), _p(P))
    if rc != 0:
        raise ValueError("invalid graph")
    return P


def normalize(g):
    """(offsets, targets, weights) of the normalised graph, heads sorted."""
    lib = _load()
    args, keep = _graph_args(g)
    m = C.c_uint64()
    if lib.orc_normalize(*args, C.byref(m), None, None, None) != 0:
        raise ValueError("invalid graph")
    off = np.empty(g.n + 1, np.uint64)
    tgt = np.empty(m.value, np.uint32)
    w = np.empty(m.value, np.uint32)
    lib.orc_normalize(*args, C.byref(m), _p(off), _p(tgt), _p(w))
    return off, tgt, w


def hop_limited(g, hop_limit: int, src: int) -> np.ndarray:
    """d_H(src, v) for every v on the normalised input graph."""
    args, keep = _graph_args(g)
    d = np.empty(g.n, np.uint32)
    if _load().orc_hop_limited(*args, hop_limit, src, _p(d)) != 0:
        raise ValueError("invalid graph or source")
    return d


def dijkstra(g, src: int) -> np.ndarray:
    """Exact distances from ``src`` on the normalised input graph."""
    args, keep = _graph_args(g)
    d = np.empty(g.n, np.uint32)
    if _load().orc_dijkstra(*args, src, _p(d)) != 0:
        raise ValueError("invalid graph or source")
    return d


def dijkstra_pairs(g, s, t) -> np.ndarray:
    """Exact s-t distances on the input graph for arrays of pairs."""
    args, keep = _graph_args(g)
    s = np.ascontiguousarray(s, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.uint32)
    out = np.empty(s.size, np.uint32)
    if s.size and _load().orc_dijkstra_pairs(*args, s.size, _p(s), _p(t), _p(out)) != 0:
        raise ValueError("invalid graph or pair")
    return out
