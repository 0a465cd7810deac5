"""Python binding of ``libch.so`` (the C ABI declared in ``include/ch.h``).

Argument marshalling only: every step of construction and querying runs in
the library's CUDA kernels. Device buffers come from PyTorch CUDA tensors
(``data_ptr()``); host buffers from NumPy arrays. There is no CPU fallback:
if the library cannot be loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

from . import build as _build

CH_OK = 0
CH_EINVAL = -1
CH_ENOMEM = -2
CH_ECUDA = -3
CH_ETIMEOUT = -4
CH_ERANGE = -5
CH_EAGAIN = -6
CH_INF = 0xFFFFFFFF
CH_TIE_HASHED = 0
CH_TIE_ID = 1
CH_PRIO_EDGE_DIFF = 0
CH_PRIO_LEARNED = 1
CH_PRIO_COMPOSITE = 2
CH_MLP_NPARAM = 5057
CH_NFEAT = 12
CH_NSTAT = 10
CH_NTIME = 6
ROUND_TIME_FIELDS = ("score_ms", "select_ms", "prep_ms", "contract_ms", "update_ms", "witness_ms")

ROUND_STAT_FIELDS = ("affected", "score_sources", "selected", "contract_sources",
                     "candidates", "kept", "merged", "inserted", "vo_after", "eo_after")


class CHError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class GraphT(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m", C.c_uint64), ("offsets", C.c_void_p),
                ("targets", C.c_void_p), ("weights", C.c_void_p), ("on_device", C.c_int32)]


class ParamsT(C.Structure):
    _fields_ = [("hop_limit", C.c_uint32), ("priority", C.c_uint32), ("tie_break", C.c_uint32),
                ("tie_seed", C.c_uint32), ("max_candidates_per_vertex", C.c_uint64),
                ("stream", C.c_void_p), ("mlp_weights", C.c_void_p), ("trace", C.c_int32),
                ("witness_route_deg", C.c_uint32), ("witness_ball_limit", C.c_uint32),
                ("witness_memo_limit", C.c_uint32), ("witness_level_work", C.c_uint32),
                ("witness_prune", C.c_uint32), ("witness_settle_cap", C.c_uint32),
                ("reserved", C.c_uint32)]


class TuneRowT(C.Structure):
    _fields_ = [("hop_limit", C.c_uint32), ("witness_route_deg", C.c_uint32),
                ("build_ms", C.c_double), ("query_ms", C.c_double), ("cost", C.c_double),
                ("shortcuts", C.c_uint64), ("core_vertices", C.c_uint64)]


class QueryConfigT(C.Structure):
    _fields_ = [("layout", C.c_uint32), ("threads", C.c_uint32), ("small_first", C.c_uint32),
                ("stall", C.c_uint32), ("delta", C.c_uint32)]


CH_QUERY_BLOCK_FLAT = 0
CH_QUERY_WARP_FLAT = 1
# (layout, threads, small_first, stall) in the autotuner's order
# The autotuner's candidates as (layout, threads, small_first, stall,
# delta in weight scales), in its timing order; delta = 0 is off.
QUERY_CONFIGS = (tuple((lay, thr, sf, 0, 0) for sf in (0, 1)
                       for lay in (CH_QUERY_BLOCK_FLAT, CH_QUERY_WARP_FLAT) for thr in (128, 256)) +
                 tuple((CH_QUERY_WARP_FLAT, thr, sf, 1, 0) for sf in (0, 1) for thr in (128, 256)) +
                 tuple((CH_QUERY_WARP_FLAT, 256, 1, 1, mult) for mult in (64, 128, 256)))


class ServerParamsT(C.Structure):
    _fields_ = [("blocks", C.c_uint32), ("ring", C.c_uint32), ("pool", C.c_uint64),
                ("idle_ms", C.c_uint32), ("reserved", C.c_uint32)]


class TrainT(C.Structure):
    _fields_ = [("epochs", C.c_uint32), ("batch", C.c_uint32), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class StatsT(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m_input", C.c_uint64), ("rounds", C.c_uint32),
                ("shortcuts", C.c_uint64), ("up_edges", C.c_uint64), ("down_edges", C.c_uint64),
                ("build_ms", C.c_double), ("witness_sources", C.c_uint64),
                ("witness_fallback", C.c_uint64),
                ("normalise_ms", C.c_double), ("score_ms", C.c_double), ("select_ms", C.c_double),
                ("prep_ms", C.c_double), ("contract_ms", C.c_double), ("update_ms", C.c_double),
                ("postprocess_ms", C.c_double), ("witness_ms", C.c_double),
                ("witness_launches", C.c_uint64), ("witness_bytes", C.c_uint64),
                ("witness_dense", C.c_uint64), ("trace_rows", C.c_uint64),
                ("core_vertices", C.c_uint64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libch.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libch.so not found at {path}; run the build first")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.ch_default_params.argtypes = [C.POINTER(ParamsT)]
    lib.ch_default_params.restype = None
    lib.ch_build.argtypes = [C.POINTER(GraphT), C.POINTER(ParamsT), C.POINTER(P)]
    lib.ch_query_batch.argtypes = [P, P, P, C.c_uint64, P, P, P]
    lib.ch_query_batch_host.argtypes = [P, P, P, C.c_uint64, P, P]
    lib.ch_query_status.argtypes = [P, P]
    lib.ch_get_stats.argtypes = [P, C.POINTER(StatsT)]
    lib.ch_get_round_stats.argtypes = [P, P, C.c_uint32]
    lib.ch_get_round_times.argtypes = [P, P, C.c_uint32]
    lib.ch_export.argtypes = [P, P, P, P, P, P, P]
    for f in ("ch_build", "ch_query_batch", "ch_query_batch_host", "ch_query_status",
              "ch_get_stats", "ch_get_round_stats", "ch_get_round_times", "ch_export"):
        getattr(lib, f).restype = C.c_int
    lib.ch_export_trace.argtypes = [P, P, P, P]
    lib.ch_mlp_train.argtypes = [P, P, C.c_uint64, C.POINTER(TrainT), P, P, P, P]
    lib.ch_mlp_forward.argtypes = [P, P, C.c_uint64, P, P]
    lib.ch_mlp_targets.argtypes = [P, C.c_uint64, P, P]
    lib.ch_core_table.argtypes = [P, C.c_uint64, P]
    lib.ch_core_table.restype = C.c_int
    for f in ("ch_export_trace", "ch_mlp_train", "ch_mlp_forward", "ch_mlp_targets"):
        getattr(lib, f).restype = C.c_int
    lib.ch_server_start.argtypes = [P, C.POINTER(ServerParamsT), C.POINTER(P)]
    lib.ch_server_submit.argtypes = [P, C.c_uint32, P, C.c_uint32, C.POINTER(C.c_uint64)]
    lib.ch_server_poll.argtypes = [P, C.c_uint64, P, C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]
    lib.ch_server_replay.argtypes = [P, C.c_uint64, P, P, P, P, P, P, P, P, C.c_double]
    lib.ch_server_stop.argtypes = [P]
    lib.ch_server_blocks.argtypes = [P]
    lib.ch_server_blocks.restype = C.c_uint32
    lib.ch_server_running.argtypes = [P]
    lib.ch_server_running.restype = C.c_int
    for f in ("ch_server_start", "ch_server_submit", "ch_server_poll", "ch_server_replay",
              "ch_server_stop"):
        getattr(lib, f).restype = C.c_int
    lib.ch_build_autotune.argtypes = [C.POINTER(GraphT), C.POINTER(ParamsT), P, C.c_uint32, P,
                                      C.c_uint32, C.c_uint64, C.c_double, C.POINTER(P),
                                      C.POINTER(TuneRowT), C.POINTER(C.c_uint32)]
    lib.ch_build_autotune.restype = C.c_int
    lib.ch_query_one_to_many.argtypes = [P, C.c_uint32, P, C.c_uint64, P, P]
    lib.ch_one_to_all.argtypes = [P, P, C.c_uint64, P, P]
    lib.ch_save.argtypes = [P, C.c_char_p]
    lib.ch_load.argtypes = [C.c_char_p, C.POINTER(P)]
    for f in ("ch_query_one_to_many", "ch_one_to_all", "ch_save", "ch_load"):
        getattr(lib, f).restype = C.c_int
    lib.ch_set_query_config.argtypes = [P, C.POINTER(QueryConfigT)]
    lib.ch_get_query_config.argtypes = [P, C.POINTER(QueryConfigT)]
    lib.ch_query_autotune.argtypes = [P, C.c_uint64, C.c_uint32, P, C.POINTER(QueryConfigT), P]
    lib.ch_query_work.argtypes = [P, P, P]
    lib.ch_query_graph_create.argtypes = [P, P, P, C.c_uint64, P, C.POINTER(P)]
    lib.ch_query_graph_launch.argtypes = [P, P]
    for f in ("ch_set_query_config", "ch_get_query_config", "ch_query_autotune", "ch_query_work",
              "ch_query_graph_create", "ch_query_graph_launch"):
        getattr(lib, f).restype = C.c_int
    lib.ch_query_graph_free.argtypes = [P]
    lib.ch_query_graph_free.restype = None
    lib.ch_free.argtypes = [P]
    lib.ch_free.restype = None
    lib.ch_last_error.restype = C.c_char_p
    lib.ch_version.restype = C.c_char_p
    lib.ch_kernel_launches.restype = C.c_uint64
    lib.ch_trim_memory.restype = C.c_size_t
    lib.ch_debug_fail_alloc.argtypes = [C.c_int64]
    lib.ch_debug_fail_alloc.restype = C.c_int64
    _lib = lib
    return lib


def _check(rc: int):
    if rc != CH_OK:
        raise CHError(rc, _lib.ch_last_error().decode(errors="replace"))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _need_cuda_ids(t, name: str):
    """The device entry points take contiguous 32-bit CUDA tensors of ids."""
    if not _is_torch(t) or not t.is_cuda or not t.is_contiguous() or t.element_size() != 4:
        raise ValueError(f"{name} must be a contiguous 32-bit CUDA tensor of vertex ids")


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return a.ctypes.data_as(C.c_void_p) if a.size else None


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def default_params() -> ParamsT:
    p = ParamsT()
    load().ch_default_params(C.byref(p))
    return p


class CH:
    """A contraction hierarchy owned by libch.so."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle
        # servers and captured graphs whose device work reads this handle's
        # memory; close() ends them first
        self._deps = weakref.WeakSet()

    # -- construction -----------------------------------------------------
    @staticmethod
    def _marshal(graph, n, offsets, targets, weights, hop_limit, tie_break, tie_seed, stream,
                 mlp_weights, trace, max_candidates_per_vertex, witness_route_deg,
                 witness_ball_limit=None, witness_memo_limit=None, witness_level_work=None,
                 witness_prune=False, witness_settle_cap=None, composite=False):
        if graph is not None:
            n, offsets, targets, weights = graph.n, graph.offsets, graph.targets, graph.weights
        g = GraphT()
        g.n = int(n)
        keep = []
        if _is_torch(offsets):
            import torch
            for t in (offsets, targets, weights):
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError("device CSR tensors must be contiguous CUDA tensors")
            if offsets.dtype != torch.int64 or targets.element_size() != 4 or weights.element_size() != 4:
                raise ValueError("offsets must be int64, targets/weights 32-bit")
            g.m = int(targets.numel())
            g.offsets, g.targets, g.weights = offsets.data_ptr(), targets.data_ptr(), weights.data_ptr()
            g.on_device = 1
            st = _stream_ptr(stream)
        else:
            off = _host(offsets, np.uint64)
            tgt = _host(targets, np.uint32)
            w = _host(weights, np.uint32)
            keep = [off, tgt, w]
            g.m = int(tgt.size)
            g.offsets, g.targets, g.weights = _hp(off), _hp(tgt), _hp(w)
            g.on_device = 0
            st = C.c_void_p(None) if stream is None else _stream_ptr(stream)
        p = default_params()
        # a level-work bound of 0 leaves only the first hop level, which is
        # the search of hop limit 1; the ABI's 0 means "no bound"
        if witness_level_work is not None and int(witness_level_work) == 0:
            hop_limit, witness_level_work = min(int(hop_limit), 1), None
        p.hop_limit = hop_limit
        p.tie_break = tie_break
        p.tie_seed = tie_seed & 0xFFFFFFFF
        p.stream = st
        p.trace = int(bool(trace))
        p.witness_route_deg = int(witness_route_deg)
        p.witness_ball_limit = 0 if witness_ball_limit is None else int(witness_ball_limit)
        p.witness_memo_limit = 0 if witness_memo_limit is None else int(witness_memo_limit)
        p.witness_level_work = 0 if witness_level_work is None else int(witness_level_work)
        p.witness_prune = int(bool(witness_prune))
        p.witness_settle_cap = 0 if witness_settle_cap is None else int(witness_settle_cap)
        if max_candidates_per_vertex is not None:
            p.max_candidates_per_vertex = int(max_candidates_per_vertex)
        if mlp_weights is not None:
            wts = np.ascontiguousarray(mlp_weights, dtype=np.float32)
            if wts.size != CH_MLP_NPARAM:
                raise ValueError(f"mlp_weights needs {CH_MLP_NPARAM} floats")
            keep.append(wts)
            p.priority = CH_PRIO_LEARNED
            p.mlp_weights = wts.ctypes.data_as(C.c_void_p)
        if composite:
            if mlp_weights is not None:
                raise ValueError("composite and learned priorities exclude each other")
            p.priority = CH_PRIO_COMPOSITE
        return g, p, keep

    @classmethod
    def build(cls, graph=None, *, n=None, offsets=None, targets=None, weights=None,
              hop_limit: int = 5, tie_break: int = CH_TIE_HASHED, tie_seed: int = 0,
              stream=None, mlp_weights=None, trace: bool = False,
              max_candidates_per_vertex: int | None = None, witness_route_deg: int = 0,
              witness_ball_limit: int | None = None,
              witness_memo_limit: int | None = None,
              witness_level_work: int | None = None, witness_prune: bool = False,
              witness_settle_cap: int | None = None, composite: bool = False) -> "CH":
        """ch_build on a graph given as an ``inputs.Graph`` / NumPy CSR (host
        memory) or as CUDA tensors ``offsets`` (int64), ``targets`` and
        ``weights`` (int32 views of uint32 values) in device memory.
        ``max_candidates_per_vertex`` (Cmax) bounds |N_in| * |N_out| of a
        contractible vertex; None contracts every vertex.
        ``witness_ball_limit`` (θ) stops a witness search after the first hop
        level at which more than θ vertices hold a label; None = unbounded.
        ``witness_memo_limit`` memoises witness distances across rounds and
        clears them after a round that leaves more pairs; None = off.
        ``witness_level_work`` skips a hop level (from the second on) whose
        frontier has more out-edges than that (0 runs the first level only,
        as hop limit 1 does); None = off. ``witness_prune``
        deletes overlay edges heavier than their pair's witness distance
        after each round's rescoring searches. ``witness_settle_cap`` (θ)
        replaces the hop-limited search by Alg. 3's Dijkstra capped at θ
        settled vertices; None = off. ``composite`` scores vertices by
        CH_PRIO_COMPOSITE (4 * edge difference + degree + 8 * depth)."""
        g, p, keep = cls._marshal(graph, n, offsets, targets, weights, hop_limit, tie_break,
                                  tie_seed, stream, mlp_weights, trace, max_candidates_per_vertex,
                                  witness_route_deg, witness_ball_limit, witness_memo_limit,
                                  witness_level_work, witness_prune, witness_settle_cap, composite)
        h = C.c_void_p()
        _check(load().ch_build(C.byref(g), C.byref(p), C.byref(h)))
        del keep
        return cls(h)

    @classmethod
    def build_autotune(cls, graph=None, *, hop_limits=(2, 3, 4, 5), route_degs=(32, 64, 128),
                       sample: int = 1 << 15, queries_per_build: float = 1e6, n=None,
                       offsets=None, targets=None, weights=None, tie_break: int = CH_TIE_HASHED,
                       tie_seed: int = 0, stream=None, mlp_weights=None,
                       max_candidates_per_vertex: int | None = None,
                       witness_ball_limit: int | None = None, level_works=(None,)):
        """ch_build_autotune: builds once per (hop limit, routing threshold),
        keeps the cheapest. ``level_works`` adds the witness level-work bound
        as a third dimension (one ch_build_autotune call per value; None =
        no bound). Returns (CH, rows as dicts with their ``level_work``,
        chosen index)."""
        rd = np.ascontiguousarray(route_degs, dtype=np.uint32)
        best, out, best_i = None, [], 0
        for lw in level_works:
            # level work 0 is the search of hop limit 1 (see _marshal)
            hl = (np.unique(np.minimum(np.ascontiguousarray(hop_limits, dtype=np.uint32), 1))
                  if lw is not None and int(lw) == 0 else np.ascontiguousarray(hop_limits, dtype=np.uint32))
            g, p, keep = cls._marshal(graph, n, offsets, targets, weights, 5, tie_break, tie_seed,
                                      stream, mlp_weights, False, max_candidates_per_vertex, 0,
                                      witness_ball_limit, None, lw)
            rows = (TuneRowT * (hl.size * rd.size))()
            chosen = C.c_uint32()
            h = C.c_void_p()
            rc = load().ch_build_autotune(C.byref(g), C.byref(p), _hp(hl), hl.size, _hp(rd), rd.size,
                                          sample, float(queries_per_build), C.byref(h), rows,
                                          C.byref(chosen))
            del keep
            if rc != CH_OK:
                if best is not None:
                    best.close()
                _check(rc)
            base = len(out)
            out += [dict({f: getattr(r, f) for f, _ in TuneRowT._fields_}, level_work=lw) for r in rows]
            k = base + int(chosen.value)
            cand = cls(h)
            if best is None or out[k]["cost"] < out[best_i]["cost"]:
                if best is not None:
                    best.close()
                best, best_i = cand, k
            else:
                cand.close()
        return best, out, best_i

    # -- queries ----------------------------------------------------------
    def query(self, src, dst, want_settled: bool = False, stream=None):
        """Batched s-t distances. CUDA tensors -> async on ``stream`` (device
        outputs returned as int32 tensors holding uint32 bit patterns); NumPy
        arrays -> synchronous host call returning uint32 arrays."""
        lib = load()
        if _is_torch(src):
            import torch
            if src.shape != dst.shape:
                raise ValueError("sources and targets differ in length")
            k = src.numel()
            out = torch.empty(k, dtype=torch.int32, device=src.device)
            settled = torch.empty(k, dtype=torch.int32, device=src.device) if want_settled else None
            _check(lib.ch_query_batch(self._h, src.data_ptr(), dst.data_ptr(), k, out.data_ptr(),
                                      settled.data_ptr() if settled is not None else None,
                                      _stream_ptr(stream)))
            return (out, settled) if want_settled else out
        s = _host(src, np.uint32)
        t = _host(dst, np.uint32)
        if s.shape != t.shape:
            raise ValueError("sources and targets differ in length")
        out = np.empty(s.size, np.uint32)
        settled = np.empty(s.size, np.uint32) if want_settled else None
        _check(lib.ch_query_batch_host(self._h, _hp(s), _hp(t), s.size, _hp(out),
                                       _hp(settled) if settled is not None else None))
        return (out, settled) if want_settled else out

    def query_status(self, stream=None):
        _check(load().ch_query_status(self._h, _stream_ptr(stream)))

    def query_batch_raw(self, src_ptr: int, dst_ptr: int, k: int, out_ptr: int,
                        settled_ptr: int | None, stream_ptr: int):
        """ch_query_batch on raw device pointers (used inside timed loops)."""
        _check(load().ch_query_batch(self._h, src_ptr, dst_ptr, k, out_ptr, settled_ptr,
                                     stream_ptr))

    def query_one_to_many(self, s: int, dst, stream=None):
        """Distances from s to every target of the CUDA tensor ``dst``
        (int32 view of uint32 ids), asynchronous on ``stream``."""
        import torch
        _need_cuda_ids(dst, "dst")
        out = torch.empty_like(dst)
        _check(load().ch_query_one_to_many(self._h, int(s), dst.data_ptr(), dst.numel(),
                                           out.data_ptr(), _stream_ptr(stream)))
        return out

    def one_to_all(self, src, stream=None):
        """Distances from each source of the CUDA tensor ``src`` (int32 view
        of uint32 ids) to every vertex: an int32 tensor [len(src), n] holding
        uint32 bit patterns, asynchronous on ``stream``."""
        import torch
        _need_cuda_ids(src, "src")
        n = self.stats()["n"]
        out = torch.empty((src.numel(), n), dtype=torch.int32, device=src.device)
        _check(load().ch_one_to_all(self._h, src.data_ptr(), src.numel(), out.data_ptr(),
                                    _stream_ptr(stream)))
        return out

    def core_table(self, max_bytes: int = 16 << 30, stream=None):
        """ch_core_table: the core's all-pairs distance table; queries then
        join their upward searches through it instead of searching inside
        the core."""
        _check(load().ch_core_table(self._h, int(max_bytes), _stream_ptr(stream)))

    # -- saving and loading -------------------------------------------------
    def save(self, path: str):
        _check(load().ch_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "CH":
        h = C.c_void_p()
        _check(load().ch_load(os.fsencode(path), C.byref(h)))
        return cls(h)

    # -- query configuration, autotuning, work, graphs ----------------------
    def set_query_config(self, layout: int, threads: int, small_first: int = 0, stall: int = 0,
                         delta: int = 0):
        _check(load().ch_set_query_config(self._h, C.byref(QueryConfigT(layout, threads, small_first,
                                                                        stall, delta))))

    def query_config(self) -> tuple[int, int, int, int, int]:
        """(layout, threads, small_first, stall, delta); delta in weight units."""
        c = QueryConfigT()
        _check(load().ch_get_query_config(self._h, C.byref(c)))
        return c.layout, c.threads, c.small_first, c.stall, c.delta

    def autotune_queries(self, sample: int = 1 << 16, seed: int = 1, stream=None):
        """Time every query configuration on ``sample`` random queries and keep
        the fastest. Returns (chosen (layout, threads, small_first, stall,
        delta), ms per configuration in QUERY_CONFIGS order)."""
        c = QueryConfigT()
        ms = np.zeros(len(QUERY_CONFIGS), np.float64)
        _check(load().ch_query_autotune(self._h, sample, seed, _stream_ptr(stream), C.byref(c),
                                        _hp(ms)))
        return (c.layout, c.threads, c.small_first, c.stall, c.delta), ms

    def query_work(self, stream=None) -> tuple[int, int]:
        """(expansions, edges scanned) of the query searches since the last call."""
        out = np.zeros(2, np.uint64)
        _check(load().ch_query_work(self._h, _stream_ptr(stream), _hp(out)))
        return int(out[0]), int(out[1])

    def query_graph(self, src, dst, out) -> "QueryGraph":
        """Capture a query batch on fixed CUDA tensors into a CUDA graph."""
        if src.shape != dst.shape or out.shape != src.shape:
            raise ValueError("sources, targets and outputs differ in length")
        h = C.c_void_p()
        _check(load().ch_query_graph_create(self._h, src.data_ptr(), dst.data_ptr(), src.numel(),
                                            out.data_ptr(), C.byref(h)))
        g = QueryGraph(h, (src, dst, out), self)
        self._deps.add(g)
        return g

    # -- introspection ----------------------------------------------------
    def stats(self) -> dict:
        s = StatsT()
        _check(load().ch_get_stats(self._h, C.byref(s)))
        return {name: getattr(s, name) for name, _ in StatsT._fields_}

    def round_stats(self) -> np.ndarray:
        r = self.stats()["rounds"]
        out = np.zeros((r, CH_NSTAT), np.uint64)
        if r:
            _check(load().ch_get_round_stats(self._h, _hp(out), r))
        return out

    def round_times(self) -> np.ndarray:
        """Per-round device time (ms) of each phase, ROUND_TIME_FIELDS columns."""
        r = self.stats()["rounds"]
        out = np.zeros((r, CH_NTIME), np.float64)
        if r:
            _check(load().ch_get_round_times(self._h, _hp(out), r))
        return out

    def export(self) -> dict:
        st = self.stats()
        n = st["n"]
        level = np.empty(n, np.uint32)
        prio = np.empty(n, np.int32)
        rank = np.empty(n, np.uint32)
        sc = np.empty((st["shortcuts"], 5), np.uint32)
        up = np.empty((st["up_edges"], 3), np.uint32)
        down = np.empty((st["down_edges"], 3), np.uint32)
        _check(load().ch_export(self._h, _hp(level), _hp(prio), _hp(rank), _hp(sc), _hp(up),
                                _hp(down)))
        return dict(level=level, priority=prio, rank=rank, shortcuts=sc, up=up, down=down)

    def export_trace(self) -> dict:
        """Rows (round, vertex, 12 features), the priority of each row, and
        the per-vertex training labels (builds made with trace=True)."""
        st = self.stats()
        k = st["trace_rows"]
        rows = np.empty((k, 14), np.int64)
        prio = np.empty(k, np.int32)
        labels = np.empty(st["n"], np.int32)
        _check(load().ch_export_trace(self._h, _hp(rows), _hp(prio), _hp(labels)))
        return dict(rows=rows, prio=prio, labels=labels)

    def close(self):
        """Stop this hierarchy's servers and free its captured graphs, then
        free the hierarchy. If a server does not stop, its kernel may still
        read the hierarchy, so the hierarchy's memory is left allocated for
        the rest of the process and the error is raised."""
        if not self._h:
            return
        for dep in list(self._deps):
            try:
                if isinstance(dep, Server):
                    dep.stop()
                else:
                    dep.close()
            except Exception:
                self._h = None  # never freed: device work may still use it
                raise
        h, self._h = self._h, None
        load().ch_free(h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class QueryGraph:
    """A query batch captured as a CUDA graph (see ch_query_graph_create)."""

    def __init__(self, handle, buffers, owner):
        self._h = handle
        self._keep = buffers  # the graph reads and writes these tensors
        self._owner = owner

    def launch(self, stream=None):
        _check(load().ch_query_graph_launch(self._h, _stream_ptr(stream)))

    def close(self):
        if self._h:
            h, self._h = self._h, None
            load().ch_query_graph_free(h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Query server (continuous batching) over a built hierarchy."""

    def __init__(self, ch: CH, blocks: int = 0, ring: int = 1 << 14, pool: int = 1 << 22,
                 idle_ms: int = 1000):
        self._ch = ch
        p = ServerParamsT(blocks, ring, pool, idle_ms, 0)
        self._h = C.c_void_p()
        _check(load().ch_server_start(ch._h, C.byref(p), C.byref(self._h)))
        ch._deps.add(self)

    @property
    def blocks(self) -> int:
        """Blocks of the device loop."""
        return int(load().ch_server_blocks(self._h))

    def running(self) -> bool:
        """ch_server_running: whether the device loop's kernel runs now (it
        ends after idle_ms without requests and is launched again by the next
        submit or poll)."""
        rc = load().ch_server_running(self._h)
        if rc < 0:
            _check(rc)
        return rc == 1

    def submit(self, s: int, targets) -> int | None:
        """Ticket of the published request, or None when the server is full."""
        t = _host(targets, np.uint32)
        tk = C.c_uint64()
        rc = load().ch_server_submit(self._h, int(s), _hp(t), t.size, C.byref(tk))
        if rc == CH_EAGAIN:
            return None
        _check(rc)
        return tk.value

    def poll(self, ticket: int, k: int):
        """Answers (uint32[k]) once served, else None."""
        out = np.empty(k, np.uint32)
        done = C.c_int32()
        _check(load().ch_server_poll(self._h, ticket, _hp(out), C.byref(done), None))
        return out if done.value else None

    def replay(self, src, ks, targets, arrival_ns, limit_s: float = 300.0):
        """Serve a schedule: request i = (src[i], targets[toff[i]:toff[i]+ks[i]])
        due at arrival_ns[i]. Returns (answers per target, latency_ns,
        service_ns) arrays."""
        src = _host(src, np.uint32)
        ks = _host(ks, np.uint32)
        toff = np.zeros(ks.size, np.uint64)
        if ks.size:
            toff[1:] = np.cumsum(ks[:-1], dtype=np.uint64)
        tg = _host(targets, np.uint32)
        arr = _host(arrival_ns, np.uint64)
        ans = np.empty(tg.size, np.uint32)
        lat = np.empty(ks.size, np.uint64)
        svc = np.empty(ks.size, np.uint64)
        _check(load().ch_server_replay(self._h, ks.size, _hp(src), _hp(ks), _hp(toff), _hp(tg),
                                       _hp(arr), _hp(ans), _hp(lat), _hp(svc), limit_s))
        return ans, lat, svc

    def stop(self):
        if self._h:
            h, self._h = self._h, None
            _check(load().ch_server_stop(h))

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.stop()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def training_labels(rows, stream=None) -> np.ndarray:
    """ch_mlp_targets: the training target of each trace row (float32),
    computed on the device from the row's edge difference and hierarchy
    depth. ``rows`` is a host int64 array [n, 14] or a CUDA tensor; the
    result is a host array for host input, else a CUDA tensor."""
    import torch
    on_host = not isinstance(rows, torch.Tensor)
    d = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int64)).cuda() if on_host else rows
    if d.dtype != torch.int64 or d.dim() != 2 or d.shape[1] != 14 or not d.is_cuda:
        raise ValueError("rows must be an int64 [n, 14] array")
    d = d.contiguous()
    y = torch.empty(d.shape[0], dtype=torch.float32, device=d.device)
    _check(load().ch_mlp_targets(d.data_ptr(), d.shape[0], y.data_ptr(), _stream_ptr(stream)))
    if on_host:
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return y.cpu().numpy()
    return y


def mlp_init(seed: int = 0, scale: float = 0.3) -> np.ndarray:
    """Initial MLP weights (float32, CH_MLP_NPARAM): normal weights scaled by
    scale / sqrt(fan_in), zero biases."""
    rng = np.random.default_rng(seed)
    nin, nh = CH_NFEAT, 64
    w1 = rng.normal(0, scale / np.sqrt(nin), (nin, nh))
    w2 = rng.normal(0, scale / np.sqrt(nh), (nh, nh))
    w3 = rng.normal(0, scale / np.sqrt(nh), nh)
    return np.concatenate([w1.ravel(), np.zeros(nh), w2.ravel(), np.zeros(nh), w3,
                           [0.0]]).astype(np.float32)


def mlp_train(rows, labels, weights, epochs=3, batch=8192, lr=2e-3, beta1=0.9,
              beta2=0.999, eps=1e-8, stream=None):
    """ch_mlp_train on CUDA tensors: rows int64 [n, 14], labels float32 [n],
    weights float32 [CH_MLP_NPARAM] (updated in place). With epochs=0
    returns the gradient of the first batch instead of training."""
    import torch
    tp = TrainT(epochs, batch, lr, beta1, beta2, eps)
    n = rows.shape[0]
    loss = np.zeros(max(epochs, 1), np.float32)
    grad = torch.zeros(CH_MLP_NPARAM, dtype=torch.float32, device=weights.device)
    _check(load().ch_mlp_train(rows.data_ptr(), labels.data_ptr(), n, C.byref(tp),
                               weights.data_ptr(), _hp(loss), grad.data_ptr(),
                               _stream_ptr(stream)))
    return (grad, loss) if epochs == 0 else loss


def mlp_forward(weights, rows, stream=None):
    """ch_mlp_forward: MLP outputs for trace rows (CUDA int64 tensor [n, 14])."""
    import torch
    w = np.ascontiguousarray(weights, dtype=np.float32)
    y = torch.empty(rows.shape[0], dtype=torch.float32, device=rows.device)
    _check(load().ch_mlp_forward(_hp(w), rows.data_ptr(), rows.shape[0], y.data_ptr(),
                                 _stream_ptr(stream)))
    return y


def version() -> str:
    return load().ch_version().decode()


def kernel_launches() -> int:
    """CUDA kernels libch.so has launched in this process."""
    return int(load().ch_kernel_launches())


def trim_memory() -> int:
    """ch_trim_memory: waits for the current device and returns the library's
    cached device blocks to CUDA; the bytes released."""
    return int(load().ch_trim_memory())


def debug_fail_alloc(after: int) -> int:
    """Failure injection (ch_debug_fail_alloc): the library's device
    allocation after the next ``after`` ones fails with CH_ENOMEM, once; a
    negative value turns it off. Returns the previous setting."""
    return int(load().ch_debug_fail_alloc(int(after)))
