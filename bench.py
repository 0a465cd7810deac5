#!/usr/bin/env python3
"""Benchmark: CH construction + a batch of s-t queries on one GB300 per rank.

One step = the whole hot path on the road-like workload: ``ch_build`` of the
1M-vertex geometric 3-NN graph (inputs already in device memory) followed by
one batch of 1M uniform random s-t queries through ``ch_query_batch``.

Headline ``value``: CH build seconds per step (the paper's headline metric,
lower is better). The same line carries the shortcut count, the queries/sec
of the batch, the per-kernel roofline of the dominant kernel, the CPU oracle
timed on a bounded sample, the SM clocks seen during the timed region and an
end-to-end measurement through host buffers.

Multi-GPU: the path does not shard (a round needs the global selection and
merge), so ``--gpus N`` runs N independent replicas, one per rank; the
reported times are the maximum over ranks.

``--impl reference`` times the CPU oracle (the only reference this method
has: the paper ships no code) on host cores, on a bounded sample of the same
workload, scaled to the workload's size.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2412_18008_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    # name: (n, graph seed, query seed, queries)
    "geo1M": (1_000_000, 3, 4, 1_000_000),
    "geo256K": (256_000, 100, 101, 1_000_000),
    # RMAT stress graph: 2^21 vertices, 2^25 edge samples (a=.57, b=c=.19),
    # weights U[1,1000]; built with a finite candidate bound (--cmax)
    "rmat2M": (1 << 21, 8, 9, 100_000),
    # the same family scaled down (16 edge samples per vertex)
    "rmat128K": (1 << 17, 8, 9, 100_000),
    "rmat32K": (1 << 15, 8, 9, 100_000),
}


def make_graph(name: str, sample: bool = False):
    """The workload's graph, or (sample=True) the small graph of the same
    family whose oracle build stands in for the CPU baseline."""
    n, gseed, _, _ = WORKLOADS[name]
    if name.startswith("rmat"):
        if sample:  # same samples per vertex (16) at 2^12 vertices
            return I.rmat_graph(scale=12, nsamples=1 << 16, wmax=1000, seed=7)
        scale = n.bit_length() - 1
        return I.rmat_graph(scale=scale, nsamples=16 << scale, wmax=1000, seed=gseed)
    if sample:
        return I.geometric_knn_graph(100_000, seed=7)
    return I.geometric_knn_graph(n, seed=gseed)
METRIC = "CH build seconds & shortcut count; batched s-t queries/sec; p99 query latency"
L2_BYTES = 129 * 1024 * 1024
# DRAM bytes (read + write) of the k_query_block launches of the full 1M
# query batch (first pass + overflow redo), from an ncu capture of the
# current kernel on this workload (set to None when the kernel changes).
QUERY_TRAFFIC_PER_LAUNCH = None
# L2 bytes per query of that kernel in the configuration named (layout,
# threads, small_first, stall, delta) (lts__t_sectors * 32 over a
# 200K-query pass of the same workload; L2 traffic is per-query work, so it
# scales with the queries of a batch).
QUERY_L2_CONFIG = (1, 256, 1, 1, 256)
QUERY_L2_BYTES_PER_QUERY = 217_501


def max_over_ranks(values, world: int, device):
    """Per-rank timings -> their maximum over the ranks (on every rank).
    Replicas run the same workload each; the slowest rank sets the time."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def query_latency(h, s_d, t_d, stream, samples: int = 2000):
    """p50/p99 (us) of single s-t queries, one ch_query_batch call each, timed
    on the device; None (with the error) if the probe cannot run."""
    try:
        import torch
        k = min(samples, s_d.numel())
        out = torch.empty(1, dtype=torch.int32, device=s_d.device)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        sp = stream.cuda_stream
        for _ in range(16):  # warm-up
            h.query_batch_raw(s_d[0:].data_ptr(), t_d[0:].data_ptr(), 1, out.data_ptr(), None, sp)
        for i in range(k):
            a, b = ev[i]
            a.record(stream)
            h.query_batch_raw(s_d[i:].data_ptr(), t_d[i:].data_ptr(), 1, out.data_ptr(), None, sp)
            b.record(stream)
        stream.synchronize()
        us = np.array([a.elapsed_time(b) * 1e3 for a, b in ev])
        return {"p50_us": float(np.percentile(us, 50)), "p99_us": float(np.percentile(us, 99)),
                "samples": int(k), "how": "one-pair ch_query_batch calls, CUDA events on the stream"}
    except Exception as e:  # the probe must never cost the benchmark line
        return {"p50_us": None, "p99_us": None, "error": repr(e)[:200]}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="geo1M", choices=sorted(WORKLOADS))
    ap.add_argument("--hop-limit", type=int, default=5)
    ap.add_argument("--cmax", type=int, default=None,
                    help="candidate bound |N_in|*|N_out| of a contractible vertex (default: none)")
    ap.add_argument("--witness-ball", type=int, default=None,
                    help="witness ball bound: stop a search after the first hop level that "
                         "reaches more than this many vertices (default: none)")
    ap.add_argument("--memo", type=int, default=None,
                    help="memoise witness distances across rounds, clearing the map after a "
                         "round that leaves more pairs than this (default: off)")
    ap.add_argument("--level-work", type=int, default=None,
                    help="skip a witness hop level (from the second on) whose frontier has more "
                         "out-edges than this (default: off)")
    ap.add_argument("--prune", action="store_true",
                    help="prune overlay edges heavier than their pair's witness distance")
    ap.add_argument("--theta", type=int, default=None,
                    help="Alg. 3's witness search: a Dijkstra capped at this many settled "
                         "vertices, in place of the hop-limited search (default: off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the learned-priority (1M) and 16M serving records of the default line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default query kernel configuration")
    ap.add_argument("--build-only", action="store_true",
                    help="time the CH build alone (profiling the build kernels)")
    ap.add_argument("--queries", type=int, default=None,
                    help="query batch size (default: the workload's)")
    ap.add_argument("--compare-learned", action="store_true",
                    help="train the learned priority on traces of 20 seeded 256K-vertex graphs "
                         "of the family and compare it with the edge difference on the held-out "
                         "1M-vertex graph (seed 5)")
    ap.add_argument("--serve", action="store_true",
                    help="continuous-batching server: max throughput, then Poisson arrivals at "
                         "50/80/95%% of it (p50/p99 latency), against one batch call per request")
    ap.add_argument("--serve-workload", default="geo1M",
                    help="geo1M or geo16M (16M-vertex graph of the same family, seed 6)")
    ap.add_argument("--serve-requests", type=int, default=40_000)
    ap.add_argument("--train-graphs", type=int, default=20)
    ap.add_argument("--tune-build", action="store_true",
                    help="with --compare-learned: pick the hop limit and witness routing with the "
                         "build autotuner first")
    ap.add_argument("--train-epochs", type=int, default=4)
    return ap.parse_args()


def l2_read_gbs(dev, mbytes: int = 48, reps: int = 50) -> float:
    """L2 read bandwidth, measured: a float32 sum over a buffer that stays
    in the 129 MB L2 (warmed first), timed with CUDA events. A lower bound
    of the L2 peak (the reduction also has to issue its arithmetic)."""
    import torch
    x = torch.ones(mbytes * (1 << 20) // 4, dtype=torch.float32, device=dev)
    for _ in range(5):
        x.sum()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        x.sum()
    e1.record()
    torch.cuda.synchronize()
    return reps * x.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.devnull if False else f"/tmp/ch_clocks_{os.getpid()}.csv", "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.out.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_info():
    """Host cores and CPU model (from /proc/cpuinfo: 'model name' on x86,
    implementer/part ids on Arm)."""
    import platform
    info = {"nproc": os.cpu_count(), "machine": platform.machine()}
    model = None
    try:
        fields = {}
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip().lower(), v.strip()
                if k in ("model name", "cpu implementer", "cpu part") and k not in fields:
                    fields[k] = v
        model = fields.get("model name") or (
            f"implementer {fields.get('cpu implementer')} part {fields.get('cpu part')}"
            if fields else None)
    except OSError:
        pass
    info["cpu_model"] = model
    return info


def oracle_sample_sizes(workload: str):
    """Two sample graphs of the workload's family (the smaller first): the
    oracle is timed on both and the time extrapolated to the workload along
    the power law through the two points."""
    n = WORKLOADS[workload][0]
    if workload.startswith("rmat"):
        return [(1 << sc, lambda sc=sc: I.rmat_graph(scale=sc, nsamples=16 << sc, wmax=1000, seed=7))
                for sc in (11, 12)]
    return [(k, lambda k=k: I.geometric_knn_graph(k, seed=7)) for k in (min(n, 100_000), min(n, 200_000))]


def oracle_build_s(g, args, threads=False):
    import oracle as O
    t0 = time.perf_counter()
    O.build_ch(g, args.hop_limit, cmax=O.CMAX_ALL if args.cmax is None else args.cmax,
               ball=O.CMAX_ALL if args.witness_ball is None else args.witness_ball, threads=threads,
               memo=args.memo or 0,
               level_work=O.CMAX_ALL if args.level_work is None else args.level_work,
               prune=args.prune, theta=args.theta or 0)
    return time.perf_counter() - t0


def power_law(n1, t1, n2, t2, n):
    """t(n) through (n1, t1) and (n2, t2) on t = a * n^b; returns (t(n), b)."""
    b = float(np.log(t2 / t1) / np.log(n2 / n1)) if n2 != n1 and t1 > 0 and t2 > 0 else 1.0
    return t2 * (n / n2) ** b, b


def cpu_baseline_record(args):
    """The oracle on this host: its -DORACLE_THREADS build (all host threads
    for the witness searches and the query batch; the same output as one
    thread) on the full workload, once; and the single-thread oracle on the
    two sample graphs, extrapolated to the workload along the power law
    through them (an estimate: the oracle's time grows faster than that law
    at larger sizes, so it reads low)."""
    n = WORKLOADS[args.workload][0]
    hi = host_info()
    oracle_build_s(I.geometric_knn_graph(2000, seed=7), args)  # load + warm
    full = oracle_build_s(make_graph(args.workload), args, threads=True)
    (n1, g1f), (n2, g2f) = oracle_sample_sizes(args.workload)
    t1 = oracle_build_s(g1f(), args)
    t2 = oracle_build_s(g2f(), args)
    est, b = power_law(n1, t1, n2, t2, n)
    return {"value": full, "unit": "s", "cores": hi["nproc"], "kind": "oracle",
            "sample": f"the full workload ({n} vertices), one build of the -DORACLE_THREADS oracle "
                      f"on {hi['nproc']} host threads",
            "host": hi,
            "single_thread_estimate": {
                "value": est, "unit": "s", "cores": 1,
                "sample": f"one-thread oracle builds of {n1}- and {n2}-vertex graphs of the family "
                          f"({t1:.2f} s and {t2:.2f} s), extrapolated along the power law through "
                          f"them (exponent {b:.2f}); an underestimate at this size"}}


def run_reference(args):
    """The oracle as the reference arm, its -DORACLE_THREADS build on every
    host thread: the warm-up steps build the smaller sample graph of the
    family, the timed steps the larger one; value = the timed mean
    extrapolated to the workload along the power law through the two means
    (the oracle's time grows faster than that law at larger sizes, so the
    value reads low). ms_per_step is the timed step as run."""
    n = WORKLOADS[args.workload][0]
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    (n1, g1f), (n2, g2f) = oracle_sample_sizes(args.workload)
    g1, g2 = g1f(), g2f()
    oracle_build_s(I.geometric_knn_graph(2000, seed=7), args, threads=True)  # load + warm
    warm = [oracle_build_s(g1, args, threads=True) for _ in range(max(1, args.warmup))]
    times = [oracle_build_s(g2, args, threads=True) for _ in range(args.steps)]
    t1, t2 = statistics.mean(warm), statistics.mean(times)
    value, b = power_law(n1, t1, n2, t2, n)
    hi = host_info()
    sample = (f"timed steps: -DORACLE_THREADS oracle build ({hi['nproc']} host threads) of a "
              f"{n2}-vertex graph of the same family ({args.workload}), mean {t2:.2f} s; warm-up "
              f"steps: {n1} vertices, mean {t1:.2f} s; value extrapolated to {n} vertices along the "
              f"power law through the two (exponent {b:.2f}), which reads low at this size")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t2 * 1000, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "vertices": n, "hop_limit": args.hop_limit,
                   "cmax": args.cmax, "sample_vertices": n2},
        "cpu_baseline": {"value": value, "unit": "s", "cores": hi["nproc"], "kind": "oracle",
                         "sample": sample, "host": hi},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def modes_record(args, g, off, tgt, wt, s_d, t_d, stream, steps=2, warmup=1):
    """The method's other construction modes on the same graph and GPU:
    memoised witness distances across rounds (Alg. 3's dist), with overlay
    pruning, Alg. 3's settled-vertex cap, the composite priority; build
    seconds (CUDA events), shortcuts, rounds, witness searches, mean search
    space and queries/s on the first 100K pairs of the batch, whose answers
    must equal the plain build's. Then one-to-all distances (PHAST sweeps)
    on the plain hierarchy: 64 sources, microseconds per source and the
    sweeps' algorithmic HBM bytes."""
    import torch
    from paper_2412_18008_gb300 import ch
    nq = min(100_000, s_d.numel())
    ds, dt = s_d[:nq], t_d[:nq]
    modes = [("plain", {}), ("memo", {"witness_memo_limit": 1 << 30}),
             ("memo_prune", {"witness_memo_limit": 1 << 30, "witness_prune": True}),
             ("settle_cap_100", {"witness_settle_cap": 100}),
             ("composite", {"composite": True})]
    out, ref = {}, None
    for name, kw in modes:
        times = []
        for k in range(warmup + steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = ch.CH.build(n=g.n, offsets=off, targets=tgt, weights=wt, hop_limit=args.hop_limit,
                            stream=stream, **kw)
            e1.record(stream)
            stream.synchronize()
            if k >= warmup:
                times.append(e0.elapsed_time(e1))
            if k + 1 < warmup + steps:
                h.close()
        st = h.stats()
        d, sett = h.query(ds, dt, want_settled=True, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.query(ds, dt, stream=stream)
        e1.record(stream)
        stream.synchronize()
        d = d.cpu().numpy()
        if ref is None:
            ref = d
        out[name] = {"build_s": statistics.mean(times) / 1e3, "shortcuts": st["shortcuts"],
                     "rounds": st["rounds"], "witness_searches": st["witness_sources"],
                     "witness_ms": st["witness_ms"],
                     "mean_search_space": float(sett.cpu().numpy().view(np.uint32).mean()),
                     "queries_per_s": nq / (e0.elapsed_time(e1) * 1e-3),
                     "answers_equal_plain": bool(np.array_equal(d, ref))}
        if name == "plain":
            # one-to-all on the plain hierarchy: one pass of 64 sources
            src = s_d[:64]
            h.one_to_all(src, stream=stream)  # warm
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = h.one_to_all(src, stream=stream)
            e1.record(stream)
            stream.synchronize()
            h.query_status(stream)
            ms = e0.elapsed_time(e1)
            # algorithmic bytes of one pass of 64 sources: per vertex and
            # sweep a 256-B label row read and written, per CH edge 8 B plus
            # a 256-B row, per vertex 256 B read and 256 B written by the
            # output pass
            m_ch = st["up_edges"] + st["down_edges"]
            bytes_pass = 2 * 512 * g.n + 264 * m_ch + 512 * g.n
            peak, _ = load_peaks()
            gbs = bytes_pass / (ms * 1e-3) / 1e9
            # spot check against the query kernel: the distances of pairs
            # (source, target) read from the rows equal the batch's answers
            tt = t_d[:64].long()
            row_d = res[torch.arange(64, device=res.device), tt].cpu().numpy()
            out["one_to_all"] = {"sources": 64, "ms": ms, "us_per_source": ms * 1e3 / 64,
                                 "achieved_gbs": gbs, "hbm_frac": gbs / peak,
                                 "matches_pair_queries": bool(np.array_equal(row_d, ref[:64]))}
        h.close()
    return out


def rmat_record(args, steps=2, warmup=1, nq=50):
    """The RMAT stress graph (2^21 vertices, 2^25 edge samples) with a finite
    candidate bound and the core it leaves: build seconds (CUDA events),
    rounds, core, shortcuts, witness time, and queries/s of a small batch,
    whose searches cover the core. (Its hierarchy and answers are checked
    against the oracle by tests/test_rmat_full_size.py, not here.)"""
    import torch
    from paper_2412_18008_gb300 import ch
    dev = torch.device("cuda", 0)
    g = make_graph("rmat2M")
    kw = dict(hop_limit=2, max_candidates_per_vertex=256, witness_ball_limit=256,
              witness_level_work=1024, witness_memo_limit=1 << 30)
    off = torch.from_numpy(g.offsets.view(np.int64)).to(dev)
    tgt = torch.from_numpy(g.targets.view(np.int32)).to(dev)
    wt = torch.from_numpy(g.weights.view(np.int32)).to(dev)
    times = []
    for k in range(warmup + steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h = ch.CH.build(n=g.n, offsets=off, targets=tgt, weights=wt, **kw)
        e1.record()
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e1))
        if k + 1 < warmup + steps:
            h.close()
    st = h.stats()
    s_h, t_h = I.random_pairs(g.n, nq, seed=9)
    ds = torch.from_numpy(s_h.view(np.int32)).to(dev)
    dt = torch.from_numpy(t_h.view(np.int32)).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    d = h.query(ds, dt)
    e1.record()
    torch.cuda.synchronize()
    h.close()
    return {"workload": "rmat2M", "vertices": g.n, "edge_samples": int(g.m),
            "params": {"hop_limit": 2, "cmax": 256, "witness_ball": 256, "witness_level_work": 1024,
                       "witness_memo": 1 << 30},
            "build_s": statistics.mean(times) / 1e3, "rounds": st["rounds"],
            "core_vertices": st["core_vertices"], "shortcuts": st["shortcuts"],
            "witness_ms": st["witness_ms"], "queries": nq,
            "queries_per_s": nq / (e0.elapsed_time(e1) * 1e-3)}


def compare_learned(args, steps=None, warmup=None):
    """Learned priority vs edge difference (one JSON line). geo1M: trained on
    traces of 20 seeded 256K-vertex graphs of the family, compared on a
    held-out 1M graph (seed 5). rmat2M: trained on traces of seeded 2^17-vertex
    RMAT graphs (2^21 samples each) under the same candidate bound, compared
    on the 2M stress graph, with the hop limit and witness routing chosen by
    the build autotuner (--tune-build)."""
    import torch
    from paper_2412_18008_gb300 import ch
    dev = torch.device("cuda", 0)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    rmat = args.workload.startswith("rmat")
    cmax = args.cmax
    hop_limit, route_deg, tune_rows = args.hop_limit, 0, None
    if rmat:
        g = make_graph(args.workload)
        tscale = g.n.bit_length() - 3  # training graphs a quarter of the size
        train_graph = lambda seed: I.rmat_graph(scale=tscale, nsamples=16 << tscale, wmax=1000, seed=seed)
        seeds = range(200, 200 + args.train_graphs)
        test_seed, nq_cmp, n_ss = WORKLOADS[args.workload][1], 100_000, 10_000
    else:
        train_graph = lambda seed: I.geometric_knn_graph(256_000, seed=seed)
        seeds = range(100, 100 + args.train_graphs)
        g = I.geometric_knn_graph(1_000_000, seed=5)
        test_seed, nq_cmp, n_ss = 5, 1_000_000, 100_000
    ball = args.witness_ball
    if args.tune_build:
        h, tune_rows, k = ch.CH.build_autotune(g, hop_limits=(1, 2, 3, 4, 5), route_degs=(32, 64, 128),
                                               sample=1 << 14, queries_per_build=nq_cmp,
                                               max_candidates_per_vertex=cmax, witness_ball_limit=ball)
        hop_limit, route_deg = tune_rows[k]["hop_limit"], tune_rows[k]["witness_route_deg"]
        h.close()
    t0 = time.perf_counter()
    rows, labels = [], []
    for seed in seeds:
        tr = ch.CH.build(train_graph(seed), hop_limit=hop_limit, trace=True,
                         max_candidates_per_vertex=cmax, witness_route_deg=route_deg,
                         witness_ball_limit=ball).export_trace()
        rows.append(tr["rows"])
        labels.append(ch.training_labels(tr["rows"]))
    rows = np.concatenate(rows)
    labels = np.concatenate(labels)
    t_traces = time.perf_counter() - t0
    drows = torch.from_numpy(rows).to(dev)
    dlab = torch.from_numpy(labels).to(dev)
    w = torch.from_numpy(ch.mlp_init(11)).to(dev)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss = ch.mlp_train(drows, dlab, w, epochs=args.train_epochs, batch=8192)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    weights = w.cpu().numpy()
    s_h, t_h = I.random_pairs(g.n, nq_cmp, seed=6)
    off = torch.from_numpy(g.offsets.view(np.int64)).to(dev)
    tgt = torch.from_numpy(g.targets.view(np.int32)).to(dev)
    wt = torch.from_numpy(g.weights.view(np.int32)).to(dev)
    ds = torch.from_numpy(s_h.view(np.int32)).to(dev)
    dt = torch.from_numpy(t_h.view(np.int32)).to(dev)
    res = {}
    answers = {}
    for name, mw in (("edge_difference", None), ("learned", weights)):
        times = []
        for k in range(warmup + steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            h = ch.CH.build(n=g.n, offsets=off, targets=tgt, weights=wt, hop_limit=hop_limit,
                            mlp_weights=mw, max_candidates_per_vertex=cmax,
                            witness_route_deg=route_deg, witness_ball_limit=ball)
            e1.record()
            torch.cuda.synchronize()
            if k >= warmup:
                times.append(e0.elapsed_time(e1))
            if k + 1 < warmup + steps:
                h.close()
        st = h.stats()
        d, sett = h.query(ds[:n_ss], dt[:n_ss], want_settled=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        full = h.query(ds, dt)
        e1.record()
        torch.cuda.synchronize()
        answers[name] = full.cpu().numpy()
        res[name] = {"build_s": statistics.mean(times) / 1000.0, "shortcuts": st["shortcuts"],
                     "rounds": st["rounds"], "core_vertices": st["core_vertices"],
                     "queries_per_s": nq_cmp / (e0.elapsed_time(e1) * 1e-3),
                     "mean_search_space": float(sett.cpu().numpy().view(np.uint32).mean())}
        h.close()
    line = {
        "metric": "learned vs edge-difference priority: CH build seconds, shortcut count, "
                  "mean upward search-space size",
        "config": {"workload": f"{args.workload}-learned", "vertices": g.n, "edges": int(g.m),
                   "test_seed": test_seed, "train_graphs": args.train_graphs,
                   "train_vertices_each": (1 << tscale) if rmat else 256_000,
                   "train_rows": int(rows.shape[0]), "train_epochs": args.train_epochs,
                   "cmax": cmax, "witness_ball_limit": ball, "hop_limit": hop_limit,
                   "witness_route_deg": route_deg},
        "build_autotune": tune_rows,
        "results": res,
        "distances_identical": bool(np.array_equal(answers["edge_difference"], answers["learned"])),
        "queries_compared": nq_cmp,
        "train_loss_per_epoch": [float(x) for x in loss],
        "trace_seconds": t_traces, "train_seconds": t_train,
        "steps": steps, "warmup": warmup, "dtype": "bf16 MLP / u32 graph",
    }
    return line


def serve_bench(args, workload=None, nreq=None):
    """Serving: throughput and latency percentiles (a dict for one JSON line)."""
    import torch
    from paper_2412_18008_gb300 import ch
    dev = torch.device("cuda", 0)
    workload = args.serve_workload if workload is None else workload
    if workload == "geo16M":
        n, gseed = 16_000_000, 6
    else:
        n, gseed = 1_000_000, 3
    g = I.geometric_knn_graph(n, seed=gseed)
    h = ch.CH.build(g, hop_limit=args.hop_limit)
    st = h.stats()
    nreq = args.serve_requests if nreq is None else nreq
    src, ks, tg = I.request_mix(n, nreq, seed=7)
    expected = h.query(np.repeat(src, ks), tg)

    def pct(lat_ns):
        return {"p50_us": float(np.percentile(lat_ns, 50)) / 1e3,
                "p99_us": float(np.percentile(lat_ns, 99)) / 1e3}

    out = {}
    with ch.Server(h, blocks=0, ring=1 << 14, pool=1 << 24, idle_ms=20_000) as sv:
        nblocks = sv.blocks
        # saturated: everything due at once
        t0 = time.perf_counter()
        ans, lat, svc = sv.replay(src, ks, tg, np.zeros(nreq, np.uint64), limit_s=1200.0)
        makespan = float(lat.max()) * 1e-9
        assert np.array_equal(ans, expected), "served answers differ from batch answers"
        max_rps = nreq / makespan
        out["saturated"] = {"requests_per_s": max_rps, "queries_per_s": float(ks.sum()) / makespan,
                            **pct(lat), "service": pct(svc)}
        for frac in (0.5, 0.8, 0.95):
            arr = I.poisson_arrivals(nreq, max_rps * frac, seed=int(100 * frac))
            ans, lat, svc = sv.replay(src, ks, tg, arr, limit_s=1200.0)
            assert np.array_equal(ans, expected)
            span = (float(arr[-1]) + float(lat[-1])) * 1e-9
            out[f"poisson_{int(frac * 100)}pct"] = {
                "offered_requests_per_s": max_rps * frac, "achieved_requests_per_s": nreq / span,
                **pct(lat), "service": pct(svc)}
    # unbatched baseline: one synchronous batch call per request
    m = min(nreq, 2000)
    ds = torch.from_numpy(np.repeat(src[:m], ks[:m]).view(np.int32)).to(dev)
    dt = torch.from_numpy(tg[:int(ks[:m].sum())].view(np.int32)).to(dev)
    dout = torch.empty_like(dt)
    offs = np.concatenate([[0], np.cumsum(ks[:m].astype(np.int64))]).astype(np.int64)
    stream = torch.cuda.Stream()
    lat_u = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(m):
        a, b = int(offs[i]), int(offs[i + 1])
        t1 = time.perf_counter()
        h.query_batch_raw(ds[a:].data_ptr(), dt[a:].data_ptr(), b - a, dout[a:].data_ptr(), None,
                          stream.cuda_stream)
        stream.synchronize()
        lat_u.append((time.perf_counter() - t1) * 1e9)
    span_u = time.perf_counter() - t0
    assert np.array_equal(dout.cpu().numpy().view(np.uint32), expected[:int(ks[:m].sum())])
    out["unbatched_one_call_per_request"] = {"requests_per_s": m / span_u,
                                             **pct(np.array(lat_u))}
    line = {
        "metric": "served queries: requests/s and p50/p99 latency, continuous batching vs one "
                  "batch call per request",
        "config": {"workload": f"{workload}-serve", "vertices": n, "edges": int(g.m),
                   "requests": nreq, "mean_targets_per_request": float(ks.mean()),
                   "one_to_many_fraction": 0.2, "targets_max": 1024,
                   "server_blocks": nblocks, "build_s": st["build_ms"] / 1e3},
        "results": out, "dtype": "u32", "data": "synthetic",
    }
    h.close()
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serve:
        print(json.dumps(serve_bench(args)), flush=True)
        return
    if args.compare_learned:
        print(json.dumps(compare_learned(args)), flush=True)
        return
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2412_18008_gb300 import ch

    n, gseed, qseed, nq = WORKLOADS[args.workload]
    if args.queries is not None:
        nq = args.queries
    g = make_graph(args.workload)
    s_h, t_h = I.random_pairs(n, nq, seed=qseed)
    off_d = torch.from_numpy(g.offsets.view(np.int64)).to(dev)
    tgt_d = torch.from_numpy(g.targets.view(np.int32)).to(dev)
    w_d = torch.from_numpy(g.weights.view(np.int32)).to(dev)
    s_d = torch.from_numpy(s_h.view(np.int32)).to(dev)
    t_d = torch.from_numpy(t_h.view(np.int32)).to(dev)
    out_d = torch.empty(nq, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream

    qcfg = None  # query kernel configuration, chosen by the autotuner during warm-up

    def step():
        h = ch.CH.build(n=n, offsets=off_d, targets=tgt_d, weights=w_d,
                        hop_limit=args.hop_limit, stream=stream, max_candidates_per_vertex=args.cmax,
                        witness_ball_limit=args.witness_ball, witness_memo_limit=args.memo,
                        witness_level_work=args.level_work, witness_prune=args.prune,
                        witness_settle_cap=args.theta)
        if qcfg is not None:
            h.set_query_config(*qcfg)
        if not args.build_only:
            h.query_batch_raw(s_d.data_ptr(), t_d.data_ptr(), nq, out_d.data_ptr(), None, sp)
        return h

    torch.cuda.synchronize()
    tune_ms = None
    for wi in range(args.warmup):
        with torch.cuda.stream(stream):
            h = step()
        stream.synchronize()
        if wi == 0 and not args.no_autotune:
            qcfg, tune_ms = h.autotune_queries(sample=1 << 16, seed=11, stream=stream)
        h.close()

    # timed region
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = ch.kernel_launches()
    step_ms, build_ms, query_ms = [], [], []
    stats = None
    handles = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)  # evict the inputs from L2 (outside the events)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            h = ch.CH.build(n=n, offsets=off_d, targets=tgt_d, weights=w_d,
                            hop_limit=args.hop_limit, stream=stream,
                            max_candidates_per_vertex=args.cmax, witness_ball_limit=args.witness_ball,
                            witness_memo_limit=args.memo, witness_level_work=args.level_work,
                            witness_prune=args.prune,
                            witness_settle_cap=args.theta)
            if qcfg is not None:
                h.set_query_config(*qcfg)
            e1.record(stream)
            if not args.build_only:
                h.query_batch_raw(s_d.data_ptr(), t_d.data_ptr(), nq, out_d.data_ptr(), None, sp)
            e2.record(stream)
        stream.synchronize()
        step_ms.append(e0.elapsed_time(e2))
        build_ms.append(e0.elapsed_time(e1))
        query_ms.append(e1.elapsed_time(e2))
        stats = h.stats()
        handles.append(h)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = ch.kernel_launches() - launches0
    clocks = sampler.stop()
    h_last = handles[-1]
    h_last.query_status(stream)
    q_exp, q_edges = h_last.query_work(stream)  # the last step's batch
    for h in handles[:-1]:
        h.close()

    mean_step = statistics.mean(step_ms)
    mean_build = statistics.mean(build_ms)
    mean_query = statistics.mean(query_ms)
    mean_step, mean_build, mean_query = max_over_ranks([mean_step, mean_build, mean_query], world, dev)

    # per-round profile: the paper observes that most of the work sits in the
    # first rounds; report the split
    rt = h_last.round_times()
    rs = h_last.round_stats()
    k10 = min(10, len(rt))
    round_profile = {
        "rounds": int(len(rt)),
        "ms_first_10_rounds": float(rt[:k10, :5].sum()),
        "ms_other_rounds": float(rt[k10:, :5].sum()),
        "witness_ms_first_10_rounds": float(rt[:k10, 5].sum()),
        "vertices_left_after_10_rounds": int(rs[k10 - 1, 8]) if k10 else 0,
    }

    # search-space size on a sample of the batch (the paper's query iterations)
    samp = min(100_000, nq)
    dd, st = h_last.query(s_d[:samp], t_d[:samp], want_settled=True, stream=stream)
    stream.synchronize()
    mean_ss = float(st.cpu().numpy().view(np.uint32).mean())

    # single-query latency: one-pair batches on an idle GPU, each timed with
    # CUDA events on the stream (outside the timed region)
    latency = query_latency(h_last, s_d, t_d, stream, samples=2000)

    # roofline of the dominant kernel: the query block kernel (k_query_block,
    # one persistent launch per batch of up to 4M queries). Algorithmic bytes
    # per launch: 12 B per expanded frontier entry (its two CSR offsets and
    # its label), 8 B per adjacency entry scanned (id + weight), 20 B per
    # query (source, target, answer, two rank lookups); counted by the kernel.
    peak, peak_src = load_peaks()
    wit_gbs = stats["witness_bytes"] / (stats["witness_ms"] * 1e-3) / 1e9 if stats["witness_ms"] else 0.0
    phases = {k: stats[k] for k in ("normalise_ms", "score_ms", "select_ms", "prep_ms",
                                    "contract_ms", "update_ms", "postprocess_ms")}
    if args.build_only:
        roofline = {
            "kernel": "k_witness (score + contract witness searches)",
            "bound": "hbm", "achieved": round(wit_gbs, 1), "peak": peak, "unit": "GB/s",
            "frac": round(wit_gbs / peak, 4), "traffic": None, "peak_source": peak_src,
            "bytes_per_launch": stats["witness_bytes"] / max(1, stats["witness_launches"]),
            "ms_per_launch": stats["witness_ms"] / max(1, stats["witness_launches"]),
        }
    else:
        # with stalling each expansion also reads the other CSR's two offsets
        stall = bool(qcfg[3]) if qcfg else False
        l2_record = None
        if args.workload == "geo1M" and qcfg is not None and tuple(qcfg) == QUERY_L2_CONFIG:
            l2_peak = l2_read_gbs(dev)
            l2_gbs = QUERY_L2_BYTES_PER_QUERY * nq / (mean_query * 1e-3) / 1e9
            l2_record = {"bytes_per_query": QUERY_L2_BYTES_PER_QUERY, "achieved": round(l2_gbs, 1),
                         "peak": round(l2_peak, 1), "unit": "GB/s", "frac": round(l2_gbs / l2_peak, 4),
                         "peak_source": "measured: float32 sum over a 48 MB L2-resident buffer",
                         "bytes_source": "ncu lts__t_sectors of a 200K-query pass, per query"}
        q_bytes = (20 if stall else 12) * q_exp + 8 * q_edges + 20 * nq
        q_gbs = q_bytes / (mean_query * 1e-3) / 1e9
        roofline = {
            "kernel": "k_query_block (pruned bidirectional upward searches, one launch per batch)",
            "bound": "hbm", "achieved": round(q_gbs, 1), "peak": peak, "unit": "GB/s",
            "frac": round(q_gbs / peak, 4),
            # the captured traffic belongs to this workload in the default
            # configuration (warp layout, 256 threads, small tables, stalling)
            "traffic": (QUERY_TRAFFIC_PER_LAUNCH if args.workload == "geo1M" and nq == 1_000_000
                        and qcfg is not None and tuple(qcfg) == QUERY_L2_CONFIG else None),
            "peak_source": peak_src, "bytes_per_launch": q_bytes, "ms_per_launch": mean_query,
            "launch": "one batch = the small-table pass + its overflow redo (two launches)",
            "expansions_per_query": q_exp / nq, "edges_per_query": q_edges / nq,
            "query_config": {"layout": ["block_flat", "warp_flat"][qcfg[0]] if qcfg else "default",
                             "threads": qcfg[1] if qcfg else None,
                             "small_tables_first": bool(qcfg[2]) if qcfg else None,
                             "stall_on_demand": bool(qcfg[3]) if qcfg else None,
                             "delta": qcfg[4] if qcfg else None,
                             "autotune_ms": [round(float(x), 3) for x in tune_ms] if tune_ms is not None else None},
            "l2": l2_record,
            "witness": {"achieved": round(wit_gbs, 1), "frac": round(wit_gbs / peak, 4),
                        "share_of_build": round(stats["witness_ms"] / mean_build, 3) if mean_build else None},
        }

    # end to end through host buffers (H2D of the CSR and the queries, D2H of
    # the answers, inside the timed region)
    e2e = None
    if not args.no_e2e:
        e2e_build, e2e_q = [], []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh = ch.CH.build(g, hop_limit=args.hop_limit, max_candidates_per_vertex=args.cmax,
                             witness_ball_limit=args.witness_ball, witness_memo_limit=args.memo,
                             witness_level_work=args.level_work, witness_prune=args.prune,
                             witness_settle_cap=args.theta)
            if qcfg is not None:
                hh.set_query_config(*qcfg)
            t1 = time.perf_counter()
            hh.query(s_h, t_h)
            t2 = time.perf_counter()
            e2e_build.append(t1 - t0)
            e2e_q.append(t2 - t1)
            hh.close()
        h2d = g.offsets.nbytes + g.targets.nbytes + g.weights.nbytes + s_h.nbytes + t_h.nbytes
        e2e = {"value": statistics.mean(e2e_build), "unit": "s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(nq * 4),
               "queries_per_s": nq / statistics.mean(e2e_q)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record(args)

    # the other workloads of the method, measured in the same run: the
    # learned priority against the edge difference (1M, trained on 20
    # 256K-vertex graphs) and the server on the 16M-vertex graph
    configs = None
    if rank == 0 and world == 1 and not args.no_configs and args.workload == "geo1M":
        h_last.close()
        handles = []
        configs = {}
        for name, fn in (("modes_geo1M", lambda: modes_record(args, g, off_d, tgt_d, w_d, s_d, t_d, stream)),
                         ("learned_geo1M", lambda: compare_learned(args, steps=3, warmup=1)),
                         ("rmat2M", lambda: rmat_record(args)),
                         ("serve_geo16M", lambda: serve_bench(args, "geo16M", 20_000))):
            t0 = time.perf_counter()
            try:
                configs[name] = fn()
            except Exception as e:  # a side record must not cost the line
                configs[name] = {"error": repr(e)[:300]}
            configs[name]["wall_s"] = round(time.perf_counter() - t0, 1)
            ch.trim_memory()

    if rank == 0:
        line = {
            "metric": METRIC, "value": mean_build / 1000.0, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": mean_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "vertices": n, "edges": int(g.m),
                       "cmax": args.cmax, "witness_ball": args.witness_ball,
                       "witness_memo": args.memo, "witness_level_work": args.level_work,
                       "witness_prune": args.prune, "witness_settle_cap": args.theta,
                       "core_vertices": stats["core_vertices"],
                       "queries": nq, "hop_limit": args.hop_limit,
                       "parallelism": f"replicas{world}",
                       "l2": "flushed before each step (2x L2 buffer write)"},
            "shortcuts": stats["shortcuts"], "rounds": stats["rounds"],
            # every replica answers its own batch: whole-job queries over the
            # slowest rank's batch time
            "queries_per_s": world * nq / (mean_query / 1000.0), "query_batch_ms": mean_query,
            "mean_search_space": mean_ss,
            "query_latency": latency,
            "build_phases_ms": phases,
            "round_profile": round_profile,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "configs": configs,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    if configs is None:
        h_last.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
