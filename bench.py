#!/usr/bin/env python
"""Benchmark: single-source SimRank queries/s at eps = 0.1 on a synthetic R-MAT graph.

Headline workload (one GPU): R-MAT (a,b,c,d) = (.57,.19,.19,.05), n = 2^20, m = 2^24 distinct edges, seeded;
query nodes drawn uniformly from the nodes with in-degree >= 1; c = 0.6, eps = 0.1, delta = 0.01
(n_r = 3,325), deterministic PROBE, FP32 scores.  A step is one single-source query through the C ABI
(walks, tree, level loop, estimates), queries run one at a time; L2 is flushed between steps (outside the
timed events).  Also reported, each on its own line of the JSON object:
  batched      the same queries in calls of 2, 4 and 8, against the same queries one at a time
  switch       the Sec. 4.4 switch (c0 = 0.01) on the same graph, one at a time and in calls of 8
  mixed_eps_topk  R-MAT 2^22 (m = 2^26): 256 queries in one top-50 call, eps 0.1 / 0.05 alternating
               (n_r 3,574 / 14,296), switch mode
  serving      Poisson arrivals into the continuous-batching server at rates bracketing its capacity, top-k
               with k uniform over {10, 50, 100}, one window with edge-update batches every 100 ms
  serving_2p23 R-MAT 2^23 (m = 2^27), eps uniform over {0.1, 0.05, 0.025}, switch mode, update batches of
               10k edges every 100 ms, Poisson rates bracketing capacity
  billion_edge_topk  R-MAT 2^25 with 10^9 edges, drawn and built on the GPU: top-50 in calls of 64 queries at
               eps = 0.1, switch mode
  accuracy_pooling  Precision@50, NDCG@50 and Kendall tau of each engine's top-50 lists against a pooled ground
               truth gauged by the GPU pairwise Monte Carlo (Sec. 6's large-graph protocol)
  e2e          the headline with host output buffers (the scores copied back inside the timed region)
  roofline     the PROBE level kernel's achieved bandwidth against the measured HBM copy peak
  cpu_baseline the FP64 oracle on every host core, on a bounded sample of the headline workload
The timed steps run with profiling off; per-phase times and the pull's own duration come from a second,
profiled pass over the first (up to ten) queries, in which the level loop runs on one stream.

``--impl reference`` times the CPU oracle (the reference implementation of this build) on the same
workload and metric, on every host core.  Multi-GPU runs (torchrun) are replicas: each rank owns a copy of the
graph and its own share of queries, with no collective on the data path.
"""
import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("single-source SimRank queries/sec @ε=0.1 (batched serving vs 1-at-a-time), p50/p99 ms, HBM GB/s")
WORKLOAD = "rmat-20"
EPS = 0.1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batches", default="2,4,8", help="queries per call in the batched legs")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-walks-per-core", type=int, default=2, help="CPU-baseline sample size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-rates", default="10,20,30,35,40,50",
                    help="Poisson arrival rates of the serving sweep on the headline graph (q/s)")
    ap.add_argument("--serve-update-rate", type=float, default=20.0,
                    help="rate of the serving window with edge-update batches (0 = none)")
    ap.add_argument("--serve-updates", type=int, default=10000, help="edges per update batch, one batch per 100 ms")
    ap.add_argument("--serve-workers", type=int, default=3, help="server workers (concurrent batch pipelines)")
    ap.add_argument("--serve-max-batch", type=int, default=2, help="largest batch a server worker takes")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="arrival window of each serving rate")
    ap.add_argument("--switch-c0", type=float, default=0.01, help="c0 of the switch legs (Sec. 4.4)")
    ap.add_argument("--mixed-batch", type=int, default=256,
                    help="queries of the mixed-eps top-50 call on R-MAT 2^22 (0 = off)")
    ap.add_argument("--serve23-rates", default="2,4,6,8,10,20",
                    help="arrival rates of the serving leg on R-MAT 2^23 (empty = off); capacity is near 9 q/s, so "
                         "10 and 20 (the low end of the configuration's sweep) show the queue building")
    ap.add_argument("--serve23-seconds", type=float, default=5.0)
    ap.add_argument("--billion-batches", type=int, default=16,
                    help="calls of 64 top-50 queries on R-MAT 2^25 with 10^9 edges (0 = off; 16 = 1,024 queries)")
    ap.add_argument("--billion-edges", type=float, default=1e9, help="edges of that graph")
    ap.add_argument("--accuracy-queries", type=int, default=5, help="queries of the pooling accuracy leg (0 = off)")
    ap.add_argument("--profile-case", choices=["frontier", "billion", "pull"], default=None,
                    help="run one fixed case for an ncu capture and exit (see profile_case)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_query_id(rank, i):
    """Query id (and Philox key) of the i-th query of a rank: the ranks of a replica run draw disjoint ids."""
    return rank * 100003 + i


def whole_job_rate(local_ms, steps, world, device=None):
    """Whole-job queries/s of a replica run: every rank timed `steps` queries in `local_ms`; the job's time is
    the slowest rank's (a max over ranks), and the job processed world * steps queries."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
    return world * steps / (local_ms / 1e3), local_ms


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001 -- file absent on some boxes
        return 6800.0, "fallback"


def recorded_pull_counters():
    """From the committed ncu summary of the PROBE level kernel, valid only while the kernel source is unchanged
    since the captures (checked by its hash): the full-size DRAM / algorithmic byte ratio, and the share of its
    L1 data pipe's wavefront peak it used (the unit that bounds it).  (None, None) when absent or stale."""
    import hashlib
    src = os.path.join(ROOT, "paper_1709_06955_gb300", "csrc", "pull.cu")
    summ = os.path.join(ROOT, "profiles", "k_pull_traffic.txt")
    ratio = pipe = None
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(summ):
            parts = line.split()
            if len(parts) >= 3 and parts[2] == h:
                if parts[0] == "ratio":
                    ratio = float(parts[1])
                elif parts[0] == "l1pipe":
                    pipe = float(parts[1])
    except Exception:  # noqa: BLE001
        pass
    return ratio, pipe


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:  # noqa: BLE001 -- no nvidia-smi
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(getattr(self, "out", ""))) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def describe_workload(name, n, m):
    """The workload's text for the JSON line, from its name and actual sizes."""
    import math
    kind = "R-MAT (.57,.19,.19,.05)" if name.startswith("rmat") else "Chung-Lu (exponent 2.1)"
    return "%s n=2^%d m=%d seed 1, eps=%g delta=0.01 c=0.6" % (kind, int(round(math.log2(n))), m, EPS)


def load_workload(name):
    from paper_1709_06955_gb300 import synth
    n, s, d = synth.config_graph(name)
    qs = synth.queries(n, d, 100, seed=2)
    return n, s, d, qs


def oracle_sample_rate(O, qs, nr, walks, budget_s=None, threads=None):
    """The oracle (Alg. 1, FP64) on a bounded sample of a workload, on every host core: the samples are walks
    0..walks-1 of each query in ``qs`` (a walk k of query u is Alg. 1 restricted to walk k, weighted 1/n_r), run
    by one thread per core (the C oracle releases the GIL, so the threads run in parallel); with ``budget_s``, no
    walk starts after the budget.  Returns (queries/s = walks/s / n_r, walks done, seconds, threads)."""
    import concurrent.futures
    threads = threads or len(os.sched_getaffinity(0))
    items = [(t, k) for k in range(walks) for t in range(len(qs))]
    lock = threading.Lock()
    it = iter(items)
    done = [0]
    t0 = time.perf_counter()

    def work():
        while True:
            with lock:
                if budget_s is not None and time.perf_counter() - t0 >= budget_s:
                    return
                nxt = next(it, None)
            if nxt is None:
                return
            t, k = nxt
            O.single_source(int(qs[t]), eps=EPS, seed=3, qid=t, walk_begin=k, walk_end=k + 1)
            with lock:
                done[0] += 1

    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        for f in [ex.submit(work) for _ in range(threads)]:
            f.result()
    el = time.perf_counter() - t0
    return done[0] / el / nr, done[0], el, threads


def cpu_baseline(n, s, d, qs, walks_per_core):
    """The oracle on every host core over a fixed sample of the headline workload: walks 0..K-1 of 4 queries,
    K = walks_per_core * cores / 4, every walk run to the end (no time cut-off, which would keep the short walks
    and bias the rate); queries/s extrapolated from walks/s and n_r."""
    from oracle import build as obuild, core
    obuild.build()
    O = core.Graph(n, s, d)
    nr = core.num_walks(0.6, EPS, 0.01, n)
    th = len(os.sched_getaffinity(0))
    K = max(1, (walks_per_core * th + 3) // 4)
    rate, k, el, th = oracle_sample_rate(O, qs[:4], nr, K, threads=th)
    return {"value": rate, "unit": "queries/s", "cores": th, "kind": "oracle",
            "sample": "walks 0..%d of 4 queries (%d walks, n_r=%d each) on the %d-node graph, Alg. 1 FP64, one "
                      "thread per host core, %.1f s; queries/s = walks/s / n_r (extrapolated)" % (K - 1, k, nr, n, el)}


def serving_leg(probesim, G, n, src, dst, qs, rates, seconds, updates_per_tick, rank, workers=3, max_batch=2,
                eps_choices=(EPS,), seed_base=4, qid_base=900000):
    """For each arrival rate: queries arrive as a Poisson process for `seconds` into a fresh continuous-batching
    server (top-k, k uniform over {10, 50, 100}, eps uniform over eps_choices), while every 100 ms an update
    batch of updates_per_tick edges (half random inserts, half deletes of edges of the original graph) enters
    the same FIFO.  Returns one record per rate: throughput, p50/p99 latency, mean batch size, updates applied."""
    import numpy as np
    rng = np.random.default_rng(seed_base + rank)
    out = []
    for rate in rates:
        S = probesim.Server(G, workers=workers, max_batch=max_batch, kmax=100)
        gaps = rng.exponential(1.0 / rate, size=int(rate * seconds * 3) + 10)
        arrivals = np.cumsum(gaps)
        arrivals = arrivals[arrivals < seconds]
        ks = np.array([10, 50, 100])[rng.integers(0, 3, arrivals.size)]
        es = np.array(eps_choices)[rng.integers(0, len(eps_choices), arrivals.size)]
        ticks = np.arange(0.0, seconds, 0.1) if updates_per_tick > 0 else np.zeros(0)
        events = sorted([(t, 0, i) for i, t in enumerate(arrivals)] + [(t, 1, j) for j, t in enumerate(ticks)])
        half = updates_per_tick // 2
        t0 = time.perf_counter()
        done = 0
        for ta, kind, i in events:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            if kind == 0:
                S.submit(probesim.make_queries([qs[i % len(qs)]], eps=float(es[i]), k=int(ks[i]),
                                               query_ids=[qid_base + i]))
            else:
                S.update(rng.integers(0, n, half), rng.integers(0, n, half), insert=True)
                pick = rng.integers(0, src.size, half)
                S.update(src[pick], dst[pick], insert=False)
            done += len(S.poll(64, wait_ms=0))
        while done < arrivals.size:
            done += len(S.poll(64, wait_ms=500))
        st = S.stats()
        S.close()
        out.append({"arrival_rate_qps": rate, "queries": int(arrivals.size), "qps": st["qps"], "p50_ms": st["p50_ms"],
                    "p99_ms": st["p99_ms"], "mean_batch": st["mean_batch"], "update_batches": st["updates_applied"],
                    "edges_per_update_tick": updates_per_tick, "workers": workers, "max_batch": max_batch,
                    "k": "uniform {10, 50, 100}", "eps": "uniform {%s}" % ", ".join("%g" % e for e in eps_choices)})
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import build as obuild, core
    obuild.build()
    n, s, d, qs = load_workload(args.workload)
    O = core.Graph(n, s, d)
    nr = core.num_walks(0.6, EPS, 0.01, n)
    threads = len(os.sched_getaffinity(0))
    # a step: one walk per host core (Alg. 1 restricted to that walk), walks taken in order over 4 queries
    oracle_sample_rate(O, qs[:4], nr, max(1, (args.warmup * threads + 3) // 4), threads=threads)
    walks = max(1, (args.steps * threads + 3) // 4)
    rate, k, el, th = oracle_sample_rate(O, qs[:4], nr, walks, threads=threads)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe_workload(args.workload, n, len(s)),
                       "step": "one walk per host core (Alg. 1 on it), queries/s = walks/s / n_r"},
            "cpu_baseline": {"value": rate, "unit": "queries/s", "cores": th, "kind": "oracle",
                             "sample": "%d walks: walks 0..%d of 4 queries (n_r=%d each), one thread per core"
                                       % (k, walks - 1, nr)},
            "e2e": {"value": rate, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_calls(G, calls, out, stream, flush):
    """CUDA-event milliseconds of each call (L2 flushed before each, outside the events)."""
    import torch
    ms = []
    for q in calls:
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.single_source(q, out=out, stream=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_06955_gb300 import build, probesim, synth
    build.build()
    n, s, d, qs = load_workload(args.workload)
    G = probesim.Graph(n, s, d)
    tuning = G.autotune()  # launch shape of the pull kernel, chosen on this graph before timing
    nr_headline = G.num_walks(EPS)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    nq = len(qs)

    def query(i, **kw):
        j = replica_query_id(rank, i)
        return probesim.make_queries([qs[j % nq]], eps=kw.get("eps", EPS), k=50, query_ids=[j])

    def qbatch(i0, B):
        ids = [replica_query_id(rank, i0 + j) for j in range(B)]
        return probesim.make_queries([qs[j % nq] for j in ids], eps=EPS, query_ids=ids)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 129 MB L2
    out = torch.zeros((1, n), dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    for i in range(args.warmup):
        G.single_source(query(i), out=out, stream=sptr)
    torch.cuda.synchronize(dev)

    # timed: K queries one at a time, device-resident output (profiling off: the path a caller gets)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    agg = {"probe_bytes": 0.0, "probe_launches": 0, "kernel_launches": 0, "edge_gathers": 0,
           "vectors": 0, "tree_nodes": 0, "walks": 0}
    with ClockSampler(local) as clk:
        barrier()
        w0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            G.single_source(query(args.warmup + i), out=out, stream=sptr)
            evs[i][1].record(stream)
            st = G.stats()  # describes the last call
            for k in agg:
                agg[k] += st[k]
        barrier()
        wall = time.perf_counter() - w0
    lat = [a.elapsed_time(b) for a, b in evs]
    value, tot_ms = whole_job_rate(sum(lat), args.steps, world, dev)

    # profiled pass over the first queries again: per-phase CUDA-event times and the pull's own duration
    # (profiling records events around every launch and runs the level loop on one stream)
    G.set_profiling(True)
    np_ = min(args.steps, 10)
    prof = {"probe_ms": 0.0, "probe_bytes": 0.0, "probe_launches": 0, "edge_gathers": 0, "step_ms": 0.0}
    phases = {}
    for i in range(np_):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.single_source(query(args.warmup + i), out=out, stream=sptr)
        b.record(stream)
        st = G.stats()
        b.synchronize()
        prof["step_ms"] += a.elapsed_time(b)
        for k in ("probe_ms", "probe_bytes", "probe_launches", "edge_gathers"):
            prof[k] += st[k]
        for k, v in st["phase_ms"].items():
            phases[k] = phases.get(k, 0.0) + v
    G.set_profiling(False)
    torch.cuda.synchronize(dev)

    # batched legs: the timed leg's queries again, B per call, against the same queries one at a time
    batched = []
    for B in [int(x) for x in args.batches.split(",") if x]:
        nb = max(1, args.steps // B)
        outb = torch.zeros((B, n), dtype=torch.float32, device=dev)
        calls = [qbatch(args.warmup + i * B, B) for i in range(nb)]
        G.single_source(calls[0], out=outb, stream=sptr)
        barrier()
        bms = sum(timed_calls(G, calls, outb, stream, flush))
        barrier()
        batched.append({"batch": B, "value": nb * B / (bms / 1e3), "unit": "queries/s", "calls": nb,
                        "queries": nb * B, "same_queries_one_at_a_time": nb * B / (sum(lat[:nb * B]) / 1e3)})
        del outb
    best = max(batched, key=lambda r: r["value"]) if batched else None

    # top-50 lists of a few queries from each engine, for the pooling accuracy leg below
    acc_nodes = [qs[replica_query_id(rank, 7000 + j) % nq] for j in range(args.accuracy_queries)]
    acc_q = probesim.make_queries(acc_nodes, eps=EPS, k=50,
                                  query_ids=[replica_query_id(rank, 7000 + j) for j in range(len(acc_nodes))])
    acc_lists = {}
    if acc_nodes:
        acc_lists["deterministic"] = G.topk(acc_q, kmax=50)[0]

    # the switch of Sec. 4.4 on the same graph: a few queries one at a time and in calls of 8
    GS = probesim.Graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=args.switch_c0)
    GS.single_source(query(0), out=out, stream=sptr)
    sq = min(args.steps, 40)
    sw_ms = timed_calls(GS, [query(args.warmup + i) for i in range(sq)], out, stream, flush)
    sst = GS.stats()
    out8 = torch.zeros((8, n), dtype=torch.float32, device=dev)
    n8 = max(1, sq // 8)
    sw8_ms = timed_calls(GS, [qbatch(args.warmup + 8 * i, 8) for i in range(n8)], out8, stream, flush)
    switch = {"c0": args.switch_c0, "eps": EPS, "value": sq / (sum(sw_ms) / 1e3), "unit": "queries/s", "queries": sq,
              "batched8_value": 8 * n8 / (sum(sw8_ms) / 1e3),
              "last_query": {k: sst[k] for k in ("probes", "switched", "edge_gathers", "levels", "max_table_slots")}}
    if acc_nodes:
        acc_lists["switch c0=%g" % args.switch_c0] = GS.topk(acc_q, kmax=50)[0]
        # the same queries at eps / 4 (16 times the walks): how far the lists' order is set by the estimates' noise
        acc_fine = probesim.make_queries(acc_nodes, eps=EPS / 4, k=50,
                                         query_ids=[replica_query_id(rank, 7000 + j) for j in range(len(acc_nodes))])
        acc_lists["switch c0=%g eps=%g" % (args.switch_c0, EPS / 4)] = GS.topk(acc_fine, kmax=50)[0]
    GS.close()
    del out8

    # randomized PROBE (Alg. 3) on the same graph: a few queries one at a time
    GR = probesim.Graph(n, s, d, probe_mode=probesim.PROBE_RANDOMIZED)
    rq = 10
    GR.single_source(query(0), out=out, stream=sptr)
    rand_ms = timed_calls(GR, [query(args.warmup + i) for i in range(rq)], out, stream, flush)
    rst = GR.stats()
    if acc_nodes:
        acc_lists["randomized"] = GR.topk(acc_q, kmax=50)[0]
    GR.close()
    randomized = {"value": rq / (sum(rand_ms) / 1e3), "unit": "queries/s", "queries": rq,
                  "candidates_last_query": rst["edge_gathers"], "levels_last_query": rst["levels"]}

    # accuracy by pooling (Sec. 6, large graphs): each query's top-50 lists of the three engines are merged, every
    # pooled node gauged by the GPU pairwise Monte Carlo, and the best 50 taken as the ground truth
    accuracy = None
    if acc_nodes:
        from paper_1709_06955_gb300 import accuracy as A
        t0 = time.perf_counter()
        per = {m: [] for m in acc_lists}
        pool_sizes, ranks = [], []
        for t, u in enumerate(acc_nodes):
            truth, score = A.pool(G, int(u), [acc_lists[m][t] for m in acc_lists], 50, eps=2e-4, delta=1e-4,
                                  key_base=(1 << 30) + 4096 * t)
            pool_sizes.append(len(score))
            ranks.append([score[int(truth[i])] for i in (0, 9, min(49, len(truth) - 1))])
            for m in acc_lists:
                per[m].append(A.evaluate(acc_lists[m][t], truth, lambda v, sc=score: sc.get(v, 0.0)))
        accuracy = {"queries": len(acc_nodes), "k": 50, "eps": EPS,
                    "expert": "pairwise Monte Carlo on the GPU, eps 2e-4, delta 1e-4 (%d walk pairs per node)"
                              % A.mc_walk_pairs(2e-4, 1e-4),
                    "mean_pool": float(np.mean(pool_sizes)), "seconds": time.perf_counter() - t0,
                    "truth_scores_at_rank_1_10_50": [float(x) for x in np.mean(np.array(ranks), axis=0)],
                    "methods": {m: {k: float(np.mean([r[k] for r in per[m]])) for k in ("precision", "ndcg", "tau")}
                                for m in per}}

    # end-to-end through the C ABI with host buffers: query struct in, pinned host scores out.  Each call is timed
    # on the host from its start to its return (the call synchronises); the L2 flush between calls is outside.
    host_out = torch.empty((1, n), dtype=torch.float32, pin_memory=True)
    e2e_steps = args.steps
    barrier()
    e2e_s = 0.0
    for i in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0 = time.perf_counter()
        G.single_source(query(args.warmup + i), out=host_out, stream=sptr)
        e2e_s += time.perf_counter() - e0
    barrier()
    e2e_qps = e2e_steps / e2e_s

    # serving sweep on the headline graph (last for this graph: the update window changes it)
    rates = [float(r) for r in args.serve_rates.split(",") if r]
    serving = serving_leg(probesim, G, n, s, d, qs, rates, args.serve_seconds, 0, rank, args.serve_workers,
                          args.serve_max_batch)
    if args.serve_update_rate > 0:
        serving += serving_leg(probesim, G, n, s, d, qs, [args.serve_update_rate], args.serve_seconds,
                               args.serve_updates, rank, args.serve_workers, args.serve_max_batch)
    G.close()
    torch.cuda.synchronize(dev)

    # R-MAT 2^22: 256 queries in one top-50 call, eps alternating 0.1 / 0.05 (uneven n_r), switch mode
    mixed = None
    if args.mixed_batch > 0:
        n22, s22, d22 = synth.rmat_device(22, 16 << 22, seed=1, device=dev)
        torch.cuda.empty_cache()  # the generator's scratch goes back to the device before the library allocates
        q22 = synth.queries(n22, d22, args.mixed_batch, seed=2)
        t0 = time.perf_counter()
        G22 = probesim.Graph(n22, s22, d22, probe_mode=probesim.PROBE_SWITCH, c0=args.switch_c0)
        create_s = time.perf_counter() - t0
        MB = args.mixed_batch
        eps_mix = [EPS if j % 2 == 0 else EPS / 2 for j in range(MB)]
        mids = torch.empty((MB, 50), dtype=torch.int32, device=dev)
        mvals = torch.empty((MB, 50), dtype=torch.float32, device=dev)
        G22.topk(probesim.make_queries(q22[:8], eps=EPS, k=50, query_ids=np.arange(8) + 70000), kmax=50,
                 ids=mids[:8], vals=mvals[:8], stream=sptr)  # warm-up
        Qm = probesim.make_queries(q22, eps=eps_mix, k=50, query_ids=[replica_query_id(rank, 5000 + j) for j in range(MB)])
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G22.topk(Qm, kmax=50, ids=mids, vals=mvals, stream=sptr)
        b.record(stream)
        barrier()
        mms = a.elapsed_time(b)
        mst = G22.stats()
        mixed = {"graph": "R-MAT (.57,.19,.19,.05) n=2^22 m=%d (drawn on the GPU), seed 1" % int(s22.numel()),
                 "queries": MB, "calls": 1, "eps": "%g / %g alternating" % (EPS, EPS / 2), "k": 50,
                 "probe": "switch (Sec. 4.4), c0=%g" % args.switch_c0, "value": MB / (mms / 1e3),
                 "unit": "queries/s", "ms": mms, "graph_create_s": create_s,
                 "n_r": [int(G22.num_walks(EPS)), int(G22.num_walks(EPS / 2))],
                 "probes": mst["probes"], "switched": mst["switched"], "det_edge_pushes": mst["edge_gathers"]}
        G22.close()
        del n22, s22, d22, mids, mvals
        torch.cuda.empty_cache()

    # serving on R-MAT 2^23: eps uniform over {0.1, 0.05, 0.025}, k over {10, 50, 100}, switch mode, 10k-edge
    # update batches every 100 ms
    serving23 = None
    r23 = [float(r) for r in args.serve23_rates.split(",") if r]
    if r23:
        n23, s23, d23 = synth.rmat_device(23, 16 << 23, seed=1, device=dev)
        torch.cuda.empty_cache()
        q23 = synth.queries(n23, d23, 1000, seed=2)
        G23 = probesim.Graph(n23, s23, d23, probe_mode=probesim.PROBE_SWITCH, c0=args.switch_c0)
        s23h, d23h = s23.cpu().numpy(), d23.cpu().numpy()
        del s23, d23
        G23.single_source(probesim.make_queries(q23[:1], eps=EPS, query_ids=[1]), out=torch.zeros((1, n23), device=dev))
        serving23 = serving_leg(probesim, G23, n23, s23h, d23h, q23, r23, args.serve23_seconds, args.serve_updates,
                                rank, args.serve_workers, args.serve_max_batch, eps_choices=(0.1, 0.05, 0.025),
                                seed_base=40, qid_base=800000)
        G23.close()
        del s23h, d23h
        torch.cuda.empty_cache()

    # R-MAT 2^25 with 10^9 edges, built on the device: top-50 in calls of 64 queries at eps 0.1, switch mode (the
    # randomized PROBE takes the high-degree frontiers)
    billion = None
    if args.billion_batches > 0:
        t0 = time.perf_counter()
        n25, s25, d25 = synth.rmat_device(25, int(args.billion_edges), seed=1, device=dev)
        torch.cuda.synchronize(dev)
        gen_s = time.perf_counter() - t0
        torch.cuda.empty_cache()
        BB = 64
        q25 = synth.queries(n25, d25, BB * args.billion_batches, seed=2)
        t0 = time.perf_counter()
        G25 = probesim.Graph(n25, s25, d25, probe_mode=probesim.PROBE_SWITCH, c0=args.switch_c0)
        torch.cuda.synchronize(dev)
        create_s = time.perf_counter() - t0
        m25 = G25.info()[1]
        del s25, d25
        torch.cuda.empty_cache()
        bids = torch.empty((BB, 50), dtype=torch.int32, device=dev)
        bvals = torch.empty((BB, 50), dtype=torch.float32, device=dev)
        G25.topk(probesim.make_queries(q25[:4], eps=EPS, k=50, query_ids=np.arange(4) + 95000), kmax=50,
                 ids=bids[:4], vals=bvals[:4], stream=sptr)  # warm-up
        barrier()
        bms = []
        for bi in range(args.billion_batches):
            Qb = probesim.make_queries(q25[bi * BB:(bi + 1) * BB], eps=EPS, k=50,
                                       query_ids=[replica_query_id(rank, 900000 + bi * BB + j) for j in range(BB)])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G25.topk(Qb, kmax=50, ids=bids, vals=bvals, stream=sptr)
            b.record(stream)
            b.synchronize()
            bms.append(a.elapsed_time(b))
        barrier()
        bst = G25.stats()
        billion = {"graph": "R-MAT (.57,.19,.19,.05) n=2^25 m=%d (drawn on the GPU), seed 1" % m25,
                   "queries": BB * args.billion_batches, "calls": args.billion_batches, "batch": BB, "eps": EPS,
                   "k": 50, "probe": "switch (Sec. 4.4), c0=%g" % args.switch_c0,
                   "value": BB * len(bms) / (sum(bms) / 1e3), "unit": "queries/s", "ms_per_call": bms,
                   "n_r": int(G25.num_walks(EPS)), "generate_s": gen_s, "graph_create_s": create_s,
                   "probes": bst["probes"], "switched": bst["switched"]}
        G25.close()
        del bids, bvals
        torch.cuda.empty_cache()

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return 0

    peak, peak_kind = measured_peak_hbm()
    # the pull's roofline, from the profiled pass (CUDA events around every pull launch)
    achieved = prof["probe_bytes"] / (prof["probe_ms"] / 1e3) / 1e9 if prof["probe_ms"] > 0 else None
    ratio, l1pipe = recorded_pull_counters()
    per_launch = prof["probe_bytes"] / max(1, prof["probe_launches"])
    roof = {"kernel": "k_pull (PROBE level pull, pull.cu)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "peak_kind": peak_kind + " hbm_gbs (copy)", "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": (ratio * per_launch) if ratio else None,
            "algorithmic_bytes_per_launch": per_launch, "launches": prof["probe_launches"],
            "profiled_queries": np_,
            "kernel_ms_share_of_step": prof["probe_ms"] / prof["step_ms"] if prof["step_ms"] else None,
            "l2_gather_GBps": 4.0 * prof["edge_gathers"] / (prof["probe_ms"] / 1e3) / 1e9 if prof["probe_ms"] else None,
            "binding_unit": {"unit": "L1 data-pipe wavefronts (ncu, profiles/k_pull_rmat18_one_query.md)",
                             "frac": l1pipe}}
    lat_sorted = sorted(lat)

    def pct(p):
        return lat_sorted[min(len(lat_sorted) - 1, int(round(p / 100.0 * (len(lat_sorted) - 1))))]

    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe_workload(args.workload, n, len(s)) +
                                   " (n_r=%d), deterministic PROBE, one query per call" % nr_headline,
                       "queries": "uniform over nodes with in-degree >= 1", "l2": "flushed between steps (256 MB write)",
                       "pull_tuning": tuning,
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "p50_ms": pct(50), "p99_ms": pct(99), "wall_s": wall,
            "batched": {"best": best, "sweep": batched},
            "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": 32, "d2h_bytes_per_step": 4 * n,
                    "steps": e2e_steps},
            "roofline": roof, "clocks": clk.summary(), "gpu_launches": agg["kernel_launches"],
            "phases_ms_per_query": {k: v / np_ for k, v in phases.items()},
            "profiled_ms_per_query": prof["step_ms"] / np_,
            "switch": switch,
            "randomized_probe": randomized,
            "accuracy_pooling": accuracy,
            "mixed_eps_topk": mixed,
            "serving": serving,
            "serving_2p23": serving23,
            "billion_edge_topk": billion,
            "work": {"walks_per_query": agg["walks"] / args.steps, "tree_nodes_per_query": agg["tree_nodes"] / args.steps,
                     "vectors_per_query": agg["vectors"] / args.steps,
                     "edge_gathers_per_query": agg["edge_gathers"] / args.steps}}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n, s, d, qs, args.cpu_walks_per_core)
    if world > 1:
        torch.distributed.barrier()
    print(json.dumps(line), flush=True)
    return 0


def profile_case(args):
    """A small, fixed invocation of one engine for kernel captures (no timing, no JSON line).

    frontier: R-MAT 2^20 drawn on the GPU, switch mode c0 = 0.01, two calls of four queries at eps = 0.1.
    billion:  R-MAT 2^25 with 10^9 edges drawn and built on the GPU, switch mode c0 = 0.01, one call of 64 top-50
              queries at eps = 0.1 (the billion-edge leg's call).
    pull:     R-MAT 2^18 (the host generator, m = 2^22), deterministic PROBE with the full tiles pinned to single
              32-column tiles at 8 blocks per SM (no tuner, so a capture does not depend on timings taken under a
              profiler), two queries at eps = 0.1 one per call."""
    import numpy as np
    import torch
    from paper_1709_06955_gb300 import build, probesim, synth
    build.build()
    if args.profile_case == "pull":
        n, s, d = synth.config_graph("rmat-18")
        qs = synth.queries(n, d, 2, seed=2)
        G = probesim.Graph(n, s, d)
        G.set_tuning(32, [16, 16, 16, 16, 16, 8, 3, 1])
        out = torch.zeros((1, n), dtype=torch.float32, device="cuda")
        for i in range(2):
            G.single_source(probesim.make_queries(qs[i:i + 1], eps=EPS, query_ids=[i]), out=out)
    elif args.profile_case == "billion":
        n, s, d = synth.rmat_device(25, int(args.billion_edges), seed=1)
        torch.cuda.empty_cache()
        qs = synth.queries(n, d, 64, seed=2)
        G = probesim.Graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.01)
        del s, d
        torch.cuda.empty_cache()
        ids = torch.empty((64, 50), dtype=torch.int32, device="cuda")
        vals = torch.empty((64, 50), dtype=torch.float32, device="cuda")
        G.topk(probesim.make_queries(qs, eps=EPS, k=50, query_ids=np.arange(64) + 900000), kmax=50, ids=ids, vals=vals)
    else:
        n, s, d = synth.rmat_device(20, 16 << 20, seed=1)
        torch.cuda.empty_cache()
        qs = synth.queries(n, d, 8, seed=2)
        G = probesim.Graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.01)
        out = torch.zeros((4, n), dtype=torch.float32, device="cuda")
        for i in range(2):
            G.single_source(probesim.make_queries(qs[4 * i:4 * i + 4], eps=EPS, query_ids=np.arange(4) + 4 * i),
                            out=out)
    torch.cuda.synchronize()
    st = G.stats()
    print("profile case %s done: %d deterministic edge pushes, %d levels, %d of %d probes switched"
          % (args.profile_case, st["edge_gathers"], st["levels"], st["switched"], st["probes"]))
    return 0


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
