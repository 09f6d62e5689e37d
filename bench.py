#!/usr/bin/env python
"""Benchmark: single-source SimRank queries/s at eps = 0.1 on a synthetic R-MAT graph.

Workload (one GPU): R-MAT (a,b,c,d) = (.57,.19,.19,.05), n = 2^20, m = 2^24 distinct edges, seeded; query
nodes drawn uniformly from the nodes with in-degree >= 1; c = 0.6, eps = 0.1, delta = 0.01 (n_r = 3,325),
deterministic PROBE, FP32 scores.  A step is one single-source query through the C ABI (walks, tree,
level loop, estimates), queries run one at a time; L2 is flushed between steps (outside the timed events).
Also reported: the same queries in batches, the end-to-end number with host buffers, p50/p99 latency,
the PROBE level kernel's achieved bandwidth against the measured HBM copy peak, and the CPU oracle on a
bounded sample of the same workload.  The timed steps run with profiling off; per-phase times and the
pull's own duration come from a second, profiled pass over the first (up to ten) queries, in which the
level loop runs on one stream.

``--impl reference`` times the CPU oracle (the reference implementation of this build) on the same
workload and metric.  Multi-GPU runs (torchrun) are replicas: each rank owns a copy of the graph and its
own share of queries, with no collective on the data path.
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
    ap.add_argument("--batch", type=int, default=8, help="queries per call in the batched leg")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-rates", default="12,60", help="Poisson arrival rates of the serving leg (q/s), comma-separated")
    ap.add_argument("--serve-updates", type=int, default=10000, help="edges per update batch, one batch per 100 ms")
    ap.add_argument("--serve-plain-rate", type=float, default=60.0,
                    help="an extra serving window at this rate without updates (0 = none)")
    ap.add_argument("--serve-workers", type=int, default=3, help="server workers (concurrent batch pipelines)")
    ap.add_argument("--serve-max-batch", type=int, default=2, help="largest batch a server worker takes")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="arrival window of the serving leg")
    ap.add_argument("--mixed-batch", type=int, default=0,
                    help="queries of the optional mixed-eps top-k leg (eps 0.1 / 0.05 alternating, k = 50); 0 = off")
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


def recorded_traffic():
    """DRAM bytes / algorithmic bytes of the PROBE level kernel from the committed ncu summary, valid only
    while the kernel source is unchanged since the capture (checked by its hash)."""
    import hashlib
    src = os.path.join(ROOT, "paper_1709_06955_gb300", "csrc", "pull.cu")
    summ = os.path.join(ROOT, "profiles", "k_pull_traffic.txt")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(summ):
            if line.startswith("ratio "):
                _, ratio, src_hash = line.split()[:3]
                if src_hash == h:
                    return float(ratio)
    except Exception:  # noqa: BLE001
        pass
    return None


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


def cpu_baseline(n, s, d, qs, budget_s):
    """The oracle (Alg. 1, FP64, one thread) on walks 0, 1, 2, ... of query 0 until budget_s has passed;
    queries/s extrapolated from the time per walk."""
    from oracle import build as obuild, core
    obuild.build()
    O = core.Graph(n, s, d)
    nr = core.num_walks(0.6, EPS, 0.01, n)
    u = int(qs[0])
    t0 = time.perf_counter()
    k = 0
    while True:
        O.single_source(u, eps=EPS, seed=3, qid=0, walk_begin=k, walk_end=k + 1)
        k += 1
        el = time.perf_counter() - t0
        if el >= budget_s or k >= 256:
            break
    per_walk = el / k
    return {"value": 1.0 / (per_walk * nr), "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": "walks 0..%d of 1 query (of n_r=%d) on %s, Alg. 1 FP64 single-threaded, %.1f s; "
                      "queries/s extrapolated from the time per walk" % (k - 1, nr, "%d-node graph" % n, el)}


def serving_leg(probesim, G, n, src, dst, qs, rates, seconds, updates_per_tick, rank, workers=3, max_batch=2):
    """For each arrival rate: queries arrive as a Poisson process for `seconds` into a fresh continuous-batching
    server (top-k, k uniform over {10, 50, 100}), while every 100 ms an update batch of updates_per_tick edges
    (half random inserts, half deletes of edges of the original graph) enters the same FIFO.  Returns one
    record per rate: throughput, p50/p99 latency, mean batch size, updates applied."""
    import numpy as np
    rng = np.random.default_rng(4 + rank)
    out = []
    for rate in rates:
        S = probesim.Server(G, workers=workers, max_batch=max_batch, kmax=100)
        gaps = rng.exponential(1.0 / rate, size=int(rate * seconds * 3) + 10)
        arrivals = np.cumsum(gaps)
        arrivals = arrivals[arrivals < seconds]
        ks = np.array([10, 50, 100])[rng.integers(0, 3, arrivals.size)]
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
                S.submit(probesim.make_queries([qs[i % len(qs)]], eps=EPS, k=int(ks[i]), query_ids=[900000 + i]))
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
                    "k": "uniform {10, 50, 100}", "eps": EPS})
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
    # one step: one walk of one query through Alg. 1 (a bounded sample of the query)
    for i in range(args.warmup):
        O.single_source(int(qs[i % len(qs)]), eps=EPS, seed=3, qid=i, walk_begin=0, walk_end=1)
    t0 = time.perf_counter()
    for i in range(args.steps):
        q = i % len(qs)
        O.single_source(int(qs[q]), eps=EPS, seed=3, qid=q, walk_begin=i // len(qs), walk_end=i // len(qs) + 1)
    el = time.perf_counter() - t0
    qps = args.steps / el / nr
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe_workload(args.workload, n, len(s)),
                       "step": "one walk of one query (Alg. 1 on it), queries/s = walks/s / n_r"},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": "%d walks over %d queries (of n_r=%d each)" % (args.steps, min(args.steps, len(qs)), nr)},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_06955_gb300 import build, probesim
    build.build()
    n, s, d, qs = load_workload(args.workload)
    G = probesim.Graph(n, s, d)
    tuning = G.autotune()  # launch shape of the pull kernel, chosen on this graph before timing
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    nq = len(qs)

    def query(i):
        j = replica_query_id(rank, i)
        return probesim.make_queries([qs[j % nq]], eps=EPS, k=50, query_ids=[j])

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

    # batched leg: the same number of queries, args.batch per call
    B = max(1, args.batch)
    nb = max(1, args.steps // B)
    outb = torch.zeros((B, n), dtype=torch.float32, device=dev)
    Qb = [probesim.make_queries([qs[replica_query_id(rank, args.warmup + i * B + j) % nq] for j in range(B)],
                                eps=EPS, query_ids=[replica_query_id(rank, args.warmup + i * B + j) for j in range(B)])
          for i in range(nb)]
    G.single_source(Qb[0], out=outb, stream=sptr)
    bev = []
    barrier()
    for i in range(nb):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.single_source(Qb[i], out=outb, stream=sptr)
        b.record(stream)
        bev.append((a, b))
    barrier()
    bms = sum(a.elapsed_time(b) for a, b in bev)
    batched_qps = nb * B / (bms / 1e3)
    # the batches hold the first nb * B queries of the timed leg: the same queries one at a time
    single_same_qps = nb * B / (sum(lat[:nb * B]) / 1e3)

    # optional mixed-eps top-k leg (the batched configuration's pattern): one call of --mixed-batch queries,
    # eps alternating 0.1 / 0.05 (uneven n_r), top-50 per query; the library cuts the call into batches that
    # fit its workspace budget
    mixed = None
    if args.mixed_batch > 0:
        MB = args.mixed_batch
        eps_mix = [EPS if j % 2 == 0 else EPS / 2 for j in range(MB)]
        Qm = probesim.make_queries([qs[replica_query_id(rank, 5000 + j) % nq] for j in range(MB)], eps=eps_mix, k=50,
                                   query_ids=[replica_query_id(rank, 5000 + j) for j in range(MB)])
        mids = torch.empty((MB, 50), dtype=torch.int32, device=dev)
        mvals = torch.empty((MB, 50), dtype=torch.float32, device=dev)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.topk(Qm, kmax=50, ids=mids, vals=mvals, stream=sptr)
        b.record(stream)
        barrier()
        mms = a.elapsed_time(b)
        mixed = {"queries": MB, "eps": "%g / %g alternating" % (EPS, EPS / 2), "k": 50, "value": MB / (mms / 1e3),
                 "unit": "queries/s", "ms": mms,
                 "n_r": [int(G.num_walks(EPS)), int(G.num_walks(EPS / 2))]}

    # randomized PROBE (Alg. 3) on the same graph: a few queries one at a time
    GR = probesim.Graph(n, s, d, probe_mode=probesim.PROBE_RANDOMIZED)
    rq = 10
    GR.single_source(query(0), out=out, stream=sptr)
    rsum = {"edge_gathers": 0, "levels": 0, "walk_nodes": 0}
    rand_s = 0.0
    for i in range(rq):
        barrier()
        r0 = time.perf_counter()
        GR.single_source(query(args.warmup + i), out=out, stream=sptr)
        barrier()
        rand_s += time.perf_counter() - r0
        rst = GR.stats()  # describes the last call
        for k in rsum:
            rsum[k] += rst[k]
    GR.close()
    randomized = {"value": rq / rand_s, "unit": "queries/s", "queries": rq,
                  "candidates_per_query": rsum["edge_gathers"] / rq, "levels_per_query": rsum["levels"] / rq,
                  "walk_nodes_per_query": rsum["walk_nodes"] / rq}

    # end-to-end through the C ABI with host buffers: query struct in, pinned host scores out
    host_out = torch.empty((1, n), dtype=torch.float32, pin_memory=True)
    e2e_steps = min(args.steps, 30)
    barrier()
    e0 = time.perf_counter()
    for i in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        G.single_source(query(args.warmup + i), out=host_out, stream=sptr)
    barrier()
    e2e_s = time.perf_counter() - e0
    e2e_qps = e2e_steps / e2e_s

    # serving leg (last: its update batches change the graph): Poisson arrivals into the continuous-batching
    # server at each rate, with edge-update batches every 100 ms
    rates = [float(r) for r in args.serve_rates.split(",") if r]
    serving = serving_leg(probesim, G, n, s, d, qs, rates, args.serve_seconds, args.serve_updates, rank,
                          args.serve_workers, args.serve_max_batch)
    if args.serve_plain_rate > 0:  # the same at a saturating rate without updates: comparable to one per call
        serving += serving_leg(probesim, G, n, s, d, qs, [args.serve_plain_rate], args.serve_seconds, 0, rank,
                               args.serve_workers, args.serve_max_batch)

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return 0

    peak, peak_kind = measured_peak_hbm()
    # the pull's roofline, from the profiled pass (CUDA events around every pull launch)
    achieved = prof["probe_bytes"] / (prof["probe_ms"] / 1e3) / 1e9 if prof["probe_ms"] > 0 else None
    ratio = recorded_traffic()
    per_launch = prof["probe_bytes"] / max(1, prof["probe_launches"])
    roof = {"kernel": "k_pull (PROBE level pull, pull.cu)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "peak_kind": peak_kind + " hbm_gbs (copy)", "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": (ratio * per_launch) if ratio else None,
            "algorithmic_bytes_per_launch": per_launch, "launches": prof["probe_launches"],
            "profiled_queries": np_,
            "kernel_ms_share_of_step": prof["probe_ms"] / prof["step_ms"] if prof["step_ms"] else None,
            "l2_gather_GBps": 4.0 * prof["edge_gathers"] / (prof["probe_ms"] / 1e3) / 1e9 if prof["probe_ms"] else None}
    lat_sorted = sorted(lat)

    def pct(p):
        return lat_sorted[min(len(lat_sorted) - 1, int(round(p / 100.0 * (len(lat_sorted) - 1))))]

    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe_workload(args.workload, n, len(s)) +
                                   " (n_r=%d), deterministic PROBE, one query per call" % G.num_walks(EPS),
                       "queries": "uniform over nodes with in-degree >= 1", "l2": "flushed between steps (256 MB write)",
                       "pull_tuning": tuning,
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "p50_ms": pct(50), "p99_ms": pct(99), "wall_s": wall,
            "batched": {"batch": B, "value": batched_qps, "unit": "queries/s", "calls": nb,
                        "same_queries_one_at_a_time": single_same_qps},
            "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": 32, "d2h_bytes_per_step": 4 * n,
                    "steps": e2e_steps},
            "roofline": roof, "clocks": clk.summary(), "gpu_launches": agg["kernel_launches"],
            "phases_ms_per_query": {k: v / np_ for k, v in phases.items()},
            "profiled_ms_per_query": prof["step_ms"] / np_,
            "randomized_probe": randomized,
            "mixed_eps_topk": mixed,
            "serving": serving,
            "work": {"walks_per_query": agg["walks"] / args.steps, "tree_nodes_per_query": agg["tree_nodes"] / args.steps,
                     "vectors_per_query": agg["vectors"] / args.steps,
                     "edge_gathers_per_query": agg["edge_gathers"] / args.steps}}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n, s, d, qs, args.cpu_seconds)
    if world > 1:
        torch.distributed.barrier()
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
