#!/usr/bin/env python
"""Benchmark of the SKIS hot path on GB300.

One step = one pass of the whole hot path over the Chung-Lu workload
(n = 1M, m = 10M, exponent 2.1, trivalency probabilities, 10M IIS samples,
greedy max-coverage k = 50): graph load (canonical in-CSR, thresholds,
fixed-point gamma, alias table), IIS sampling, greedy max-coverage (with the
inverted index it builds) and one batch of 64 influence queries (seed sets
of 10 uniform vertices).

`value` is RR sets/s with the edge arrays already in HBM; `e2e` is the same
metric through the C ABI with host buffers (pinned), the host->device copy
of the inputs and the device->host read of the results inside the timed
region. `--impl reference` times the CPU oracle on the same workload.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one rank per GPU, each rank an independent replica
(its own sketch seed), value = all ranks' samples / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "RR sets/s and sampled edges/s (% HBM roofline); oracle queries/s with p50/p99"
WORKLOAD = "chunglu-1e6-tri"
QUERIES, QUERY_SIZE = 64, 10
SKETCH_SEED = 0x5EED0002
FALLBACK_HBM_GBS = 6800.0


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    help=f"{WORKLOAD} (the benchmark line), rmat-2^25-wc (bounded-sample rates) or "
                         "chunglu-4e7-wc-dssa (DSSA doubling)")
    ap.add_argument("--samples", type=int, default=200_000,
                    help="samples of the R-MAT run (200K: a bounded run; 100000000: the full count)")
    ap.add_argument("--dssa-max-samples", type=int, default=1 << 26, help="sample cap of the DSSA run")
    ap.add_argument("--rmat-scale", type=int, default=25,
                    help="R-MAT levels of the bounded run (25; smaller for profiler captures)")
    ap.add_argument("--no-autotune", action="store_true", help="R-MAT run: default tier split")
    ap.add_argument("--first-step", default="bucket", choices=["bucket", "rejection"],
                    help="form of Alg. 1's conditioned first step (Eq. probn buckets, or rejection rounds)")
    ap.add_argument("--profile-step", action="store_true",
                    help="run exactly one step and exit (the command profiled with ncu)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(x: float, op: str = "max") -> float:
    """Max (or sum) of a per-rank scalar over all ranks; identity on one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _traffic_per_sample(first_step: str):
    """Measured DRAM bytes per sample of the sampling tiers from the
    committed ncu summary, if it was taken on the current kernel source and
    the same form of the first step."""
    path = os.path.join(ROOT, "profiles", "iis_sampler_dram.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    src = open(os.path.join(ROOT, "paper_1709_03565_gb300", "csrc", "sample.cu"), "rb").read()
    if d.get("sample_cu_sha256") != hashlib.sha256(src).hexdigest() or d.get("first_step") != first_step:
        return None
    return float(d["dram_bytes_per_sample"])


def algorithmic_bytes(T: int, entries: int, coins: int, per_edge_tau: bool) -> int:
    """Algorithmic HBM bytes of one IIS sampling launch (random gathers at
    32-byte sector granularity): per sample one alias-entry sector and a
    32-byte header; per member one row-record sector and a 4-byte write; per
    non-source member one source-id sector (the live edge that added it);
    per coin a 4-byte threshold when thresholds are per edge."""
    return 32 * T + 32 * T + 36 * entries + 32 * (entries - T) + (4 * coins if per_edge_tau else 0)


# -------------------------------------------------------------- reference
# The oracle on every host core: worker processes (spawned, never forked after
# CUDA is up) each hold the oracle's graph and sample disjoint id ranges.
_REF_GRAPH = None


def _ref_init(n, src, dst, p, bucket):
    global _REF_GRAPH, _REF_BUCKET
    import oracle

    _REF_GRAPH = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    _REF_BUCKET = bucket


def _ref_sample(job):
    seed, start, count = job
    out = _REF_GRAPH.sample_ids(seed, np.arange(start, start + count, dtype=np.uint64), bucket=_REF_BUCKET)
    return int(out["coins"].sum())


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(n, src, dst, p, bucket, cores):
    import multiprocessing as mp

    import oracle

    oracle.build()  # once, before the workers load it
    return mp.get_context("spawn").Pool(cores, initializer=_ref_init, initargs=(n, src, dst, p, bucket))


def pool_step(pool, seed, start, per_core, cores):
    jobs = [(seed, start + i * per_core, per_core) for i in range(cores)]
    return sum(pool.map(_ref_sample, jobs))


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    import synth

    spec, src, dst, p = synth.workload(WORKLOAD)
    cores = host_cores()
    per_core = 50_000
    per_step = per_core * cores
    pool = oracle_pool(spec["n"], src, dst, p, args.first_step == "bucket", cores)
    nxt = 0

    def step():
        nonlocal nxt
        c = pool_step(pool, SKETCH_SEED, nxt, per_core, cores)
        nxt += per_step
        return c

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    coins = 0
    for _ in range(args.steps):
        coins += step()
    dt = time.perf_counter() - t0
    pool.close()
    pool.join()
    value = args.steps * per_step / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "RR sets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": spec["n"], "m": spec["m"], "samples": spec["samples"],
                   "k": spec["k"], "step": f"{per_step} consecutive sample ids of the workload",
                   "first_step": args.first_step},
        "sampled_edges_per_s": coins / dt,
        "cpu_baseline": {"value": value, "unit": "RR sets/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} sample ids per step, the C oracle in {cores} worker processes"},
        "e2e": {"value": value, "unit": "RR sets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------- serving
SERVE_WORKLOAD = "chunglu-4e6-wc-serve"


def serve_run(skis, s, queries, arrivals, slots, max_batch):
    """Drive the native server with requests arriving at the given times
    (seconds from start); returns per-request latency (s) and wall time."""
    srv = skis.skis_server_create(s, slots=slots, max_batch=max_batch, seed_capacity=1 << 16)
    nq = len(queries)
    done_at = np.zeros(nq)
    ticket_of = {}
    nxt = 0
    finished = 0
    t0 = time.perf_counter()
    while finished < nq:
        now = time.perf_counter() - t0
        while nxt < nq and arrivals[nxt] <= now:
            ticket_of[skis.skis_server_submit(srv, queries[nxt])] = nxt
            nxt += 1
        idle_wait = nxt == nq  # nothing left to admit: block on the GPU
        for t in skis.skis_server_progress(srv, wait=idle_wait):
            done_at[ticket_of[int(t)]] = time.perf_counter() - t0
            finished += 1
    wall = time.perf_counter() - t0
    srv.close()
    return done_at - arrivals, wall


def variants_benchmark(skis, torch, dev, stream, n, d_src, d_dst, d_p, T, seed, first_step):
    """Sampling rates of the method's variants on the bench graph (10M
    samples each, best of two, device time from the library's events):
    the other form of the first step, plain RIS, the Linear Threshold model
    (weighted-cascade weights on the same topology) and stop-at-size
    (h n ln n entries, h = 5)."""
    import math

    def best(make, run):
        out = None
        for _ in range(2):
            s = make()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = run(s)
            e1.record(stream)
            torch.cuda.synchronize()
            st = skis.skis_sketch_stats(s)
            st["call_ms"] = e0.elapsed_time(e1)
            s.close()
            if out is None or st["call_ms"] < out[0]["call_ms"]:
                out = (st, r)
        return out

    res = {}
    g = skis.skis_load_graph(n, d_src, d_dst, d_p, skis.SKIS_W_EXPLICIT_P, stream=stream)
    other = 0 if first_step == 1 else 1

    def mk(opt=None, val=None, sketch_graph=None, arena=None):
        def f():
            s = skis.skis_sketch_create(sketch_graph or g, seed, arena or int(T * 5.5), stream=stream)
            if opt is not None:
                skis.skis_sketch_set_option(s, opt, val)
            return s
        return f

    st, _ = best(mk(skis.SKIS_OPT_FIRST_STEP, other), lambda s: skis.skis_sample(s, T, stream=stream))
    res["first_step_" + ("bucket" if other else "rejection")] = {
        "rr_sets_per_s": T / (st["last_sample_ms"] / 1e3), "sample_ms": st["last_sample_ms"],
        "coins_per_sample": st["coins"] / T}
    st, _ = best(mk(skis.SKIS_OPT_SAMPLER, 1), lambda s: skis.skis_sample(s, T, stream=stream))
    res["ris"] = {"rr_sets_per_s": T / (st["last_sample_ms"] / 1e3), "sample_ms": st["last_sample_ms"],
                  "members_per_sample": st["entries"] / T, "note": "uniform source, singular samples kept"}
    target = int(5 * n * math.log(n))
    st, (app, _) = best(mk(skis.SKIS_OPT_FIRST_STEP, first_step, arena=int(target * 1.3)),
                        lambda s: skis.skis_sample_to_size(s, target, stream=stream))
    res["stop_at_size"] = {"target_entries": target, "h": 5, "samples": app, "entries": st["entries"],
                           "call_ms": st["call_ms"], "rr_sets_per_s": app / (st["call_ms"] / 1e3)}
    g.close()
    glt = skis.skis_load_graph_lt(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
    st, _ = best(mk(sketch_graph=glt), lambda s: skis.skis_sample(s, T, stream=stream))
    res["lt_wc"] = {"rr_sets_per_s": T / (st["last_sample_ms"] / 1e3), "sample_ms": st["last_sample_ms"],
                    "members_per_sample": st["entries"] / T, "walk_ms": st["last_thread_ms"],
                    "long_walk_ms": st["last_warp_ms"], "long_walks": st["to_warp"]}
    glt.close()
    return res


def coverage_benchmark(skis, torch, dev, stream, n, d_src, d_dst, d_p, T, seed, first_step, d_off, d_seeds, peak):
    """Coverage counting of one batch of 64 queries (seed sets of 10) over the
    bench sketch (10M samples), both ways: a scan of the whole sketch (headers
    and members streamed once, per-vertex query masks gathered from L2) and a
    walk of the inverted index (the lists of the queries' seeds)."""
    g = skis.skis_load_graph(n, d_src, d_dst, d_p, skis.SKIS_W_EXPLICIT_P, stream=stream)
    s = skis.skis_sketch_create(g, seed, int(T * 5.5), stream=stream)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, first_step)
    skis.skis_sample(s, T, stream=stream)
    entries = skis.skis_sketch_stats(s)["entries"]
    q = int(d_off.numel()) - 1
    d_cov = torch.empty(q, dtype=torch.int64, device=dev)
    d_est = torch.empty(q, dtype=torch.float64, device=dev)
    out = {"queries": q, "query_size": QUERY_SIZE, "samples": T, "entries": entries}
    for name, mode in (("scan", 2), ("index", 1)):
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_QUERY_INDEX, mode)
        for _ in range(3):  # warm-up (the index walk builds the index on the first call)
            skis.skis_estimate(s, d_off, d_seeds, d_cov, d_est, stream=stream)
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            skis.skis_estimate(s, d_off, d_seeds, d_cov, d_est, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_batch": ms, "queries_per_s": q / (ms / 1e3)}
        if name == "scan":  # algorithmic bytes: 12-byte header per sample, 4 bytes per member
            nbytes = 12 * T + 4 * entries
            out[name].update({"algorithmic_bytes": nbytes, "gb_per_s": nbytes / (ms / 1e3) / 1e9,
                              "frac_of_hbm_peak": nbytes / (ms / 1e3) / 1e9 / peak})
    s.close()
    g.close()
    return out


def serving_benchmark(skis, torch, dev, stream):
    """Influence-oracle serving on a device-resident sketch: saturation
    throughput (all requests at t = 0) of continuous batching versus one
    query per launch, and latency under Poisson arrivals at half the batched
    saturation rate."""
    import synth

    spec, src, dst, _ = synth.workload(SERVE_WORKLOAD)
    n, T = spec["n"], spec["samples"]
    d_src, d_dst = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    g = skis.skis_load_graph(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
    s = skis.skis_sketch_create(g, SKETCH_SEED + 2, T * 16, stream=stream)
    skis.skis_sample(s, T, stream=stream)
    st = skis.skis_sketch_stats(s)
    rng = np.random.Generator(np.random.PCG64(12345))
    nq = 3000
    sizes = synth.log_uniform_sizes(nq, 1, 1000, 44)
    off, seeds = synth.seed_sets(n, sizes, 45)
    queries = [seeds[off[b]:off[b + 1]] for b in range(nq)]
    serve_run(skis, s, queries[:200], np.zeros(200), 4, 64)  # warm-up
    lat_b, wall_b = serve_run(skis, s, queries, np.zeros(nq), 4, 64)
    sat_batched = nq / wall_b
    n1 = 300
    lat_1, wall_1 = serve_run(skis, s, queries[:n1], np.zeros(n1), 1, 1)
    sat_single = n1 / wall_1
    rate = 0.5 * sat_batched
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nq))
    lat_p, wall_p = serve_run(skis, s, queries, arrivals, 4, 64)
    # latency against offered load, swept up to saturation
    sweep = []
    for frac in (0.25, 0.75, 0.9, 1.0):
        lam = frac * sat_batched
        arr = np.cumsum(rng.exponential(1.0 / lam, size=nq))
        lat, wall = serve_run(skis, s, queries, arr, 4, 64)
        sweep.append({"offered_fraction": frac, "offered_per_s": lam, "served_per_s": nq / wall,
                      "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3)})
    s.close()
    g.close()
    return {
        "workload": SERVE_WORKLOAD, "n": n, "m": spec["m"], "samples": T, "entries": st["entries"],
        "query_sizes": "log-uniform in [1, 1000]", "requests": nq,
        "saturation_queries_per_s": sat_batched,
        "one_query_per_launch_queries_per_s": sat_single,
        "speedup_vs_one_per_launch": sat_batched / sat_single,
        "poisson_rate_per_s": rate, "queries_per_s": nq / wall_p,
        "p50_ms": float(np.percentile(lat_p, 50) * 1e3), "p99_ms": float(np.percentile(lat_p, 99) * 1e3),
        "saturation_p50_ms": float(np.percentile(lat_b, 50) * 1e3),
        "load_sweep": sweep,
        "slots": 4, "max_batch": 64,
    }


# ----------------------------------------------------------- R-MAT run
def rmat_run(args):
    """The R-MAT workload (2^25 vertices, 2^30 edges, weighted cascade):
    weighted cascade on R-MAT reaches its hubs' huge in-rows (about 10^6
    coins per sample), so 10^8 samples are about 10^14 coin flips. The
    default is a bounded number of samples whose rates set the time of any
    count; --samples 100000000 generates the full count in one call."""
    import torch

    import paper_1709_03565_gb300 as skis
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    if args.rmat_scale == 25:
        spec, src, dst, _ = synth.workload("rmat-2^25-wc")
    else:  # the same generator at a smaller scale (32 edges a vertex)
        spec = {"n": 1 << args.rmat_scale, "m": 32 << args.rmat_scale}
        src, dst = synth.rmat(args.rmat_scale, spec["m"], 0.57, 0.19, 0.19, 3)
    t_gen = time.perf_counter() - t0
    n, m = spec["n"], spec["m"]
    d_src, d_dst = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    del src, dst
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g = skis.skis_load_graph(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    load_ms = e0.elapsed_time(e1)
    del d_src, d_dst
    torch.cuda.empty_cache()
    info = skis.skis_graph_get_info(g)
    # member arena for ~93 members a sample with room to spare, plus the
    # tiers' per-warp chunk reservations: an arena that fills up makes
    # skis_sample grow it and rerun the samples that missed it
    s = skis.skis_sketch_create(g, SKETCH_SEED + 3, args.samples * 128 + (1 << 23), stream=stream)
    pilot = min(max(2000, args.samples // 20), 50_000)
    tune = None if args.no_autotune else skis.skis_sketch_autotune(s, pilot, stream=stream)
    skis.skis_sample(s, args.samples, stream=stream)
    st = skis.skis_sketch_stats(s)
    e0.record(stream)
    seeds, cov, est = skis.skis_greedy_maxcover(s, 100, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    greedy_ms = e0.elapsed_time(e1)
    free1, _ = torch.cuda.mem_get_info(dev)
    sample_s = st["last_sample_ms"] / 1e3
    line = {
        "metric": METRIC, "value": args.samples / sample_s, "unit": "RR sets/s", "n_gpus": 1, "steps": 1,
        "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "rmat-2^25-wc" if args.rmat_scale == 25 else f"rmat-2^{args.rmat_scale}-wc",
                   "graph": "R-MAT (0.57, 0.19, 0.19, 0.05), weighted cascade",
                   "n": n, "m": m, "samples": args.samples, "bounded_run": args.samples < 100_000_000},
        "sampled_edges_per_s": st["coins"] / sample_s,
        "per_sample": {"members": st["entries"] / args.samples, "coins": st["coins"] / args.samples},
        "seconds_for_1e8_samples": 1e8 / (args.samples / sample_s),
        "graph_load_ms": load_ms, "generate_s": t_gen, "Gamma": info["Gamma"],
        "tiers_ms": {"thread": st["last_thread_ms"], "warp": st["last_warp_ms"], "cta": st["last_cta_ms"]},
        "to_warp_tier": st["to_warp"], "to_cta_tier": st["deferred"], "passes": st["last_passes"],
        "autotune": tune,
        "greedy_k100_ms": greedy_ms, "greedy_coverage": int(cov[-1]), "greedy_estimate": float(est[-1]),
        "device_memory_used_gb": (free0 - free1) / 1e9,
    }
    s.close()
    g.close()
    print(json.dumps(line))


# ---------------------------------------------------------- DSSA run
def dssa_run(args):
    """DSSA-style doubling influence maximisation (two sketches grown in
    place, exact stopping test) on the Chung-Lu WC graph with n = 40M and
    m = 1.4B: k in {1, 100, 1000}, eps = 0.1, delta = 1/n, from 2^16
    samples up to a bounded cap; wall time of each whole run."""
    import torch

    import paper_1709_03565_gb300 as skis
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    spec, src, dst, _ = synth.workload("chunglu-4e7-wc-dssa")
    t_gen = time.perf_counter() - t0
    n, m = spec["n"], spec["m"]
    d_src, d_dst = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    del src, dst
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g = skis.skis_load_graph(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t1
    del d_src, d_dst
    torch.cuda.empty_cache()
    info = skis.skis_graph_get_info(g)
    eps, delta = 0.1, 1.0 / n
    runs = {}
    seeds = None
    for k in (1, 100, 1000):
        t2 = time.perf_counter()
        sk, res = skis.skis_dssa_maxinf(g, SKETCH_SEED + 7, SKETCH_SEED + 8, k, eps, delta, 0, 1 << 16,
                                        args.dssa_max_samples, stream=stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t2
        runs[str(k)] = {"seconds": wall, "samples_per_s": 2 * res["samples"] / wall,
                        "result": {key: (float(v) if isinstance(v, float) else int(v)) for key, v in res.items()}}
        if k == 100:
            seeds = sk
    g.close()
    line = {
        "metric": "DSSA doubling: seconds to an (1 - 1/e - eps)-approximate seed set (k = 100)",
        "value": runs["100"]["seconds"], "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "chunglu-4e7-wc-dssa", "graph": "Chung-Lu directed, exponent 2.0, weighted cascade",
                   "n": n, "m": m, "k": [1, 100, 1000], "eps": eps, "delta": delta, "n0": 1 << 16,
                   "n_max": args.dssa_max_samples},
        "runs": runs, "graph_load_s": load_s, "generate_s": t_gen,
        "Gamma": info["Gamma"], "seeds_head_k100": [int(x) for x in seeds[:10]],
    }
    print(json.dumps(line))


# ----------------------------------------------------------------- ours
def main():
    args = _args()
    rank, world, local = _dist()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != WORKLOAD:
        if args.workload == "rmat-2^25-wc":
            return rmat_run(args)
        if args.workload == "chunglu-4e7-wc-dssa":
            return dssa_run(args)
        raise SystemExit(f"unknown workload {args.workload}")

    import torch

    import paper_1709_03565_gb300 as skis
    import synth

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    skis.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    spec, src, dst, p = synth.workload(WORKLOAD)
    n, m, T, k = spec["n"], spec["m"], spec["samples"], spec["k"]
    q_off, q_seeds = synth.seed_sets(n, [QUERY_SIZE] * QUERIES, 11)
    d_src, d_dst, d_p = (torch.from_numpy(x).to(dev) for x in (src, dst, p))
    d_off, d_seeds = torch.from_numpy(q_off).to(dev), torch.from_numpy(q_seeds).to(dev)
    d_cov = torch.empty(QUERIES, dtype=torch.int64, device=dev)
    d_est = torch.empty(QUERIES, dtype=torch.float64, device=dev)
    seed = SKETCH_SEED + rank
    arena_hint = int(T * 5.5)
    torch.cuda.synchronize()

    first_step = 1 if args.first_step == "bucket" else 0

    def step():
        g = skis.skis_load_graph(n, d_src, d_dst, d_p, skis.SKIS_W_EXPLICIT_P, stream=stream)
        s = skis.skis_sketch_create(g, seed, arena_hint, stream=stream)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, first_step)
        skis.skis_sample(s, T, stream=stream)
        sd, sc, se = skis.skis_greedy_maxcover(s, k, stream=stream)  # builds the inverted index
        skis.skis_estimate(s, d_off, d_seeds, d_cov, d_est, stream=stream)  # walks it
        st = skis.skis_sketch_stats(s)
        s.close()
        g.close()
        return st

    if args.profile_step:
        st = step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": WORKLOAD, "samples": T, "entries": st["entries"],
                          "coins": st["coins"], "deferred": st["deferred"],
                          "launches": skis.skis_kernel_launches()}))
        return
    for _ in range(max(args.warmup, 3)):
        step()
    gpu_uuid = "0"
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_uuid = str(local)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- device-resident inputs
    clocks = ClockSampler(gpu_uuid)
    barrier()
    torch.cuda.synchronize()
    launches0 = skis.skis_kernel_launches()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0.record(stream)
    marks[0].record(stream)
    stats = []
    for i in range(args.steps):
        stats.append(step())
        marks[i + 1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]
    launches = skis.skis_kernel_launches() - launches0
    elapsed_ms = reduce_over_ranks(e0.elapsed_time(e1), "max")
    value = reduce_over_ranks(args.steps * T, "sum") / (elapsed_ms / 1e3)
    coins, entries = stats[-1]["coins"], stats[-1]["entries"]
    thread_ms = statistics.mean(s["last_thread_ms"] for s in stats)
    warp_ms = statistics.mean(s["last_warp_ms"] for s in stats)
    cta_ms = statistics.mean(s["last_cta_ms"] for s in stats)
    sample_ms = statistics.mean(s["last_sample_ms"] for s in stats)

    # ---- end to end through the C ABI with pinned host buffers
    h_src = torch.from_numpy(src).pin_memory()
    h_dst = torch.from_numpy(dst).pin_memory()
    h_p = torch.from_numpy(p).pin_memory()
    h_off = torch.from_numpy(q_off).pin_memory()
    h_seeds = torch.from_numpy(q_seeds).pin_memory()
    h_cov = torch.empty(QUERIES, dtype=torch.int64).pin_memory()
    h_est = torch.empty(QUERIES, dtype=torch.float64).pin_memory()

    def step_e2e():
        g = skis.skis_load_graph(n, h_src, h_dst, h_p, skis.SKIS_W_EXPLICIT_P, stream=stream)
        s = skis.skis_sketch_create(g, seed, arena_hint, stream=stream)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, first_step)
        skis.skis_sample(s, T, stream=stream)
        out = skis.skis_greedy_maxcover(s, k, stream=stream)
        skis.skis_estimate(s, h_off, h_seeds, h_cov, h_est, stream=stream)
        s.close()
        g.close()
        return out

    step_e2e()
    barrier()
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e2.record(stream)
    for _ in range(args.e2e_steps):
        step_e2e()
    e3.record(stream)
    torch.cuda.synchronize()
    wall_e2e = time.perf_counter() - t0
    e2e_ms = reduce_over_ranks(max(e2.elapsed_time(e3), wall_e2e * 1e3), "max")
    e2e_value = reduce_over_ranks(args.e2e_steps * T, "sum") / (e2e_ms / 1e3)
    h2d = m * (4 + 4 + 8) + q_off.nbytes + q_seeds.nbytes
    d2h = k * (4 + 8 + 8) + QUERIES * (8 + 8)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernels (the three IIS sampling tiers)
    peak, peak_kind = _peaks()
    # the three sampling launches of one skis_sample call (thread, warp and
    # CTA tiers) together produce the whole sketch
    alg = algorithmic_bytes(T, entries, coins, per_edge_tau=True)
    achieved = alg / (sample_ms / 1e3) / 1e9
    tps = _traffic_per_sample(args.first_step)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tps * T if tps is not None else None), "kernel": "k_sources + k_iis_lane + k_iis_warp + k_iis_cta",
                "algorithmic_bytes": alg, "kernel_ms": sample_ms, "peak_kind": f"{peak_kind} hbm_gbs (burst)"}

    # the second ceiling: integer ALU work of the coins, Philox4x32-10 blocks
    # (4 coins each; 10 rounds of two 32x32->64 multiplies), against 64
    # integer multiply-adds per clock per SM with each wide multiply counted
    # as two, at the maximum SM clock
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    alu_peak = sms * 64 / 40 * max_mhz * 1e6
    alu_achieved = coins / 4 / (sample_ms / 1e3)
    roofline_alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Philox blocks/s",
                    "frac": alu_achieved / alu_peak, "kernel": "k_sources + k_iis_lane + k_iis_warp + k_iis_cta",
                    "peak_kind": f"derived: {sms} SMs x 64 IMAD/clk / 40 per block x {max_mhz:.0f} MHz"}

    # ---- coverage counting (GB/s of the sketch scan) and influence-oracle serving (queries/s, p50/p99)
    coverage = coverage_benchmark(skis, torch, dev, stream, n, d_src, d_dst, d_p, T, seed, first_step, d_off, d_seeds,
                                  peak)
    serving = None if args.no_serving else serving_benchmark(skis, torch, dev, stream)
    variants = None if args.no_variants else variants_benchmark(skis, torch, dev, stream, n, d_src, d_dst, d_p, T,
                                                                seed, first_step)

    # ---- CPU baseline: the oracle, as it stands, on a bounded sample
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        og = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
        done, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < args.cpu_seconds:
            og.sample_ids(seed, np.arange(done, done + 50_000, dtype=np.uint64), bucket=args.first_step == "bucket")
            done += 50_000
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt, "unit": "RR sets/s", "cores": 1, "kind": "oracle",
               "sample": f"sample ids 0..{done - 1} of the same workload (single-threaded C oracle)"}
        # the same oracle on every host core (worker processes over disjoint id ranges)
        cores = host_cores()
        if cores > 1:
            pool = oracle_pool(n, src, dst, p, args.first_step == "bucket", cores)
            per_core = 20_000
            pool_step(pool, seed, 0, 1000, cores)  # workers ready
            start, t0 = 0, time.perf_counter()
            while time.perf_counter() - t0 < args.cpu_seconds:
                pool_step(pool, seed, start, per_core, cores)
                start += per_core * cores
            dt_all = time.perf_counter() - t0
            pool.close()
            pool.join()
            cpu["all_cores"] = {"value": start / dt_all, "unit": "RR sets/s", "cores": cores,
                                "sample": f"sample ids 0..{start - 1}, {cores} worker processes"}

    line = {
        "metric": METRIC, "value": value, "unit": "RR sets/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "graph": "Chung-Lu directed, exponent 2.1, TRI probabilities",
                   "n": n, "m": m, "samples": T, "queries": QUERIES, "query_size": QUERY_SIZE, "k": k,
                   "l2": "inputs larger than L2 (edge arrays 160 MB, arena ~170 MB, rebuilt every step)",
                   "first_step": args.first_step + (" (Eq. probn)" if args.first_step == "bucket" else " rounds"),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "sampled_edges_per_s": world * args.steps * coins / (elapsed_ms / 1e3),
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
        "sampling_only": {"rr_sets_per_s": T / (sample_ms / 1e3), "edges_per_s": coins / (sample_ms / 1e3),
                          "thread_tier_ms": thread_ms, "warp_tier_ms": warp_ms, "cta_tier_ms": cta_ms,
                          "to_warp_tier": stats[-1]["to_warp"], "to_cta_tier": stats[-1]["deferred"],
                          "passes": stats[-1]["last_passes"], "arena_capacity": stats[-1]["arena_capacity"]},
        "per_sample": {"members": entries / T, "coins": coins / T},
        "roofline": roofline,
        "roofline_alu": roofline_alu,
        "coverage": coverage,
        "serving": serving,
        "variants": variants,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "RR sets/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
