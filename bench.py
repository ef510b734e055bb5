#!/usr/bin/env python
"""Benchmark of the SKIS hot path on GB300.

The benchmark line is the R-MAT workload: n = 2^25 vertices, m = 2^30 edges
(a, b, c, d = 0.57, 0.19, 0.19, 0.05), weighted cascade, int32 in-CSR, a
stream of 10^8 IIS sample ids with the tier split chosen by the library's
autotuner. One step is one pass of the whole hot path over one block of
1,000,000 consecutive sample ids of that stream (step i draws ids
[i 10^6, (i + 1) 10^6); under N ranks, block i N + r on rank r): graph load
(canonical in-CSR, thresholds, fixed-point gamma, alias table), IIS sampling
of the block, greedy max-coverage (k = 100, with the inverted index it
builds) and one batch of 64 influence queries (seed sets of 10 uniform
vertices). With N > 1 the ranks' blocks form one sketch: greedy and the
queries exchange counts through an NCCL all-reduce (the library's sharded
entry points).

`value` is RR sets/s of the whole job with the edge arrays already in HBM;
`e2e` is the same metric through the C ABI with pinned host buffers, the
host->device copy of the edge list and queries and the device->host read of
the results inside the timed region. `--impl reference` times the CPU oracle
on the same workload, on every host core.

Secondary keys: the Chung-Lu TRI workload (n = 1M, m = 10M, 10M samples,
greedy k = 50) as its own step loop, coverage GB/s of the sketch scan, the
influence-oracle server (queries/s, p50/p99) and the method's variants.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "RR sets/s and sampled edges/s (% HBM roofline); oracle queries/s with p50/p99"
WORKLOAD = "rmat-2^25-wc"
STEP_IDS = 1_000_000
K_GREEDY = 100
QUERIES, QUERY_SIZE = 64, 10
SKETCH_SEED = 0x5EED0003
C2_WORKLOAD, C2_SEED = "chunglu-1e6-tri", 0x5EED0002
FALLBACK_HBM_GBS = 6800.0
PHILOX_IMAD = 40  # 10 rounds of two 32x32->64 products, each counted as two multiply-adds


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
    ap.add_argument("--no-secondary", action="store_true", help="skip the Chung-Lu line and coverage benchmark")
    ap.add_argument("--workload", default=WORKLOAD,
                    help=f"{WORKLOAD} (the benchmark line), {C2_WORKLOAD} (its own line) or "
                         "chunglu-4e7-wc-dssa (DSSA doubling)")
    ap.add_argument("--rmat-scale", type=int, default=25,
                    help="R-MAT levels (25; smaller only for profiler captures of a small case)")
    ap.add_argument("--step-ids", type=int, default=STEP_IDS, help="sample ids per step and rank")
    ap.add_argument("--split", default=None,
                    help="thread_max_deg,thread_max_steps,warp_max_coins instead of the autotuner's choice "
                         "(profiler captures: the split a bench line recorded)")
    ap.add_argument("--full-count", action="store_true",
                    help="instead of the step loop: the whole stream of 10^8 ids in one skis_sample call")
    ap.add_argument("--dssa-max-samples", type=int, default=1 << 26, help="sample cap of the DSSA run")
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


def step_first_id(step: int, rank: int, world: int, per_rank: int) -> int:
    """First sample id of rank `rank`'s block in step `step`: the steps walk
    the id stream in blocks of per_rank ids, the ranks of one step holding
    consecutive blocks (disjoint, and together one sketch of world blocks)."""
    return (step * world + rank) * per_rank


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


def code_sha(src: bytes) -> str:
    """sha256 of a CUDA source's code: comments and blank space removed, so
    a record stays valid across comment edits but not across code changes
    (string literals in the sampler hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", src.decode(), flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()


def _sampler_sha() -> str:
    return code_sha(open(os.path.join(ROOT, "paper_1709_03565_gb300", "csrc", "sample.cu"), "rb").read())


def _profile_record(name: str, workload: str, first_step: str):
    """The committed ncu record of the sampling launches on a workload
    (per-sample DRAM bytes and L2 sectors), if it was taken on the current
    sampler source and the same form of the first step; else None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("sample_cu_sha256") != _sampler_sha() or d.get("first_step") != first_step:
        return None
    if d.get("workload_key") != workload:
        return None
    return d


def _traffic_per_sample(first_step: str, name: str = "iis_sampler_dram.json", workload: str = C2_WORKLOAD):
    """Measured DRAM bytes per sample of the sampling tiers from a committed
    ncu record taken on the current kernel source and first-step form."""
    d = _profile_record(name, workload, first_step)
    return None if d is None else float(d["dram_bytes_per_sample"])


def algorithmic_bytes(T: int, entries: int, coins: int, per_edge_tau: bool) -> int:
    """Algorithmic HBM bytes of one IIS sampling launch (random gathers at
    32-byte sector granularity): per sample one alias-entry sector and a
    32-byte header; per member one row-record sector and a 4-byte write; per
    non-source member one source-id sector (the live edge that added it);
    per coin a 4-byte threshold when thresholds are per edge (weighted
    cascade: none, the row record holds it)."""
    return 32 * T + 32 * T + 36 * entries + 32 * (entries - T) + (4 * coins if per_edge_tau else 0)


def alu_peak_blocks_per_s(sms: int, mhz: float) -> float:
    """Derived integer-multiply ceiling in Philox4x32-10 blocks per second:
    64 32-bit integer multiply-adds per clock per SM, a block's ten rounds of
    two 32x32->64 products counted as 40 of them."""
    return sms * 64.0 / PHILOX_IMAD * mhz * 1e6


def measured_alu_ceiling(skis, stream, sms: int, gpu_id: str) -> dict:
    """The coin generator's measured throughput on this GPU: the probe launch
    draws only Philox blocks (2048 threads per SM, 4096 blocks each, four
    independent blocks a step) and folds their words into one XOR, with no
    memory traffic. Per form (0: every block in full; 1: the hub loop's
    per-sample hoisting) three warm-up launches, then 40 timed ones: best and
    median, with the SM clocks sampled over the timed launches."""
    threads, per = sms * 2048, 4096
    out = {"threads": threads, "blocks_per_launch": threads * per, "kernel": "k_philox_rate"}
    for form, name in ((0, "full_blocks"), (1, "hoisted_blocks")):
        for r in range(3):
            skis.skis_philox_rate(1 + r, threads, per, form, stream=stream)
        clocks = ClockSampler(gpu_id)
        clocks.start()
        ms = sorted(skis.skis_philox_rate(1 + r, threads, per, form, stream=stream)[0] for r in range(40))
        out[name] = {"blocks_per_s": threads * per / (ms[0] / 1e3), "ms": ms[0],
                     "median_blocks_per_s": threads * per / (ms[len(ms) // 2] / 1e3), "clocks": clocks.stop()}
    return out


# -------------------------------------------------------------- oracle
# The oracle on every host core: worker processes each sample disjoint id
# ranges of the same workload. The graph is built once in the parent and the
# workers are forked from it (copy-on-write) before this process touches
# CUDA; nothing forks after the first GPU call.
_REF = {}


def _ref_sample(job):
    seed, ids = job
    out = _REF["graph"].sample_ids(seed, np.asarray(ids, dtype=np.uint64), bucket=_REF["bucket"])
    return int(out["coins"].sum())


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_graph(name: str, rmat_scale: int = 25):
    """The oracle's graph of a workload (the one whose edge list `edges` gives)."""
    import oracle

    spec, src, dst, p = edges(name, rmat_scale)
    oracle.build()
    if p is None:
        og = oracle.OracleGraph(spec["n"], src, dst, model=oracle.W_WC)
    else:
        og = oracle.OracleGraph(spec["n"], src, dst, weights=p, model=oracle.W_P)
    return spec, og


def fork_pool(og, bucket: bool, cores: int):
    import multiprocessing as mp

    _REF["graph"], _REF["bucket"] = og, bucket
    return mp.get_context("fork").Pool(cores)


def pool_step(pool, seed, start, per_core, cores):
    """Sample ids [start, start + per_core cores), one id per job: sample costs
    are heavy-tailed (a sample may or may not reach the hubs' in-rows), so
    the workers take ids as they finish rather than fixed blocks."""
    jobs = [(seed, [j]) for j in range(start, start + per_core * cores)]
    return sum(pool.map(_ref_sample, jobs, chunksize=1))


def edges(name: str, rmat_scale: int = 25):
    """Edge list (and TRI probabilities) of a workload; R-MAT at another
    scale keeps 32 edges a vertex (profiler captures of a small case)."""
    import synth

    if name == WORKLOAD and rmat_scale != 25:
        spec = dict(synth.WORKLOADS[WORKLOAD], scale=rmat_scale, n=1 << rmat_scale, m=32 << rmat_scale)
        src, dst = synth.rmat(rmat_scale, spec["m"], 0.57, 0.19, 0.19, spec["seed"])
        return spec, src, dst, None
    return synth.workload(name)


def cpu_baseline(og, seed: int, bucket: bool, seconds: float, cores: int, per_core: int, sample_note: str):
    """The oracle as it stands on one core, then on every core (forked
    workers over disjoint id ranges); bounded by `seconds` each."""
    done, t0 = 0, time.perf_counter()
    chunk = max(1, per_core)
    while time.perf_counter() - t0 < seconds:
        og.sample_ids(seed, np.arange(done, done + chunk, dtype=np.uint64), bucket=bucket)
        done += chunk
    dt = time.perf_counter() - t0
    out = {"value": done / dt, "unit": "RR sets/s", "cores": 1, "kind": "oracle",
           "sample": f"sample ids 0..{done - 1} of {sample_note} (single-threaded C oracle, {dt:.1f} s)"}
    if cores > 1:
        pool = fork_pool(og, bucket, cores)
        pool_step(pool, seed, 0, 1, cores)  # workers ready
        start, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            pool_step(pool, seed, start, chunk, cores)
            start += chunk * cores
        dt_all = time.perf_counter() - t0
        pool.close()
        pool.join()
        out["all_cores"] = {"value": start / dt_all, "unit": "RR sets/s", "cores": cores,
                            "sample": f"sample ids 0..{start - 1}, {cores} forked worker processes"}
    return out


def run_reference(args, rank, world):
    """The oracle on the benchmark workload and first-step form, every host
    core, each step a bounded block of consecutive sample ids."""
    if rank != 0:
        return
    t0 = time.perf_counter()
    spec, og = oracle_graph(WORKLOAD, args.rmat_scale)
    build_s = time.perf_counter() - t0
    cores = host_cores()
    per_core = 16
    per_step = per_core * cores
    bucket = args.first_step == "bucket"
    pool = fork_pool(og, bucket, cores)
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
        "config": {"workload": WORKLOAD if args.rmat_scale == 25 else f"rmat-2^{args.rmat_scale}-wc",
                   "n": spec["n"], "m": spec["m"], "step": f"{per_step} consecutive sample ids of the id stream",
                   "first_step": args.first_step},
        "sampled_edges_per_s": coins / dt,
        "oracle_graph_build_s": build_s,
        "cpu_baseline": {"value": value, "unit": "RR sets/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} sample ids per step, the C oracle in {cores} forked worker processes"},
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


def serving_benchmark(skis, torch, dev, stream):
    """Influence-oracle serving on a device-resident sketch: saturation
    throughput (all requests at t = 0) of continuous batching versus one
    query per launch, and latency under Poisson arrivals swept up to the
    batched saturation rate."""
    import synth

    spec, src, dst, _ = synth.workload(SERVE_WORKLOAD)
    n, T = spec["n"], spec["samples"]
    d_src, d_dst = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    g = skis.skis_load_graph(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
    s = skis.skis_sketch_create(g, 0x5EED0004, T * 16, stream=stream)
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


# ------------------------------------------------------- Chung-Lu line
def best_of(skis, torch, stream, make, run, reps=2):
    out = None
    for _ in range(reps):
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


def chunglu_line(skis, torch, dev, stream, args, peak):
    """The Chung-Lu TRI workload (n = 1M, m = 10M, 10M samples, greedy
    k = 50, 64 queries) as its own step loop, its sampling roofline, the
    coverage GB/s of the sketch scan and the variants' sampling rates."""
    import synth

    spec, src, dst, p = synth.workload(C2_WORKLOAD)
    n, m, T, k = spec["n"], spec["m"], spec["samples"], spec["k"]
    q_off, q_seeds = synth.seed_sets(n, [QUERY_SIZE] * QUERIES, 11)
    d_src, d_dst, d_p = (torch.from_numpy(x).to(dev) for x in (src, dst, p))
    d_off, d_seeds = torch.from_numpy(q_off).to(dev), torch.from_numpy(q_seeds).to(dev)
    d_cov = torch.empty(QUERIES, dtype=torch.int64, device=dev)
    d_est = torch.empty(QUERIES, dtype=torch.float64, device=dev)
    first_step = 1 if args.first_step == "bucket" else 0

    def step():
        g = skis.skis_load_graph(n, d_src, d_dst, d_p, skis.SKIS_W_EXPLICIT_P, stream=stream)
        s = skis.skis_sketch_create(g, C2_SEED, int(T * 5.5), stream=stream)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, first_step)
        skis.skis_sample(s, T, stream=stream)
        skis.skis_greedy_maxcover(s, k, stream=stream)
        skis.skis_estimate(s, d_off, d_seeds, d_cov, d_est, stream=stream)
        st = skis.skis_sketch_stats(s)
        s.close()
        g.close()
        return st

    for _ in range(3):
        step()
    steps = 10
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    coins, entries = stats[-1]["coins"], stats[-1]["entries"]
    sample_ms = statistics.mean(s["last_sample_ms"] for s in stats)
    alg = algorithmic_bytes(T, entries, coins, per_edge_tau=True)
    tps = _traffic_per_sample(args.first_step)
    out = {
        "workload": C2_WORKLOAD, "graph": "Chung-Lu directed, exponent 2.1, TRI probabilities", "n": n, "m": m,
        "samples": T, "k": k, "steps": steps, "ms_per_step": ms, "value": T / (ms / 1e3), "unit": "RR sets/s",
        "sampling_only": {"rr_sets_per_s": T / (sample_ms / 1e3), "edges_per_s": coins / (sample_ms / 1e3),
                          "thread_tier_ms": statistics.mean(s["last_thread_ms"] for s in stats),
                          "warp_tier_ms": statistics.mean(s["last_warp_ms"] for s in stats),
                          "cta_tier_ms": statistics.mean(s["last_cta_ms"] for s in stats)},
        "per_sample": {"members": entries / T, "coins": coins / T},
        "roofline": {"bound": "hbm", "achieved": alg / (sample_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / (sample_ms / 1e3) / 1e9 / peak,
                     "traffic": (tps * T if tps is not None else None), "algorithmic_bytes": alg,
                     "kernel": "k_sources + k_iis_lane + k_iis_warp + k_iis_cta", "kernel_ms": sample_ms},
    }
    # coverage: one batch of 64 queries over the 10M-sample sketch, scanned and through the index
    g = skis.skis_load_graph(n, d_src, d_dst, d_p, skis.SKIS_W_EXPLICIT_P, stream=stream)
    s = skis.skis_sketch_create(g, C2_SEED, int(T * 5.5), stream=stream)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, first_step)
    skis.skis_sample(s, T, stream=stream)
    cov = {"queries": QUERIES, "query_size": QUERY_SIZE, "samples": T, "entries": entries}
    for name, mode in (("scan", 2), ("index", 1)):
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_QUERY_INDEX, mode)
        for _ in range(3):
            skis.skis_estimate(s, d_off, d_seeds, d_cov, d_est, stream=stream)
        reps = 20
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(reps):
            skis.skis_estimate(s, d_off, d_seeds, d_cov, d_est, stream=stream)
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / reps
        kms = skis.skis_sketch_stats(s)["last_query_ms"]  # the coverage launches alone (library events)
        cov[name] = {"ms_per_batch": cms, "queries_per_s": QUERIES / (cms / 1e3), "kernel_ms": kms}
        if name == "scan":  # algorithmic bytes: one 4-byte read per member (headers only for seed hits)
            nbytes = 4 * entries
            cov[name].update({"algorithmic_bytes": nbytes, "gb_per_s": nbytes / (kms / 1e3) / 1e9,
                              "frac_of_hbm_peak": nbytes / (kms / 1e3) / 1e9 / peak,
                              "call_gb_per_s": nbytes / (cms / 1e3) / 1e9,
                              "kernel": "k_scan_ordered + k_unmark (members in sample-id order)"})
    s.close()
    out["coverage"] = cov
    if not args.no_variants:
        var = {}

        def mk(opt=None, val=None, sketch_graph=None, arena=None):
            def f():
                sk = skis.skis_sketch_create(sketch_graph or g, C2_SEED, arena or int(T * 5.5), stream=stream)
                if opt is not None:
                    skis.skis_sketch_set_option(sk, opt, val)
                return sk
            return f

        other = 0 if first_step == 1 else 1
        st, _ = best_of(skis, torch, stream, mk(skis.SKIS_OPT_FIRST_STEP, other),
                        lambda sk: skis.skis_sample(sk, T, stream=stream))
        var["first_step_" + ("bucket" if other else "rejection")] = {
            "rr_sets_per_s": T / (st["last_sample_ms"] / 1e3), "sample_ms": st["last_sample_ms"],
            "coins_per_sample": st["coins"] / T}
        st, _ = best_of(skis, torch, stream, mk(skis.SKIS_OPT_SAMPLER, 1),
                        lambda sk: skis.skis_sample(sk, T, stream=stream))
        var["ris"] = {"rr_sets_per_s": T / (st["last_sample_ms"] / 1e3), "sample_ms": st["last_sample_ms"],
                      "members_per_sample": st["entries"] / T, "note": "uniform source, singular samples kept"}
        target = int(5 * n * math.log(n))
        st, (app, _) = best_of(skis, torch, stream, mk(skis.SKIS_OPT_FIRST_STEP, first_step, arena=int(target * 1.3)),
                               lambda sk: skis.skis_sample_to_size(sk, target, stream=stream))
        var["stop_at_size"] = {"target_entries": target, "h": 5, "samples": app, "entries": st["entries"],
                               "call_ms": st["call_ms"], "rr_sets_per_s": app / (st["call_ms"] / 1e3)}
        glt = skis.skis_load_graph_lt(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
        st, _ = best_of(skis, torch, stream, mk(sketch_graph=glt), lambda sk: skis.skis_sample(sk, T, stream=stream))
        var["lt_wc"] = {"rr_sets_per_s": T / (st["last_sample_ms"] / 1e3), "sample_ms": st["last_sample_ms"],
                        "members_per_sample": st["entries"] / T, "walk_ms": st["last_thread_ms"],
                        "long_walk_ms": st["last_warp_ms"], "long_walks": st["to_warp"]}
        glt.close()
        out["variants"] = var
    g.close()
    return out


# ----------------------------------------------------------- DSSA run
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
    # warm-up: the first run on a graph pays the device memory pool's growth
    skis.skis_dssa_maxinf(g, SKETCH_SEED + 4, SKETCH_SEED + 5, 1, eps, delta, 0, 1 << 16, args.dssa_max_samples,
                          stream=stream)
    torch.cuda.synchronize()
    for k in (1, 100, 1000):
        t2 = time.perf_counter()
        sk, res = skis.skis_dssa_maxinf(g, SKETCH_SEED + 4, SKETCH_SEED + 5, k, eps, delta, 0, 1 << 16,
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
    if args.workload == "chunglu-4e7-wc-dssa":
        return dssa_run(args)
    if args.workload not in (WORKLOAD, C2_WORKLOAD):
        raise SystemExit(f"unknown workload {args.workload}")

    bucket = args.first_step == "bucket"
    workload_name = WORKLOAD if args.rmat_scale == 25 else f"rmat-2^{args.rmat_scale}-wc"
    # ---- CPU baseline first: the oracle's worker processes are forked
    # from this process before it touches CUDA
    cpu = None
    if (args.workload == WORKLOAD and rank == 0 and world == 1 and not args.no_cpu_baseline
            and not args.profile_step and not args.full_count):
        t0 = time.perf_counter()
        spec0, og = oracle_graph(WORKLOAD, args.rmat_scale)
        build_s = time.perf_counter() - t0
        cpu = cpu_baseline(og, SKETCH_SEED, bucket, args.cpu_seconds, host_cores(), 8,
                           f"the {workload_name} id stream")
        cpu["oracle_graph_build_s"] = build_s
        del og

    import torch

    import paper_1709_03565_gb300 as skis

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    skis.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = _peaks()

    if args.workload == C2_WORKLOAD and args.profile_step:  # one Chung-Lu step (the command profiled with ncu)
        import synth

        spec, src, dst, p = synth.workload(C2_WORKLOAD)
        d_src, d_dst, d_p = (torch.from_numpy(x).to(dev) for x in (src, dst, p))
        q_off, q_seeds = synth.seed_sets(spec["n"], [QUERY_SIZE] * QUERIES, 11)
        g = skis.skis_load_graph(spec["n"], d_src, d_dst, d_p, skis.SKIS_W_EXPLICIT_P, stream=stream)
        s = skis.skis_sketch_create(g, C2_SEED, int(spec["samples"] * 5.5), stream=stream)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 1 if bucket else 0)
        skis.skis_sample(s, spec["samples"], stream=stream)
        skis.skis_greedy_maxcover(s, spec["k"], stream=stream)
        skis.skis_estimate(s, q_off, q_seeds, stream=stream)  # walks the index greedy built
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_QUERY_INDEX, 2)
        skis.skis_estimate(s, q_off, q_seeds, stream=stream)  # the same batch by a scan of the sketch
        st = skis.skis_sketch_stats(s)
        print(json.dumps({"profile_step": C2_WORKLOAD, "samples": spec["samples"], "entries": st["entries"],
                          "coins": st["coins"], "sample_ms": st["last_sample_ms"],
                          "launches": skis.skis_kernel_launches()}))
        return
    if args.workload == C2_WORKLOAD:  # the Chung-Lu step loop as its own line
        line = chunglu_line(skis, torch, dev, stream, args, peak)
        line.update({"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic"})
        print(json.dumps(line))
        return

    import synth

    t0 = time.perf_counter()
    spec, src, dst, _ = edges(WORKLOAD, args.rmat_scale)
    gen_s = time.perf_counter() - t0
    n, m = spec["n"], spec["m"]
    per = args.step_ids
    q_off, q_seeds = synth.seed_sets(n, [QUERY_SIZE] * QUERIES, 13)
    d_src, d_dst = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    d_off, d_seeds = torch.from_numpy(q_off).to(dev), torch.from_numpy(q_seeds).to(dev)
    d_cov = torch.empty(QUERIES, dtype=torch.int64, device=dev)
    d_est = torch.empty(QUERIES, dtype=torch.float64, device=dev)
    arena = per * 128 + (1 << 23)  # ~93 members a sample measured, plus the tiers' chunk reservations
    first_step = 1 if bucket else 0

    # the tier split, chosen once by the library's autotuner on a pilot
    pilot = min(20_000, per)
    if args.split:
        d, st_, c = (int(x) for x in args.split.split(","))
        tune = {"max_deg": d, "max_steps": st_, "warp_max_coins": c, "candidate_ms": []}
        pilot = 0
    else:
        g0 = skis.skis_load_graph(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
        s0 = skis.skis_sketch_create(g0, SKETCH_SEED, arena, stream=stream)
        skis.skis_sketch_set_option(s0, skis.SKIS_OPT_FIRST_STEP, first_step)
        tune = skis.skis_sketch_autotune(s0, pilot, stream=stream)
        s0.close()
        g0.close()
    split = ((skis.SKIS_OPT_THREAD_MAX_DEG, tune["max_deg"]), (skis.SKIS_OPT_THREAD_MAX_STEPS, tune["max_steps"]),
             (skis.SKIS_OPT_WARP_MAX_COINS, tune["warp_max_coins"]))

    exchange = None
    if world > 1:
        import torch.distributed as dist

        exchange = torch.zeros(n + 1, dtype=torch.int64, device=dev)

        def allreduce(count):
            dist.all_reduce(exchange[:count])

    def run_step(i, src_buf, dst_buf, offs, seeds_buf, cov_buf, est_buf):
        g = skis.skis_load_graph(n, src_buf, dst_buf, None, skis.SKIS_W_WC, stream=stream)
        s = skis.skis_sketch_create(g, SKETCH_SEED, arena, stream=stream)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, first_step)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_ID, step_first_id(i, rank, world, per))
        for opt, val in split:
            skis.skis_sketch_set_option(s, opt, val)
        skis.skis_sample(s, per, stream=stream)
        if exchange is None:
            out = skis.skis_greedy_maxcover(s, K_GREEDY, stream=stream)  # builds the inverted index
            skis.skis_estimate(s, offs, seeds_buf, cov_buf, est_buf, stream=stream)  # walks it
        else:
            out = skis.skis_greedy_maxcover_sharded(s, K_GREEDY, exchange, allreduce, stream=stream)
            skis.skis_estimate_sharded(s, offs, seeds_buf, exchange, allreduce, cov_buf, est_buf, stream=stream)
        st = skis.skis_sketch_stats(s)
        s.close()
        g.close()
        return st, out

    def step(i):
        return run_step(i, d_src, d_dst, d_off, d_seeds, d_cov, d_est)[0]

    if args.full_count:
        return full_count_run(skis, torch, stream, g0_args=(n, d_src, d_dst), split=split, first_step=first_step,
                              tune=tune, workload_name=workload_name, m=m)
    if args.profile_step:
        st = step(0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": workload_name, "samples": per, "entries": st["entries"],
                          "coins": st["coins"], "deferred": st["deferred"], "cta_ms": st["last_cta_ms"],
                          "sample_ms": st["last_sample_ms"], "launches": skis.skis_kernel_launches()}))
        return
    warm = max(args.warmup, 3)
    for i in range(warm):
        step(i)
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
        stats.append(step(warm + i))
        marks[i + 1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]
    launches = skis.skis_kernel_launches() - launches0
    elapsed_ms = reduce_over_ranks(e0.elapsed_time(e1), "max")
    value = reduce_over_ranks(args.steps * per, "sum") / (elapsed_ms / 1e3)
    coins = statistics.mean(s["coins"] for s in stats)
    entries = statistics.mean(s["entries"] for s in stats)
    sample_ms = statistics.mean(s["last_sample_ms"] for s in stats)
    tiers = {k: statistics.mean(s[f"last_{k}_ms"] for s in stats) for k in ("thread", "warp", "cta")}

    # ---- end to end through the C ABI with pinned host buffers
    h_src = torch.from_numpy(src).pin_memory()
    h_dst = torch.from_numpy(dst).pin_memory()
    h_off = torch.from_numpy(q_off).pin_memory()
    h_seeds = torch.from_numpy(q_seeds).pin_memory()
    h_cov = torch.empty(QUERIES, dtype=torch.int64).pin_memory()
    h_est = torch.empty(QUERIES, dtype=torch.float64).pin_memory()
    nxt = warm + args.steps
    run_step(nxt, h_src, h_dst, h_off, h_seeds, h_cov, h_est)
    nxt += 1
    barrier()
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e2.record(stream)
    for i in range(args.e2e_steps):
        run_step(nxt + i, h_src, h_dst, h_off, h_seeds, h_cov, h_est)
    e3.record(stream)
    torch.cuda.synchronize()
    wall_e2e = time.perf_counter() - t0
    e2e_ms = reduce_over_ranks(max(e2.elapsed_time(e3), wall_e2e * 1e3), "max")
    e2e_value = reduce_over_ranks(args.e2e_steps * per, "sum") / (e2e_ms / 1e3)
    h2d = m * (4 + 4) + q_off.nbytes + q_seeds.nbytes
    d2h = K_GREEDY * (4 + 8 + 8) + QUERIES * (8 + 8)
    del h_src, h_dst

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- rooflines of the sampling launches of one skis_sample call
    # (k_sources, the lane, warp and CTA tiers): under weighted cascade a coin
    # moves no algorithmic byte (the row record holds the threshold), so the
    # binding ceiling is the integer multiplier of the Philox blocks
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    rec = _profile_record("iis_sampler_rmat.json", workload_name, args.first_step)
    traffic = rec["dram_bytes_per_sample"] * per if rec else None
    l2 = None
    if rec:
        l2_sectors = rec["lts_t_sectors_per_sample"] * per
        l2 = {"sectors_per_launch": l2_sectors, "sectors_per_s": l2_sectors / (sample_ms / 1e3),
              "pct_of_peak_under_ncu": rec.get("lts_t_sectors_pct_of_peak"),
              "source": "ncu lts__t_sectors.sum of the sampling launches, scaled per sample (profiles/)"}
    alu_peak = alu_peak_blocks_per_s(sms, max_mhz)
    alu_achieved = coins / 4 / (sample_ms / 1e3)
    kernel = "k_sources + k_iis_lane + k_iis_warp + k_iis_cta (one skis_sample call)"
    roofline = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Philox blocks/s",
                "frac": alu_achieved / alu_peak, "traffic": traffic, "kernel": kernel, "kernel_ms": sample_ms,
                "peak_kind": f"derived: {sms} SMs x 64 IMAD/clk / {PHILOX_IMAD} per block x {max_mhz:.0f} MHz",
                "l2": l2}
    ceiling = measured_alu_ceiling(skis, stream, sms, gpu_uuid)
    roofline["measured_ceiling"] = ceiling
    roofline["frac_of_measured_ceiling"] = alu_achieved / ceiling["hoisted_blocks"]["blocks_per_s"]
    alg = algorithmic_bytes(per, entries, coins, per_edge_tau=False)
    roofline_hbm = {"bound": "hbm", "achieved": alg / (sample_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": alg / (sample_ms / 1e3) / 1e9 / peak, "traffic": traffic, "algorithmic_bytes": alg,
                    "kernel": kernel, "peak_kind": f"{peak_kind} hbm_gbs (burst)"}

    # ---- the other form of the first step on this workload (sampling only)
    variants = None
    if not args.no_variants:
        other = 0 if first_step == 1 else 1
        g = skis.skis_load_graph(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)

        def mk():
            sk = skis.skis_sketch_create(g, SKETCH_SEED, arena, stream=stream)
            skis.skis_sketch_set_option(sk, skis.SKIS_OPT_FIRST_STEP, other)
            for opt, val in split:
                skis.skis_sketch_set_option(sk, opt, val)
            return sk

        st, _ = best_of(skis, torch, stream, mk, lambda sk: skis.skis_sample(sk, per, stream=stream))
        variants = {("first_step_bucket" if other else "first_step_rejection"): {
            "rr_sets_per_s": per / (st["last_sample_ms"] / 1e3), "sample_ms": st["last_sample_ms"],
            "coins_per_sample": st["coins"] / per, "retries_per_sample": st["retries"] / per,
            "philox_blocks_per_s": st["coins"] / 4 / (st["last_sample_ms"] / 1e3)}}
        g.close()
    del d_src, d_dst
    torch.cuda.empty_cache()

    secondary = None
    if not args.no_secondary:
        secondary = chunglu_line(skis, torch, dev, stream, args, peak)
    serving = None if args.no_serving else serving_benchmark(skis, torch, dev, stream)

    line = {
        "metric": METRIC, "value": value, "unit": "RR sets/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name, "graph": "R-MAT (0.57, 0.19, 0.19, 0.05), weighted cascade, int32 CSR",
                   "n": n, "m": m, "samples_per_step": per * world, "id_stream": 100_000_000,
                   "step": f"{per} consecutive sample ids per rank (graph load, sampling, greedy k = {K_GREEDY}, "
                           f"{QUERIES} queries of {QUERY_SIZE})",
                   "k": K_GREEDY, "queries": QUERIES, "query_size": QUERY_SIZE,
                   "split": {"thread_max_deg": tune["max_deg"], "thread_max_steps": tune["max_steps"],
                             "warp_max_coins": tune["warp_max_coins"], "autotune_pilot": pilot},
                   "l2": "inputs larger than L2 (edge list 8.6 GB, CSR rebuilt every step)",
                   "first_step": args.first_step + (" (Eq. probn)" if bucket else " rounds"),
                   "parallelism": f"sample-id shards over {world} GPUs" if world > 1 else "single GPU"},
        "sampled_edges_per_s": reduce_over_ranks(args.steps * coins, "sum") / (elapsed_ms / 1e3),
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
        "sampling_only": {"rr_sets_per_s": per / (sample_ms / 1e3), "edges_per_s": coins / (sample_ms / 1e3),
                          "sample_ms": sample_ms, "tiers_ms": tiers,
                          "to_warp_tier": stats[-1]["to_warp"], "to_cta_tier": stats[-1]["deferred"],
                          "passes": stats[-1]["last_passes"]},
        "per_sample": {"members": entries / per, "coins": coins / per},
        "binding_ceiling": "alu (Philox integer multiplies; under weighted cascade a coin moves no byte)",
        "roofline": roofline,
        "roofline_hbm": roofline_hbm,
        "variants": variants,
        "secondary": secondary,
        "serving": serving,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "RR sets/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "generate_s": gen_s,
        "clocks": clk,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def full_count_run(skis, torch, stream, g0_args, split, first_step, tune, workload_name, m):
    """The whole id stream (10^8 samples) in one skis_sample call, then
    greedy k = 100 over it (a one-off measurement, not the step loop)."""
    n, d_src, d_dst = g0_args
    total = 100_000_000
    g = skis.skis_load_graph(n, d_src, d_dst, None, skis.SKIS_W_WC, stream=stream)
    s = skis.skis_sketch_create(g, SKETCH_SEED, total * 128 + (1 << 23), stream=stream)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, first_step)
    for opt, val in split:
        skis.skis_sketch_set_option(s, opt, val)
    skis.skis_sample(s, total, stream=stream)
    st = skis.skis_sketch_stats(s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    seeds, cov, est = skis.skis_greedy_maxcover(s, K_GREEDY, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sample_s = st["last_sample_ms"] / 1e3
    print(json.dumps({
        "metric": METRIC, "value": total / sample_s, "unit": "RR sets/s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name, "n": n, "m": m, "samples": total, "split": tune},
        "sample_s": sample_s, "sampled_edges_per_s": st["coins"] / sample_s,
        "per_sample": {"members": st["entries"] / total, "coins": st["coins"] / total},
        "tiers_ms": {"thread": st["last_thread_ms"], "warp": st["last_warp_ms"], "cta": st["last_cta_ms"]},
        "greedy_k100_ms": e0.elapsed_time(e1), "greedy_coverage": int(cov[-1]), "passes": st["last_passes"]}))
    s.close()
    g.close()


if __name__ == "__main__":
    main()
