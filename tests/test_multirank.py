"""Multi-rank host logic on CPU with the gloo backend (world size 2): the
benchmark's max-over-ranks timing and sum of work, and the sharded
estimator's exchange — per-rank coverage counts over disjoint sample-id
ranges, summed with an int64 all-reduce, equal the single-process count."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import synth

    # timing: max over ranks, work: sum over ranks
    mx = bench.reduce_over_ranks(10.0 + rank, "max")
    sm = bench.reduce_over_ranks(1000 * (rank + 1), "sum")
    # sharded coverage: rank r holds sample ids [r T/2, (r+1) T/2)
    n, m, T = 400, 3000, 4000
    src, dst = synth.er(n, m, 5)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    ids = np.arange(rank * T // world, (rank + 1) * T // world, dtype=np.uint64)
    smp = g.sample_ids(77, ids)
    off, seeds = synth.seed_sets(n, [1, 5, 20], 3)
    cov = torch.zeros(3, dtype=torch.int64)
    mo, mem = smp["member_off"], smp["members"]
    for b in range(3):
        S = set(seeds[off[b]:off[b + 1]].tolist())
        cov[b] = sum(1 for t in range(len(ids)) if S & set(mem[mo[t]:mo[t + 1]].tolist()))
    dist.all_reduce(cov, op=dist.ReduceOp.SUM)
    out[rank] = (mx, sm, cov.tolist())
    dist.destroy_process_group()


def test_two_rank_reductions_and_sharded_coverage():
    import oracle
    import synth

    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = dict(out)
    assert res[0][0] == res[1][0] == 11.0
    assert res[0][1] == res[1][1] == 3000.0
    n, m, T = 400, 3000, 4000
    src, dst = synth.er(n, m, 5)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    sk = oracle.OracleSketch(g, 77, T)
    off, seeds = synth.seed_sets(n, [1, 5, 20], 3)
    cov, _ = sk.coverage(off, seeds)
    assert res[0][2] == res[1][2] == cov.tolist()


def _greedy_worker(rank, world, port, out):
    """The sharded greedy of the multi-GPU design: per-rank Delta counts over
    the rank's samples, summed (int64 all-reduce); each round every rank
    takes the same exact-key argmax on the summed counts (u128 key Delta W +
    T (2^f - w_v), ties to the lowest id), covers its own samples holding
    the winner and all-reduces its dense decrement vector."""
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth

    n, m, T, k = 600, 5000, 6000, 12
    src, dst = synth.chunglu(n, m, 2.1, 7)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    a = g.arrays()
    ids = np.arange(rank * T // world, (rank + 1) * T // world, dtype=np.uint64)
    smp = g.sample_ids(91, ids)
    mo, mem = smp["member_off"], smp["members"]
    members = [mem[mo[t]:mo[t + 1]] for t in range(len(ids))]
    delta = torch.zeros(n, dtype=torch.int64)
    for R in members:
        delta[torch.from_numpy(R.astype(np.int64))] += 1
    dist.all_reduce(delta, op=dist.ReduceOp.SUM)
    covered = np.zeros(len(ids), bool)
    inS = np.zeros(n, bool)
    W, f = g.W, g.f
    seeds, covs = [], []
    cov = 0
    for _ in range(k):
        best, best_key = -1, -1
        for v in range(n):
            if inS[v]:
                continue
            key = int(delta[v]) * W + T * ((1 << f) - int(a["w"][v]))  # exact Python integers
            if key > best_key:
                best, best_key = v, key
        inS[best] = True
        cov += int(delta[best])
        seeds.append(best)
        covs.append(cov)
        dec = torch.zeros(n, dtype=torch.int64)
        for t, R in enumerate(members):
            if not covered[t] and best in set(R.tolist()):
                covered[t] = True
                dec[torch.from_numpy(R.astype(np.int64))] += 1
        dist.all_reduce(dec, op=dist.ReduceOp.SUM)
        delta -= dec
    out[rank] = (seeds, covs)
    dist.destroy_process_group()


def test_two_rank_sharded_greedy_equals_single_process():
    import oracle
    import synth

    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_greedy_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = dict(out)
    n, m, T, k = 600, 5000, 6000, 12
    src, dst = synth.chunglu(n, m, 2.1, 7)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    od, oc, _ = oracle.OracleSketch(g, 91, T).greedy(k)
    assert res[0] == res[1]
    assert res[0][0] == od.tolist() and res[0][1] == oc.tolist()
