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
