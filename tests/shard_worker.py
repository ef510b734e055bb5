"""One rank of the sharded-sketch test (run as a process by
tests/test_gpu_shard.py, not collected by pytest): rank r of N holds sample
ids [F_r, F_r + T_r) of one sketch, the ranks' coverage counts and Delta are
summed over a gloo process group through the library's all-reduce callback,
and the results are written to <out>.<rank>.npz."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def main():
    import torch
    import torch.distributed as dist

    import paper_1709_03565_gb300 as skis
    import synth

    out, first, count, k = sys.argv[1], int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4])
    rank = int(os.environ["RANK"])
    dist.init_process_group("gloo")
    torch.cuda.set_device(0)
    skis.lib()
    spec, src, dst, _ = synth.workload("er-1e4-wc")
    n = spec["n"]
    g = skis.skis_load_graph(n, src, dst, None, skis.SKIS_W_WC)
    s = skis.skis_sketch_create(g, 0x5EED0001)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_ID, first)
    skis.skis_sample(s, count)
    exchange = torch.zeros(n + 1, dtype=torch.int64, device="cuda")

    def allreduce(c):  # host-side sum over the gloo group, copied back
        t = exchange[:c].cpu()
        dist.all_reduce(t)
        exchange[:c].copy_(t)

    sd, sc, se = skis.skis_greedy_maxcover_sharded(s, k, exchange, allreduce)
    off, seeds = synth.seed_sets(n, [10] * 100 + [1, 2, 3, 500, 9999, 77], 7)
    cov, est = skis.skis_estimate_sharded(s, off, seeds, exchange, allreduce)
    d_off, d_seeds = torch.from_numpy(off).cuda(), torch.from_numpy(seeds).cuda()
    d_cov = torch.empty(len(off) - 1, dtype=torch.int64, device="cuda")
    d_est = torch.empty(len(off) - 1, dtype=torch.float64, device="cuda")
    skis.skis_estimate_sharded(s, d_off, d_seeds, exchange, allreduce, d_cov, d_est)
    np.savez(f"{out}.{rank}.npz", seeds=sd, cov=sc, est=se, qcov=cov, qest=est, dcov=d_cov.cpu().numpy(),
             dest=d_est.cpu().numpy())
    s.close()
    g.close()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
