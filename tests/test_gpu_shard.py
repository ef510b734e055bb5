"""The sketch sharded by sample id (Alg. 2's samples are independent and
keyed by id): ranks holding disjoint id ranges of one seed's sketch, their
counts summed through the library's all-reduce callback, give the greedy
seed sets, cumulative coverages, estimates and query answers of one process
holding the union sketch, and of the oracle, bit for bit."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis
import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SEED, K = 0x5EED0001, 50


@pytest.fixture(scope="module")
def union():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()
    spec, src, dst, _ = synth.workload("er-1e4-wc")
    T = spec["samples"]
    g = skis.skis_load_graph(spec["n"], src, dst, None, skis.SKIS_W_WC)
    s = skis.skis_sketch_create(g, SEED)
    skis.skis_sample(s, T)
    off, seeds = synth.seed_sets(spec["n"], [10] * 100 + [1, 2, 3, 500, 9999, 77], 7)
    greedy = skis.skis_greedy_maxcover(s, K)
    query = skis.skis_estimate(s, off, seeds)
    yield spec, src, dst, g, s, off, seeds, greedy, query
    s.close()
    g.close()


def test_one_rank_sharded_calls_equal_the_plain_ones(union):
    import torch

    spec, src, dst, g, s, off, seeds, greedy, query = union
    exchange = torch.zeros(spec["n"] + 1, dtype=torch.int64, device="cuda")
    calls = []
    sd, sc, se = skis.skis_greedy_maxcover_sharded(s, K, exchange, calls.append)  # one rank: the sum is itself
    assert calls == [1, spec["n"] + 1] + [spec["n"] + 1] * K
    for a, b in zip((sd, sc, se), greedy):
        assert np.array_equal(a, b)
    cov, est = skis.skis_estimate_sharded(s, off, seeds, exchange, lambda c: None)
    assert np.array_equal(cov, query[0]) and np.array_equal(est, query[1])


def test_failed_allreduce_is_reported(union):
    import torch

    spec, src, dst, g, s, off, seeds, greedy, query = union
    exchange = torch.zeros(spec["n"] + 1, dtype=torch.int64, device="cuda")

    def broken(count):
        raise RuntimeError("peer lost")

    with pytest.raises(skis.SkisError) as e:
        skis.skis_greedy_maxcover_sharded(s, 3, exchange, broken)
    assert e.value.code == skis.SKIS_ERR_EXCHANGE
    with pytest.raises(ValueError):
        skis.skis_greedy_maxcover_sharded(s, 3, exchange[: spec["n"]], lambda c: None)  # too short


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("split", [50_000, 31_337])
def test_two_ranks_on_gloo_match_the_union_and_the_oracle(union, tmp_path, split):
    spec, src, dst, g, s, off, seeds, greedy, query = union
    T = spec["samples"]
    ranges = [(0, split), (split, T - split)]
    port = _free_port()
    procs = []
    for r, (first, count) in enumerate(ranges):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "shard_worker.py"),
                                       str(tmp_path / "out"), str(first), str(count), str(K)], env=env, cwd=ROOT))
    for p in procs:
        assert p.wait(timeout=600) == 0
    osk = oracle.OracleSketch(oracle.OracleGraph(spec["n"], src, dst, model=oracle.W_WC), SEED, T)
    od, oc, oe = osk.greedy(K)
    ocov, oest = osk.coverage(off, seeds)
    for r in range(2):
        d = np.load(tmp_path / f"out.{r}.npz")
        assert np.array_equal(d["seeds"], greedy[0]) and np.array_equal(d["seeds"], od)
        assert np.array_equal(d["cov"], greedy[1]) and np.array_equal(d["cov"], oc)
        assert np.array_equal(d["est"], greedy[2])
        np.testing.assert_allclose(d["est"], oe, rtol=1e-12, atol=0)
        for c, e in (("qcov", "qest"), ("dcov", "dest")):
            assert np.array_equal(d[c], query[0]) and np.array_equal(d[c], ocov)
            assert np.array_equal(d[e], query[1])
            np.testing.assert_allclose(d[e], oest, rtol=1e-12, atol=0)
