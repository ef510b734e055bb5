"""Full-size parity on the serving workload's graph: directed Chung-Lu with
4M vertices and 70M edges (exponent 2.1, seed 4), weighted cascade, loaded
by the library and by the oracle.

- Graph structures (Sec. II-A canonical in-CSR, Eq. gamma_v, Eq. probu):
  offsets, CSR sources, thresholds, the CSR -> input permutation, w, the
  alias table, W and f, all bit-exact.
- Samples (Alg. 1) in both forms of the first step with the default tier
  split: ids [0, 20000) and blocks of 4 ids at every 400,000th id of the
  2 x 10^7-id stream the serving benchmark samples, each sample's (src,
  retries, |R|, coins, member set) bit-exact.
- Greedy max-coverage (Alg. 3, k = 50) and 64 queries (Eq. 21) on the sketch
  of ids [0, 20000): seeds and coverages bit-exact, estimates to a relative
  1e-12, by the inverted index and by the ordered scan."""
import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis
import synth

from test_gpu_parity import REL, assert_samples_equal

pytestmark = pytest.mark.gpu
SEED = 0x5EED0004
PREFIX = 20_000
BLOCK, STRIDE, NBLOCKS = 4, 400_000, 49


@pytest.fixture(scope="module")
def serve_graph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()
    spec, src, dst, _ = synth.workload("chunglu-4e6-wc-serve")
    g = skis.skis_load_graph(spec["n"], src, dst, None, skis.SKIS_W_WC)  # host arrays, copied by the library
    o = oracle.OracleGraph(spec["n"], src, dst, model=oracle.W_WC)
    del src, dst
    yield spec, g, o
    g.close()


def _sketch(g, bucket, first, count):
    s = skis.skis_sketch_create(g, SEED)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 1 if bucket else 0)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_ID, first)
    skis.skis_sample(s, count)
    return s


def test_full_serve_graph_structures(serve_graph):
    spec, g, o = serve_graph
    info = skis.skis_graph_get_info(g)
    assert (info["n"], info["m"]) == (spec["n"], spec["m"])
    assert info["W"] == o.W and info["f"] == o.f and info["row_uniform_tau"] == 1
    a, b = skis.skis_graph_export(g), o.arrays()
    for k in ("off", "src", "tau", "perm", "w", "prob", "alias"):
        assert a[k].shape == b[k].shape and np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("bucket", [True, False])
def test_full_serve_samples(serve_graph, bucket):
    spec, g, o = serve_graph
    ranges = [(0, PREFIX)] + [(i * STRIDE, BLOCK) for i in range(1, NBLOCKS + 1)]
    tiers = 0
    for first, count in ranges:
        s = _sketch(g, bucket, first, count)
        dev = skis.skis_sketch_export(s, first, count)
        ora = o.sample_ids(SEED, np.arange(first, first + count, dtype=np.uint64), bucket=bucket)
        assert_samples_equal(dev, ora)
        if count == PREFIX:
            st = skis.skis_sketch_stats(s)
            tiers = int(st["deferred"] > 0) + int(st["last_thread_ms"] > 0)
        s.close()
    assert tiers == 2  # the lane tier and the deeper tiers both took samples
    assert ranges[-1][0] + BLOCK <= 20_000_000  # every block lies in the serving benchmark's id stream


def test_full_serve_greedy_and_queries(serve_graph):
    spec, g, o = serve_graph
    s = _sketch(g, True, 0, PREFIX)
    osk = oracle.OracleSketch(o, SEED, PREFIX, bucket=True)
    sd, sc, se = skis.skis_greedy_maxcover(s, 50)
    od, oc, oe = osk.greedy(50)
    assert np.array_equal(sd, od) and np.array_equal(sc, oc)
    np.testing.assert_allclose(se, oe, rtol=REL, atol=0)
    off, seeds = synth.seed_sets(spec["n"], [10] * 64, 13)
    cov, est = skis.skis_estimate(s, off, seeds)  # through the inverted index greedy built
    ocov, oest = osk.coverage(off, seeds)
    assert np.array_equal(cov, ocov)
    np.testing.assert_allclose(est, oest, rtol=REL, atol=0)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_QUERY_INDEX, 3)  # the ordered scan, hashed filter (n > 2^20)
    cov2, est2 = skis.skis_estimate(s, off, seeds)
    assert np.array_equal(cov2, ocov) and np.array_equal(est2, est)
    s.close()
