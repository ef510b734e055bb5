"""Continuous-batching query server: every request's result is the same when
it is served alone (one query per launch) and when it is batched with other
requests in flight (exact coverage counts, identical binary64 estimates),
and both equal skis_estimate and the CPU oracle."""
import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()
    n, m = 50_000, 400_000
    src, dst = synth.chunglu(n, m, 2.1, 41)
    g = skis.skis_load_graph(n, src, dst, weight_model=skis.SKIS_W_WC)
    s = skis.skis_sketch_create(g, 0x5EED0041)
    T = 300_000
    skis.skis_sample(s, T)
    sizes = synth.log_uniform_sizes(300, 1, 1000, 42)
    off, seeds = synth.seed_sets(n, sizes, 43)
    queries = [seeds[off[b]:off[b + 1]] for b in range(len(sizes))]
    yield n, src, dst, g, s, T, off, seeds, queries
    s.close()
    g.close()


def _serve(s, queries, slots, max_batch, seed_capacity=1 << 14, chunk=None):
    srv = skis.skis_server_create(s, slots=slots, max_batch=max_batch, seed_capacity=seed_capacity)
    tickets = []
    pending = set()
    chunk = chunk or len(queries)
    i = 0
    while i < len(queries) or pending:
        # requests arrive while earlier batches are in flight
        for q in queries[i:i + chunk]:
            t = skis.skis_server_submit(srv, q)
            tickets.append(t)
            pending.add(t)
        i += chunk
        done = skis.skis_server_progress(srv, wait=not (i < len(queries)))
        pending -= set(done.tolist())
    out = [skis.skis_server_poll(srv, t) for t in tickets]
    counts = skis.skis_server_counts(srv)
    srv.close()
    assert all(st == 1 for st, _, _ in out)
    return np.array([c for _, c, _ in out]), np.array([e for _, _, e in out]), counts


def test_results_alone_equal_results_in_the_mix(served):
    n, src, dst, g, s, T, off, seeds, queries = served
    cov1, est1, c1 = _serve(s, queries, slots=1, max_batch=1)  # one query per launch
    covm, estm, cm = _serve(s, queries, slots=4, max_batch=64, chunk=37)
    assert c1["batches"] == len(queries) and cm["batches"] < len(queries) // 4
    assert np.array_equal(cov1, covm)
    assert np.array_equal(est1, estm)  # bit-identical, not merely close
    cov, est = skis.skis_estimate(s, off, seeds)
    assert np.array_equal(cov, covm) and np.array_equal(est, estm)


def test_served_results_match_the_oracle(served):
    n, src, dst, g, s, T, off, seeds, queries = served
    covm, estm, _ = _serve(s, queries[:80], slots=3, max_batch=16, chunk=10)
    og = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    osk = oracle.OracleSketch(og, 0x5EED0041, T)
    o80 = np.concatenate([[0], np.cumsum([len(q) for q in queries[:80]])]).astype(np.int64)
    ocov, oest = osk.coverage(o80, np.concatenate(queries[:80]))
    assert np.array_equal(covm, ocov)
    np.testing.assert_allclose(estm, oest, rtol=1e-12, atol=0)


def test_admission_by_staging_memory_and_bad_requests(served):
    n, src, dst, g, s, T, off, seeds, queries = served
    # a staging capacity of 1000 seeds forces small batches; results unchanged
    big = [q for q in queries if len(q) > 300][:10]
    cov_a, est_a, c = _serve(s, big, slots=2, max_batch=64, seed_capacity=1000)
    assert c["batches"] >= len(big) // 3
    cov_b, est_b, _ = _serve(s, big, slots=1, max_batch=1, seed_capacity=1000)
    assert np.array_equal(cov_a, cov_b) and np.array_equal(est_a, est_b)
    srv = skis.skis_server_create(s, slots=1, max_batch=8, seed_capacity=1000)
    for bad in ([], [1, 1], [n], [-2], list(range(1001))):
        with pytest.raises(skis.SkisError) as e:
            skis.skis_server_submit(srv, np.array(bad, np.int32))
        assert e.value.code == skis.SKIS_EINVAL
    srv.close()
