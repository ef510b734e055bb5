"""Parity of the Linear Threshold variant (Sec. "Extensions to other diffusion
models", LT) between the CUDA path and the oracle: graph structures (exact
gamma as the row weight sum), every sample in walk order, long walks on the
slot tier, queries, greedy, the RIS form, and rejection of rows whose weights
sum above 1."""
import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis
import synth

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()
    yield


def _lt_p(dst, n, seed):
    """Per-edge LT weights: uniform shares of a row budget in (0, 1]."""
    deg = np.bincount(dst, minlength=n)
    u = synth.uniform_p(len(dst), seed, 0.05, 1.0)
    return u / np.maximum(deg[dst], 1) * 0.999


def _graphs():
    n1 = 20_000
    s1, d1 = synth.chunglu(n1, 150_000, 2.1, 91)
    n2 = 5_000
    s2, d2 = synth.chunglu(n2, 40_000, 2.1, 92)
    p2 = _lt_p(d2, n2, 93)
    # a path 0 -> 1 -> ... -> 399 (WC: every row one always-kept edge) plus a
    # few shortcuts: walks far longer than the lane tier holds
    n3 = 400
    s3 = np.concatenate([np.arange(n3 - 1), [5, 17, 260]]).astype(np.int32)
    d3 = np.concatenate([np.arange(1, n3), [300, 350, 390]]).astype(np.int32)
    # a longer path: walks beyond the lane-per-walk tier's 1024 members
    n4 = 2600
    s4 = np.arange(n4 - 1).astype(np.int32)
    d4 = np.arange(1, n4).astype(np.int32)
    return {
        "chunglu-wc": (n1, s1, d1, None, skis.SKIS_W_WC, oracle.W_WC),
        "path-long-wc": (n4, s4, d4, None, skis.SKIS_W_WC, oracle.W_WC),
        "chunglu-p": (n2, s2, d2, p2, skis.SKIS_W_EXPLICIT_P, oracle.W_P),
        "path-wc": (n3, s3, d3, None, skis.SKIS_W_WC, oracle.W_WC),
    }


GRAPHS = _graphs()


def _pair(name):
    n, src, dst, w, dm, om = GRAPHS[name]
    g = skis.skis_load_graph_lt(n, src, dst, w, dm)
    o = oracle.OracleGraph(n, src, dst, weights=w, model=om, lt=True)
    return n, g, o


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_lt_graph_matches_oracle(name):
    n, g, o = _pair(name)
    info = skis.skis_graph_get_info(g)
    assert info["diffusion"] == skis.SKIS_DIFF_LT and info["f"] == 32 and info["W"] == o.W
    a, b = skis.skis_graph_export(g), o.arrays()
    for k in ("off", "src", "tau", "perm", "w", "prob", "alias"):
        assert np.array_equal(a[k], b[k]), k
    g.close()


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("ris", [False, True])
def test_lt_samples_match_oracle_in_walk_order(name, ris):
    n, g, o = _pair(name)
    T = 30_000
    seed = 0x17A0 + len(name) + (7 if ris else 0)
    s = skis.skis_sketch_create(g, seed)
    if ris:
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_SAMPLER, 1)
    skis.skis_sample(s, T)
    dev = skis.skis_sketch_export(s, 0, T)
    ora = o.sample_ids(seed, np.arange(T, dtype=np.uint64), ris=ris)
    assert np.array_equal(dev["src"], ora["src"])
    assert (dev["retries"] == 0).all()
    assert np.array_equal(dev["len"].astype(np.int64), ora["len"])
    assert np.array_equal(dev["coins"], ora["coins"])
    assert np.array_equal(dev["members"], ora["members"])  # the walk order is unique
    st = skis.skis_sketch_stats(s)
    if name == "path-wc":
        assert st["to_warp"] > 0 and dev["len"].max() > 48  # the lane-per-walk tier took part
    if name == "path-long-wc":
        assert st["deferred"] > 0 and dev["len"].max() > 1024  # the slot tier took part
        # slot queues of 32 entries: the long walks move to the pass with n-entry queues
        s2 = skis.skis_sketch_create(g, seed)
        if ris:
            skis.skis_sketch_set_option(s2, skis.SKIS_OPT_SAMPLER, 1)
        skis.skis_sketch_set_option(s2, skis.SKIS_OPT_CTA_QUEUE_CAP, 32)
        skis.skis_sample(s2, T)
        dev2 = skis.skis_sketch_export(s2, 0, T)
        for k in ("src", "len", "coins", "members"):
            assert np.array_equal(dev2[k], dev[k]), k
        s2.close()
    s.close()
    g.close()


def test_lt_queries_and_greedy_match_oracle():
    n, g, o = _pair("chunglu-wc")
    seed, T = 0x5EED, 200_000
    s = skis.skis_sketch_create(g, seed)
    skis.skis_sample(s, T)
    osk = oracle.OracleSketch(o, seed, T)
    off, seeds = synth.seed_sets(n, [1, 10, 100] * 20 + [500], 95)
    cov, est = skis.skis_estimate(s, off, seeds)
    ocov, oest = osk.coverage(off, seeds)
    assert np.array_equal(cov, ocov)
    np.testing.assert_allclose(est, oest, rtol=REL, atol=0)
    sd, sc, se = skis.skis_greedy_maxcover(s, 30)
    od, oc, oe = osk.greedy(30)
    assert np.array_equal(sd, od) and np.array_equal(sc, oc)
    np.testing.assert_allclose(se, oe, rtol=REL, atol=0)
    s.close()
    g.close()


def test_lt_rejects_rows_above_one():
    src = np.array([1, 2, 3], np.int32)
    dst = np.array([0, 0, 0], np.int32)
    with pytest.raises(skis.SkisError) as e:
        skis.skis_load_graph_lt(4, src, dst, np.array([0.5, 0.4, 0.2]), skis.SKIS_W_EXPLICIT_P)
    assert e.value.code == skis.SKIS_EINVAL
    g = skis.skis_load_graph_lt(4, src, dst, np.array([0.5, 0.3, 0.2]), skis.SKIS_W_EXPLICIT_P)
    assert skis.skis_graph_get_info(g)["diffusion"] == skis.SKIS_DIFF_LT
    g.close()


def test_lt_sketch_through_the_server_and_noalloc():
    # queries on an LT sketch through the server and the no-allocation entry
    # point give skis_estimate's exact results
    n, g, o = _pair("chunglu-wc")
    s = skis.skis_sketch_create(g, 0x1717)
    skis.skis_sample(s, 100_000)
    off, seeds = synth.seed_sets(n, [1, 5, 50] * 6, 97)
    cov, est = skis.skis_estimate(s, off, seeds)
    srv = skis.skis_server_create(s, slots=2, max_batch=8)
    tickets = [skis.skis_server_submit(srv, seeds[off[b]:off[b + 1]]) for b in range(len(off) - 1)]
    skis.skis_server_progress(srv, wait=True)
    while True:
        res = [skis.skis_server_poll(srv, t) for t in tickets]
        if all(r[0] == 1 for r in res):
            break
        skis.skis_server_progress(srv, wait=True)
    assert np.array_equal(np.array([r[1] for r in res]), cov)
    assert np.array_equal(np.array([r[2] for r in res]), est)
    srv.close()
    import torch

    dev = torch.device("cuda", 0)
    d_off, d_seeds = torch.from_numpy(off).to(dev), torch.from_numpy(seeds).to(dev)
    d_cov = torch.empty(len(off) - 1, dtype=torch.int64, device=dev)
    d_est = torch.empty(len(off) - 1, dtype=torch.float64, device=dev)
    skis.skis_estimate_noalloc(s, d_off, d_seeds, d_cov, d_est)
    assert np.array_equal(d_cov.cpu().numpy(), cov) and np.array_equal(d_est.cpu().numpy(), est)
    s.close()
    g.close()
