"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on the same seeded inputs: graph structures, every sample's
(src, retries, |R|, coins, member set), coverage counts, estimates (relative
1e-12) and greedy seed sets. Bit-exact for all integers."""
import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis
import synth

pytestmark = pytest.mark.gpu

REL = 1e-12  # FP64 estimate tolerance (numerator and denominator are exact integers)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()
    yield


def _canon(member_off, members):
    """Members sorted within each sample (the member order is unspecified)."""
    lens = np.diff(member_off)
    seg = np.repeat(np.arange(len(lens)), lens)
    order = np.lexsort((members, seg))
    return members[order]


def assert_samples_equal(dev, ora):
    assert np.array_equal(dev["src"], ora["src"])
    assert np.array_equal(dev["retries"], ora["retries"])
    assert np.array_equal(dev["len"].astype(np.int64), ora["len"])
    assert np.array_equal(dev["coins"], ora["coins"])
    assert np.array_equal(_canon(dev["member_off"], dev["members"]), _canon(ora["member_off"], ora["members"]))


def _model(name):
    return {"wc": (skis.SKIS_W_WC, oracle.W_WC), "p": (skis.SKIS_W_EXPLICIT_P, oracle.W_P),
            "tau": (skis.SKIS_W_EXPLICIT_TAU, oracle.W_TAU), "tri": (skis.SKIS_W_TRI, oracle.W_TRI)}[name]


def _pair(n, src, dst, model, weights=None, weight_seed=0):
    dm, om = _model(model)
    g = skis.skis_load_graph(n, src, dst, weights, dm, weight_seed)
    o = oracle.OracleGraph(n, src, dst, weights=weights, model=om, weight_seed=weight_seed)
    return g, o


def _long_rows(model):
    """2000 vertices with in-rows of every gamma-chain path: three rows of
    2^15 in-edges and more (walked one a thread in one-warp blocks), four of
    2^10 .. 2^13 (ordered by degree class) and an ER background (row order);
    edges shuffled; WC, or per-edge p below 1e-4 so that the long rows stay
    sparse."""
    rng = np.random.default_rng(21)
    n = 2000
    ps, pd = [], []
    for v, d in ((0, 33000), (1, 34000), (2, 40000), (3, 1500), (4, 2100), (5, 1100), (6, 5000)):
        s = rng.integers(0, n - 1, d)
        ps.append(np.where(s >= v, s + 1, s))  # no self-loop
        pd.append(np.full(d, v))
    es, ed = synth.er(n, 16000, 22)
    src = np.concatenate(ps + [es]).astype(np.int32)
    dst = np.concatenate(pd + [ed]).astype(np.int32)
    order = rng.permutation(len(src))
    src, dst = src[order], dst[order]
    return n, src, dst, model, (None if model == "wc" else synth.uniform_p(len(src), 23, 0.0, 1e-4))


GRAPHS = {
    "er-wc": lambda: (3000, *synth.er(3000, 24000, 11), "wc", None),
    "chunglu-p": lambda: (20000, *synth.chunglu(20000, 150000, 2.1, 12), "p", synth.tri(150000, 12)),
    "chunglu-tri": lambda: (5000, *synth.chunglu(5000, 40000, 2.1, 13), "tri", None),
    "rmat-tau": lambda: (4096, *synth.rmat(12, 30000, 0.57, 0.19, 0.19, 14), "tau",
                         (synth.uniform_p(30000, 14, 0.0, 0.3) * 2**32).astype(np.uint32)),
    "long-rows-wc": lambda: _long_rows("wc"),
    "long-rows-p": lambda: _long_rows("p"),
    "tiny-ragged": lambda: (7, np.array([1, 2, 3, 4, 5, 6, 0, 2, 2], np.int32),
                            np.array([0, 0, 0, 1, 1, 2, 3, 3, 3], np.int32), "p",
                            np.array([0.5, 1.0, 0.2, 0.7, 0.0, 0.9, 0.3, 0.3, 1e-9])),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_graph_structures_match_oracle(name):
    n, src, dst, model, w = GRAPHS[name]()
    g, o = _pair(n, src, dst, model, w, weight_seed=5)
    a, b = skis.skis_graph_export(g), o.arrays()
    info = skis.skis_graph_get_info(g)
    assert info["W"] == o.W and info["f"] == o.f
    for k in ("off", "src", "tau", "perm", "w", "prob", "alias"):
        assert np.array_equal(a[k], b[k]), k
    g.close()


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_samples_match_oracle(name):
    n, src, dst, model, w = GRAPHS[name]()
    g, o = _pair(n, src, dst, model, w, weight_seed=5)
    T = 20000
    seed = 0x5EED0000 + len(name)
    s = skis.skis_sketch_create(g, seed)
    assert skis.skis_sample(s, T) == T
    dev = skis.skis_sketch_export(s, 0, T)
    ora = o.sample_ids(seed, np.arange(T, dtype=np.uint64))
    assert_samples_equal(dev, ora)
    st = skis.skis_sketch_stats(s)
    assert st["T"] == T and st["entries"] == int(ora["len"].sum()) and st["coins"] == int(ora["coins"].sum())
    s.close()
    g.close()


@pytest.fixture(scope="module")
def er_small():
    """The 10,000-vertex / 100,000-edge ER workload (WC), full size."""
    spec, src, dst, _ = synth.workload("er-1e4-wc")
    g, o = _pair(spec["n"], src, dst, "wc")
    seed = 0x5EED0001
    T = spec["samples"]
    osk = oracle.OracleSketch(o, seed, T)
    return spec, src, dst, g, o, osk, seed, T


def test_er_workload_full_parity(er_small):
    spec, src, dst, g, o, osk, seed, T = er_small
    s = skis.skis_sketch_create(g, seed)
    skis.skis_sample(s, T)
    st = skis.skis_sketch_stats(s)
    assert st["deferred"] > 0 and st["to_warp"] > 0  # all three tiers took part
    dev = skis.skis_sketch_export(s, 0, T)
    a = osk.arrays()
    ora = dict(src=a["src"], retries=a["retries"], len=np.diff(a["off"]), coins=a["coins"],
               member_off=a["off"], members=a["mem"])
    assert_samples_equal(dev, ora)
    # estimator: 100 seed sets of 10 uniform vertices, plus ragged sizes
    off, seeds = synth.seed_sets(spec["n"], [10] * 100 + [1, 2, 3, 500, 9999, 77], 7)
    cov, est = skis.skis_estimate(s, off, seeds)
    ocov, oest = osk.coverage(off, seeds)
    assert np.array_equal(cov, ocov)
    np.testing.assert_allclose(est, oest, rtol=REL, atol=0)
    # greedy max-coverage, k = 50
    sd, sc, se = skis.skis_greedy_maxcover(s, 50)
    od, oc, oe = osk.greedy(50)
    assert np.array_equal(sd, od) and np.array_equal(sc, oc)
    np.testing.assert_allclose(se, oe, rtol=REL, atol=0)
    # greedy built the inverted index: the same queries now walk it
    cov2, est2 = skis.skis_estimate(s, off, seeds)
    assert np.array_equal(cov2, ocov) and np.array_equal(est2, est)
    s.close()


def test_results_do_not_depend_on_launch_configuration(er_small):
    spec, src, dst, g, o, osk, seed, T = er_small
    ref = None
    # (thread-tier degree limit, thread blocks, warp blocks, CTA slots, initial arena,
    #  warp-tier coin budget)
    configs = ((None, 0, 0, 0, 0, 0), (0, 0, 3, 1, 1000, 1), (1 << 30, 5, 1000, 7, 50_000, 0),
               (8, 1, 2, 2, 0, 40), (0, 0, 0, 0, 0, 200))
    for max_deg, thread_blocks, warp_blocks, cta_slots, arena, warp_coins in configs:
        s = skis.skis_sketch_create(g, seed, arena)
        if warp_coins:
            skis.skis_sketch_set_option(s, skis.SKIS_OPT_WARP_MAX_COINS, warp_coins)
        if max_deg is not None:
            skis.skis_sketch_set_option(s, skis.SKIS_OPT_THREAD_MAX_DEG, max_deg)
        if thread_blocks:
            skis.skis_sketch_set_option(s, skis.SKIS_OPT_THREAD_BLOCKS, thread_blocks)
        if warp_blocks:
            skis.skis_sketch_set_option(s, skis.SKIS_OPT_WARP_BLOCKS, warp_blocks)
        if cta_slots:
            skis.skis_sketch_set_option(s, skis.SKIS_OPT_CTA_SLOTS, cta_slots)
        # appended in uneven pieces: ids continue across calls
        for c in (1, 999, 30000, T - 31000):
            skis.skis_sample(s, c)
        dev = skis.skis_sketch_export(s, 0, T)
        canon = (dev["src"], dev["retries"], dev["len"], dev["coins"], _canon(dev["member_off"], dev["members"]))
        if ref is None:
            ref = canon
        else:
            for x, y in zip(ref, canon):
                assert np.array_equal(x, y)
        s.close()


def test_device_queries_and_batches_over_64(er_small):
    torch = pytest.importorskip("torch")
    spec, src, dst, g, o, osk, seed, T = er_small
    s = skis.skis_sketch_create(g, seed)
    skis.skis_sample(s, T)
    sizes = synth.log_uniform_sizes(150, 1, 1000, 3)
    off, seeds = synth.seed_sets(spec["n"], sizes, 9)
    d_off = torch.from_numpy(off).cuda()
    d_seeds = torch.from_numpy(seeds).cuda()
    ocov, oest = osk.coverage(off, seeds)
    for mode in (2, 3, 1, 0):  # scan the sketch; scan it in id order; walk the inverted index; automatic
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_QUERY_INDEX, mode)
        d_cov = torch.empty(len(sizes), dtype=torch.int64, device="cuda")
        d_est = torch.empty(len(sizes), dtype=torch.float64, device="cuda")
        skis.skis_estimate(s, d_off, d_seeds, d_cov, d_est)
        torch.cuda.synchronize()
        assert np.array_equal(d_cov.cpu().numpy(), ocov)
        np.testing.assert_allclose(d_est.cpu().numpy(), oest, rtol=REL, atol=0)
    s.close()


def test_bad_inputs_are_rejected():
    n = 10
    with pytest.raises(skis.SkisError) as e:
        skis.skis_load_graph(n, np.array([1, 2], np.int32), np.array([0, 2], np.int32))  # self-loop
    assert e.value.code == skis.SKIS_EINVAL
    with pytest.raises(skis.SkisError):
        skis.skis_load_graph(n, np.array([1, 10], np.int32), np.array([0, 0], np.int32))
    with pytest.raises(skis.SkisError):
        skis.skis_load_graph(n, np.array([1, 2], np.int32), np.array([0, 0], np.int32),
                             np.array([0.5, np.nan]), skis.SKIS_W_EXPLICIT_P)
    g = skis.skis_load_graph(n, np.array([1, 2, 3], np.int32), np.array([0, 0, 0], np.int32))
    s = skis.skis_sketch_create(g, 1)
    with pytest.raises(skis.SkisError):
        skis.skis_estimate(s, np.array([0, 1], np.int64), np.array([0], np.int32))  # no samples yet
    skis.skis_sample(s, 100)
    for sets in ([[]], [[1, 1]], [[10]], [[-1]]):
        off = np.concatenate([[0], np.cumsum([len(x) for x in sets])]).astype(np.int64)
        seeds = np.array([v for x in sets for v in x], np.int32)
        with pytest.raises(skis.SkisError) as e:
            skis.skis_estimate(s, off, seeds)
        assert e.value.code == skis.SKIS_EINVAL
    with pytest.raises(skis.SkisError):
        skis.skis_greedy_maxcover(s, n + 1)
    for opt, bad in ((skis.SKIS_OPT_WARP_MAX_COINS, 0), (skis.SKIS_OPT_WARP_MAX_COINS, (1 << 31) + 1),
                     (skis.SKIS_OPT_THREAD_MAX_STEPS, 0), (99, 1)):
        with pytest.raises(skis.SkisError) as e:
            skis.skis_sketch_set_option(s, opt, bad)
        assert e.value.code == skis.SKIS_EINVAL
    s.close()
    g.close()
    # Gamma = 0: no non-singular sample exists
    g = skis.skis_load_graph(3, np.array([1, 2], np.int32), np.array([0, 0], np.int32),
                             np.array([0, 0], np.uint32), skis.SKIS_W_EXPLICIT_TAU)
    s = skis.skis_sketch_create(g, 1)
    with pytest.raises(skis.SkisError) as e:
        skis.skis_sample(s, 10)
    assert e.value.code == skis.SKIS_EINVAL
    s.close()
    g.close()


def test_retry_cap_reports_error_with_the_oracle():
    g, o = _pair(2, np.array([1], np.int32), np.array([0], np.int32), "tau", np.array([1], np.uint32))
    s = skis.skis_sketch_create(g, 5)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_RETRY_CAP, 8)
    with pytest.raises(skis.SkisError) as e:
        skis.skis_sample(s, 50)
    assert e.value.code == skis.SKIS_ERR_RETRY_LIMIT
    dev = skis.skis_sketch_export(s, 0, 50)
    ora = o.sample_ids(5, np.arange(50, dtype=np.uint64), retry_cap=8)
    assert (ora["status"] == oracle.ORC_ERETRY).all()
    assert np.array_equal(dev["retries"], ora["retries"]) and (dev["len"] == 0).all()
    assert np.array_equal(dev["coins"], ora["coins"])
    s.close()
    g.close()


def test_always_live_giant_samples_take_the_cta_tier():
    # every edge live on a dense ER graph: each sample is a large ancestor set
    n, m = 6000, 30000
    src, dst = synth.er(n, m, 21)
    tau = np.full(m, 0xFFFFFFFF, np.uint32)
    g, o = _pair(n, src, dst, "tau", tau)
    ora = o.sample_ids(77, np.arange(T := 300, dtype=np.uint64))
    assert ora["len"].max() > 1000
    # default slot queues, then queues of 32 and 1000 entries per CTA-tier slot: the
    # samples that outgrow them move to the pass with n-entry queues
    for cap in (None, 32, 1000):
        s = skis.skis_sketch_create(g, 77, 1 << 16)
        if cap:
            skis.skis_sketch_set_option(s, skis.SKIS_OPT_CTA_QUEUE_CAP, cap)
        skis.skis_sample(s, T)
        st = skis.skis_sketch_stats(s)
        assert st["deferred"] > 0 and st["arena_capacity"] > (1 << 16)  # the arena grew
        assert_samples_equal(skis.skis_sketch_export(s, 0, T), ora)
        s.close()
    g.close()


def test_single_vertex_and_edgeless_graphs():
    g = skis.skis_load_graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    info = skis.skis_graph_get_info(g)
    assert info["W"] == 0 and info["m"] == 0
    a = skis.skis_graph_export(g)
    assert a["off"].tolist() == [0, 0]
    g.close()


# --------------------------------------------------- full-size workload
@pytest.fixture(scope="module", params=["bucket", "rejection"])
def chunglu_full(request):
    """The 1M-vertex / 10M-edge Chung-Lu TRI workload with 10M samples, in
    the launch configuration the benchmark uses (default tiers, bucket first
    step), and with the rejection first step."""
    spec, src, dst, p = synth.workload("chunglu-1e6-tri")
    seed = 0x5EED0002
    bucket = request.param == "bucket"
    g = skis.skis_load_graph(spec["n"], src, dst, p, skis.SKIS_W_EXPLICIT_P)
    s = skis.skis_sketch_create(g, seed, int(spec["samples"] * 5.5))
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 1 if bucket else 0)
    skis.skis_sample(s, spec["samples"])
    o = oracle.OracleGraph(spec["n"], src, dst, weights=p, model=oracle.W_P)
    yield spec, g, s, o, seed, bucket
    s.close()
    g.close()


def test_full_size_graph_and_sampled_ids(chunglu_full):
    spec, g, s, o, seed, bucket = chunglu_full
    a, b = skis.skis_graph_export(g), o.arrays()
    for k in ("off", "src", "tau", "perm", "w", "prob", "alias"):
        assert np.array_equal(a[k], b[k]), k
    T = spec["samples"]
    dev = skis.skis_sketch_export(s, 0, T)
    rng = np.random.default_rng(0)
    ids = np.unique(np.concatenate([np.arange(2000), np.arange(T - 2000, T), rng.integers(0, T, 30000)]))
    ora = o.sample_ids(seed, ids.astype(np.uint64), bucket=bucket)
    mo = dev["member_off"]
    sub = dict(src=dev["src"][ids], retries=dev["retries"][ids], len=dev["len"][ids], coins=dev["coins"][ids])
    lens = np.diff(mo)[ids]
    sub["member_off"] = np.concatenate([[0], np.cumsum(lens)])
    sub["members"] = np.concatenate([dev["members"][mo[i]:mo[i + 1]] for i in ids])
    assert_samples_equal(sub, ora)


def test_full_size_greedy_and_coverage(chunglu_full):
    spec, g, s, o, seed, bucket = chunglu_full
    osk = oracle.OracleSketch(o, seed, spec["samples"], bucket=bucket)
    k = spec["k"]
    sd, sc, se = skis.skis_greedy_maxcover(s, k)
    od, oc, oe = osk.greedy(k)
    assert np.array_equal(sd, od) and np.array_equal(sc, oc)
    np.testing.assert_allclose(se, oe, rtol=REL, atol=0)
    off, seeds = synth.seed_sets(spec["n"], [10] * 64, 11)
    cov, est = skis.skis_estimate(s, off, seeds)
    ocov, oest = osk.coverage(off, seeds)
    assert np.array_equal(cov, ocov)
    np.testing.assert_allclose(est, oest, rtol=REL, atol=0)
    # the same queries, and a ragged batch of 150, by the scan of the members in id order
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_QUERY_INDEX, 2)
    cov2, est2 = skis.skis_estimate(s, off, seeds)
    assert np.array_equal(cov2, ocov) and np.array_equal(est2, est)
    off3, seeds3 = synth.seed_sets(spec["n"], synth.log_uniform_sizes(150, 1, 1000, 12), 13)
    cov3, est3 = skis.skis_estimate(s, off3, seeds3)
    ocov3, oest3 = osk.coverage(off3, seeds3)
    assert np.array_equal(cov3, ocov3)
    np.testing.assert_allclose(est3, oest3, rtol=REL, atol=0)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_QUERY_INDEX, 0)


def test_autotuned_split_gives_the_same_samples(er_small):
    spec, src, dst, g, o, osk, seed, T = er_small
    s = skis.skis_sketch_create(g, seed)
    tune = skis.skis_sketch_autotune(s, 20_000)
    assert tune["max_deg"] in (0, 64, 128, 192, 256, 512) and tune["max_steps"] in (128, 256, 1024)
    assert tune["warp_max_coins"] in (4096, 16384, 65536, 262144)
    assert len(tune["candidate_ms"]) == 20 and all(x > 0 for x in tune["candidate_ms"])
    st = skis.skis_sketch_stats(s)
    assert (st["thread_max_deg"], st["thread_max_steps"]) == (tune["max_deg"], tune["max_steps"])
    skis.skis_sample(s, 30_000)
    dev = skis.skis_sketch_export(s, 0, 30_000)
    ora = o.sample_ids(seed, np.arange(30_000, dtype=np.uint64))
    assert_samples_equal(dev, ora)
    s.close()


@pytest.mark.parametrize("model", ["wc", "p"])
def test_ris_variant_matches_oracle(model):
    # plain RIS: uniform sources (isolated and zero-in-degree vertices too),
    # one unconditioned round, n Cov / T, coverage-only greedy
    n = 30_000
    src, dst = synth.chunglu(n - 1000, 200_000, 2.1, 61)  # vertices >= n - 1000 have no edges
    w = synth.tri(200_000, 61) if model == "p" else None
    g, o = _pair(n, src, dst, model, w)
    seed, T = 0x515, 200_000
    s = skis.skis_sketch_create(g, seed)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_SAMPLER, 1)
    skis.skis_sample(s, T)
    with pytest.raises(skis.SkisError):
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_SAMPLER, 0)  # fixed once samples exist
    dev = skis.skis_sketch_export(s, 0, T)
    osk = oracle.OracleSketch(o, seed, T, ris=True)
    a = osk.arrays()
    ora = dict(src=a["src"], retries=a["retries"], len=np.diff(a["off"]), coins=a["coins"],
               member_off=a["off"], members=a["mem"])
    assert_samples_equal(dev, ora)
    assert (dev["len"] == 1).any()  # singular samples
    off, seeds = synth.seed_sets(n, [1, 10, 100] * 30, 62)
    cov, est = skis.skis_estimate(s, off, seeds)
    ocov, oest = osk.coverage(off, seeds)
    assert np.array_equal(cov, ocov)
    np.testing.assert_allclose(est, oest, rtol=REL, atol=0)
    sd, sc, se = skis.skis_greedy_maxcover(s, 20)
    od, oc, oe = osk.greedy(20)
    assert np.array_equal(sd, od) and np.array_equal(sc, oc)
    np.testing.assert_allclose(se, oe, rtol=REL, atol=0)
    s.close()
    g.close()


def test_stop_at_size_matches_oracle(er_small):
    # sample until the total size reaches h n ln n (h = 1 here): the same
    # sample count and samples as the oracle's sequential stop rule
    spec, src, dst, g, o, osk, seed, T = er_small
    n = spec["n"]
    target = int(1.0 * n * np.log(n))
    s = skis.skis_sketch_create(g, seed)
    appended, T1 = skis.skis_sample_to_size(s, target)
    ref = oracle.OracleSketch(o, seed, 10 * target, stop_entries=target)
    assert appended == T1 == ref.T
    st = skis.skis_sketch_stats(s)
    a = ref.arrays()
    assert st["entries"] == int(a["off"][-1]) >= target > int(a["off"][-2])
    dev = skis.skis_sketch_export(s, 0, T1)
    ora = dict(src=a["src"], retries=a["retries"], len=np.diff(a["off"]), coins=a["coins"],
               member_off=a["off"], members=a["mem"])
    assert_samples_equal(dev, ora)
    off, seeds = synth.seed_sets(n, [10] * 20, 71)
    cov, est = skis.skis_estimate(s, off, seeds)
    ocov, oest = ref.coverage(off, seeds)
    assert np.array_equal(cov, ocov)
    np.testing.assert_allclose(est, oest, rtol=REL, atol=0)
    # a larger target continues from the truncated sketch with the same ids
    appended2, T2 = skis.skis_sample_to_size(s, 2 * target)
    ref2 = oracle.OracleSketch(o, seed, 10 * target, stop_entries=2 * target)
    assert T2 == ref2.T and appended2 == T2 - T1
    # greedy after a truncation: the index counts the kept samples only
    sd, sc, se = skis.skis_greedy_maxcover(s, 10)
    od, oc, oe = ref2.greedy(10)
    assert np.array_equal(sd, od) and np.array_equal(sc, oc)
    # a reached target appends nothing; max_count bounds a call
    assert skis.skis_sample_to_size(s, target) == (0, T2)
    assert skis.skis_sample_to_size(s, 100 * target, max_count=1000) == (1000, T2 + 1000)
    s.close()


def test_index_after_sampling_in_several_calls(er_small):
    # the per-vertex counts kept while sampling add up over calls
    spec, src, dst, g, o, osk, seed, T = er_small
    s = skis.skis_sketch_create(g, seed)
    for part in (T // 5, T // 3, T - T // 5 - T // 3):
        skis.skis_sample(s, part)
    sd, sc, se = skis.skis_greedy_maxcover(s, 25)
    od, oc, oe = osk.greedy(25)
    assert np.array_equal(sd, od) and np.array_equal(sc, oc)
    np.testing.assert_allclose(se, oe, rtol=REL, atol=0)
    s.close()


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bucket_first_step_matches_oracle(name):
    # the bucket form of the first step (Eq. probn), on every tier
    n, src, dst, model, w = GRAPHS[name]()
    g, o = _pair(n, src, dst, model, w, weight_seed=5)
    T = 20000
    seed = 0xB0C0 + len(name)
    for max_deg in (256, 0):  # with and without the lane tier
        s = skis.skis_sketch_create(g, seed)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 1)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_THREAD_MAX_DEG, max_deg)
        skis.skis_sample(s, T)
        with pytest.raises(skis.SkisError):
            skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 0)  # fixed once samples exist
        dev = skis.skis_sketch_export(s, 0, T)
        ora = o.sample_ids(seed, np.arange(T, dtype=np.uint64), bucket=True)
        assert_samples_equal(dev, ora)
        assert (dev["retries"] == 0).all()
        s.close()
    g.close()


def test_bucket_first_step_full_er_workload(er_small):
    spec, src, dst, g, o, osk, seed, T = er_small
    s = skis.skis_sketch_create(g, seed)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 1)
    skis.skis_sample(s, T)
    st = skis.skis_sketch_stats(s)
    assert st["deferred"] > 0 and st["retries"] == 0  # the CTA tier took part
    ref = oracle.OracleSketch(o, seed, T, bucket=True)
    a = ref.arrays()
    dev = skis.skis_sketch_export(s, 0, T)
    ora = dict(src=a["src"], retries=a["retries"], len=np.diff(a["off"]), coins=a["coins"],
               member_off=a["off"], members=a["mem"])
    assert_samples_equal(dev, ora)
    off, seeds = synth.seed_sets(spec["n"], [10] * 50, 77)
    cov, est = skis.skis_estimate(s, off, seeds)
    ocov, oest = ref.coverage(off, seeds)
    assert np.array_equal(cov, ocov)
    np.testing.assert_allclose(est, oest, rtol=REL, atol=0)
    s.close()


@pytest.mark.parametrize("bucket", [False, True])
def test_hub_rows_on_every_tier_match_oracle(bucket):
    # R-MAT with weighted cascade: in-rows of thousands of edges (the top one
    # about 7K), so a sample that reaches a hub draws its whole row. Sent
    # through each tier in turn the samples are the oracle's; on the CTA tier
    # a window holding such a row deals its quads several to a lane.
    n, m = 1 << 13, 32 << 13
    src, dst = synth.rmat(13, m, 0.57, 0.19, 0.19, 17)
    g, o = _pair(n, src, dst, "wc")
    seed, T = 0x5EED0017, 600
    ora = o.sample_ids(seed, np.arange(T, dtype=np.uint64), bucket=bucket)
    assert np.bincount(dst, minlength=n).max() >= 4 * 64  # rows of 64+ quads exist
    cta = {skis.SKIS_OPT_THREAD_MAX_DEG: 0, skis.SKIS_OPT_WARP_MAX_COINS: 1}
    # on the CTA tier: the default hub threshold, no hub loop, every row
    # through the hub loop, and a low threshold mixing both in one window
    configs = ({}, {skis.SKIS_OPT_THREAD_MAX_DEG: 0}, cta, {**cta, skis.SKIS_OPT_CTA_HUB_QUADS: 0},
               {**cta, skis.SKIS_OPT_CTA_HUB_QUADS: 1}, {**cta, skis.SKIS_OPT_CTA_HUB_QUADS: 3})
    for opts in configs:
        s = skis.skis_sketch_create(g, seed)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 1 if bucket else 0)
        for k, v in opts.items():
            skis.skis_sketch_set_option(s, k, v)
        skis.skis_sample(s, T)
        assert_samples_equal(skis.skis_sketch_export(s, 0, T), ora)
        if skis.SKIS_OPT_WARP_MAX_COINS in opts:
            assert skis.skis_sketch_stats(s)["deferred"] > T // 4  # most samples ran on the CTA tier
        s.close()
    g.close()


@pytest.mark.parametrize("name", ["rmat-tau", "chunglu-p", "tiny-ragged"])
def test_cta_hub_loop_with_per_edge_thresholds(name):
    # every sample on the CTA tier and every row through its hub loop, with a
    # threshold per edge (sentinels and zero thresholds in tiny-ragged)
    n, src, dst, model, w = GRAPHS[name]()
    g, o = _pair(n, src, dst, model, w, weight_seed=5)
    T, seed = 3000, 0x4B0B
    ora = o.sample_ids(seed, np.arange(T, dtype=np.uint64))
    for hub in (1, 2):
        s = skis.skis_sketch_create(g, seed)
        for k, v in ((skis.SKIS_OPT_THREAD_MAX_DEG, 0), (skis.SKIS_OPT_WARP_MAX_COINS, 1),
                     (skis.SKIS_OPT_CTA_HUB_QUADS, hub)):
            skis.skis_sketch_set_option(s, k, v)
        skis.skis_sample(s, T)
        assert skis.skis_sketch_stats(s)["cta_hub_quads"] == hub
        assert_samples_equal(skis.skis_sketch_export(s, 0, T), ora)
        s.close()
    g.close()


@pytest.mark.parametrize("first_id", [1, 123_456_789, (1 << 40) + 17])
def test_first_id_places_the_samples_of_one_sketch(first_id):
    # a sketch whose first sample id is F holds exactly samples F, F+1, ...
    # of the one sketch the seed defines (its id-range shard)
    n, src, dst, model, w = GRAPHS["chunglu-p"]()
    g, o = _pair(n, src, dst, model, w)
    seed, T = 0x5A4D, 20000
    s = skis.skis_sketch_create(g, seed)
    skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_ID, first_id)
    assert skis.skis_sample(s, T // 4) == first_id + T // 4
    assert skis.skis_sample(s, T - T // 4) == first_id + T
    with pytest.raises(skis.SkisError):
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_ID, 0)  # fixed once samples exist
    st = skis.skis_sketch_stats(s)
    assert st["T"] == T and st["first_id"] == first_id
    ids = np.arange(first_id, first_id + T, dtype=np.uint64)
    assert_samples_equal(skis.skis_sketch_export(s, first_id, T), o.sample_ids(seed, ids))
    with pytest.raises(skis.SkisError):
        skis.skis_sketch_export(s, first_id - 1, 2)  # below the sketch's ids
    osk_ids = o.sample_ids(seed, ids)
    off, seeds = synth.seed_sets(n, [10] * 20, 5)
    cov, _ = skis.skis_estimate(s, off, seeds)
    member = [set(osk_ids["members"][osk_ids["member_off"][t]:osk_ids["member_off"][t + 1]]) for t in range(T)]
    want = [sum(1 for mset in member if mset.intersection(seeds[off[b]:off[b + 1]])) for b in range(20)]
    assert cov.tolist() == want
    s.close()
    g.close()
