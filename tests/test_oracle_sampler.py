"""Pins of the oracle's IIS sampler (Alg. 1) against the exact law of Lemma 2
obtained by enumerating every live-edge world, against plain reverse BFS on
always-live graphs, and against the retry cap and the work counters."""
from collections import Counter

import numpy as np
import pytest
from scipy import sparse
from scipy.sparse import csgraph

import oracle
import synth
from exact import SENT, iis_law, p_eff


def _tiny_graph(kind):
    if kind == "mixed":
        # 5 vertices, 10 edges incl. a parallel pair and an always-live edge
        src = [1, 2, 3, 0, 4, 2, 3, 3, 4, 1]
        dst = [0, 0, 1, 2, 2, 3, 4, 4, 0, 3]
        p = np.array([0.5, 0.3, 0.7, 0.2, 1.0, 0.45, 0.6, 0.25, 0.15, 0.35])
        return 5, src, dst, p, oracle.W_P
    if kind == "wc":
        src = [1, 2, 3, 0, 4, 2, 3, 4, 0, 1, 4]
        dst = [0, 0, 1, 2, 2, 3, 4, 1, 4, 3, 3]
        return 5, src, dst, None, oracle.W_WC
    if kind == "tri":
        src = [1, 2, 3, 4, 0, 2, 3, 4, 1]
        dst = [0, 0, 0, 0, 1, 1, 2, 3, 4]
        return 5, src, dst, None, oracle.W_TRI
    raise KeyError(kind)


def _collect(g, seed, T):
    out = g.sample_ids(seed, np.arange(T, dtype=np.uint64))
    mo = out["member_off"]
    mem = out["members"]
    cnt = Counter()
    for t in range(T):
        cnt[(int(out["src"][t]), frozenset(mem[mo[t]:mo[t + 1]].tolist()))] += 1
    return out, cnt


@pytest.mark.parametrize("kind", ["mixed", "wc", "tri"])
def test_iis_law_matches_exact_enumeration(kind):
    """Lemma 2: Pr[(src, R)] = (w_src / W) * Pr[eta^-(src) = R] / gamma_src."""
    n, src, dst, p, model = _tiny_graph(kind)
    g = oracle.OracleGraph(n, src, dst, weights=p, model=model, weight_seed=3)
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    dst_csr = np.repeat(np.arange(n), np.diff(a["off"])).tolist()
    law = iis_law(n, a["src"].tolist(), dst_csr, probs, a["w"].tolist(), g.W)
    assert abs(float(sum(law.values())) - 1.0) < 1e-12
    T = 300_000
    out, cnt = _collect(g, 0x1234 + len(kind), T)
    assert (out["status"] == 0).all()
    # no sample is singular, and every observed outcome has positive probability
    assert all(len(R) >= 2 for (_, R) in cnt)
    assert set(cnt) <= set(law)
    # chi-square over outcomes, pooling the rare ones
    exp = {k: float(v) * T for k, v in law.items()}
    big = [k for k in exp if exp[k] >= 20]
    small = [k for k in exp if exp[k] < 20]
    obs = [cnt.get(k, 0) for k in big] + [sum(cnt.get(k, 0) for k in small)]
    ex = [exp[k] for k in big] + [sum(exp[k] for k in small)]
    if ex[-1] == 0:
        obs, ex = obs[:-1], ex[:-1]
    obs, ex = np.array(obs, float), np.array(ex, float)
    chi2 = ((obs - ex) ** 2 / ex).sum()
    dof = len(ex) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof)


def test_retries_are_geometric_in_gamma():
    # in-star with a single edge of probability p: retries ~ Geometric(p)
    p = 0.05
    g = oracle.OracleGraph(2, [1], [0], weights=np.array([p]), model=oracle.W_P)
    out = g.sample_ids(99, np.arange(100_000, dtype=np.uint64))
    pe = float(p_eff(g.arrays()["tau"][0]))
    r = out["retries"].astype(float)
    mean = (1 - pe) / pe
    sd = np.sqrt((1 - pe) / pe**2 / len(r))
    assert abs(r.mean() - mean) < 5 * sd
    assert (out["len"] == 2).all() and (out["src"] == 0).all()
    # coins = d_in(src) * (retries + 1) + in-degrees of the other members (0 here)
    assert np.array_equal(out["coins"], out["retries"].astype(np.uint64) + 1)


def test_retry_cap_reports_error():
    # one edge with tau = 1: Pr[live] = 2^-32, the cap of 8 rounds is reached
    g = oracle.OracleGraph(2, [1], [0], weights=np.array([1], np.uint32), model=oracle.W_TAU)
    out = g.sample_ids(5, np.arange(50, dtype=np.uint64), retry_cap=8)
    assert (out["status"] == oracle.ORC_ERETRY).all()
    assert (out["retries"] == 8).all() and (out["len"] == 0).all()


@pytest.mark.parametrize("seed", [1, 2])
def test_always_live_sample_is_the_ancestor_set(seed):
    # every edge live: R_j is exactly the set of vertices that reach src(R_j)
    n, m = 400, 900
    src, dst = synth.er(n, m, seed)
    tau = np.full(m, SENT, np.uint32)
    g = oracle.OracleGraph(n, src, dst, weights=tau, model=oracle.W_TAU)
    a = g.arrays()
    deg = np.diff(a["off"])
    rev = sparse.csr_matrix((np.ones(m), (dst, src)), shape=(n, n))
    T = 300
    out = g.sample_ids(seed + 10, np.arange(T, dtype=np.uint64))
    mo, mem = out["member_off"], out["members"]
    for t in range(T):
        v = int(out["src"][t])
        anc = set(csgraph.breadth_first_order(rev, v, directed=True, return_predecessors=False).tolist())
        R = mem[mo[t]:mo[t + 1]]
        assert set(R.tolist()) == anc and len(R) == len(anc)
        assert out["retries"][t] == 0
        assert int(out["coins"][t]) == int(deg[R].sum())


def test_samples_are_pure_functions_of_seed_and_id():
    n, m = 1000, 8000
    src, dst = synth.er(n, m, 4)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    ids = np.array([5, 17, 123456789, 2**40 + 3], dtype=np.uint64)
    a = g.sample_ids(42, ids)
    b = g.sample_ids(42, ids[::-1].copy())
    for k in ("src", "retries", "len", "coins"):
        assert np.array_equal(a[k], b[k][::-1])
    c = g.sample_ids(43, ids)
    assert not np.array_equal(a["src"], c["src"]) or not np.array_equal(a["len"], c["len"])
    # the same graph given in another input order gives the same samples
    sh = np.random.default_rng(0).permutation(m)
    g2 = oracle.OracleGraph(n, src[sh], dst[sh], model=oracle.W_WC)
    d = g2.sample_ids(42, ids)
    for k in ("src", "retries", "len", "coins"):
        assert np.array_equal(a[k], d[k])
    for t in range(len(ids)):
        x = a["members"][a["member_off"][t]:a["member_off"][t + 1]]
        y = d["members"][d["member_off"][t]:d["member_off"][t + 1]]
        assert sorted(x.tolist()) == sorted(y.tolist())


def test_graph_without_non_singular_samples_is_rejected():
    g = oracle.OracleGraph(3, [1, 2], [0, 0], weights=np.array([0, 0], np.uint32), model=oracle.W_TAU)
    assert g.W == 0
    with pytest.raises(oracle.OracleError):
        g.sample_ids(1, np.arange(3, dtype=np.uint64))
    with pytest.raises(oracle.OracleError):
        oracle.OracleSketch(g, 1, 10)


def _coin(seed, domain, retry, j, e):
    """The coin word of edge e (reading R6), from the KAT-pinned Philox:
    counter (q mod 2^32, (q >> 32) | retry << 4 | domain << 28, j lo, j hi),
    q = e >> 2, key = (seed lo, seed hi), word e mod 4."""
    q = e >> 2
    ctr = [q & 0xFFFFFFFF, ((q >> 32) & 0xF) | ((retry & 0xFFFFFF) << 4) | (domain << 28),
           j & 0xFFFFFFFF, j >> 32]
    return int(oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])[e & 3])


def test_first_step_coin_boundary_is_strict():
    # single edge 1 -> 0 (CSR position 0): the round-0 FIRST coin x decides;
    # tau = x is dead (x < tau fails), tau = x + 1 is live
    seed = 0x5EED
    for j in (0, 1, 7, 2**33 + 5):
        x = _coin(seed, 2, 0, j, 0)
        if x >= SENT - 1:
            continue
        dead = oracle.OracleGraph(2, [1], [0], weights=np.array([x], np.uint32), model=oracle.W_TAU)
        live = oracle.OracleGraph(2, [1], [0], weights=np.array([x + 1], np.uint32), model=oracle.W_TAU)
        a = dead.sample_ids(seed, np.array([j], np.uint64))
        b = live.sample_ids(seed, np.array([j], np.uint64))
        assert a["retries"][0] >= 1 and b["retries"][0] == 0


def test_bfs_coin_boundary_is_strict():
    # path 2 -> 1 -> 0 with 1 -> 0 always live. CSR: position 0 is (1 -> 0),
    # position 1 is (2 -> 1). In a sample with source 0, vertex 2 joins R iff
    # the BFS coin of edge 1 is below its threshold.
    seed = 0xC0FFEE
    checked = 0
    for j in range(200):
        x = _coin(seed, 3, 0, j, 1)
        if x == 0 or x >= SENT - 1:
            continue
        res = []
        for t in (x, x + 1):
            g = oracle.OracleGraph(3, [1, 2], [0, 1], weights=np.array([SENT, t], np.uint32),
                                   model=oracle.W_TAU)
            o = g.sample_ids(seed, np.array([j], np.uint64))
            res.append((int(o["src"][0]), set(o["members"].tolist())))
        if res[0][0] != 0 or res[1][0] != 0:
            continue
        assert res[0][1] == {0, 1} and res[1][1] == {0, 1, 2}
        checked += 1
    assert checked >= 20


@pytest.mark.parametrize("kind", ["mixed", "wc", "tri"])
def test_bucket_first_step_has_the_iis_law(kind):
    """The bucket form of the first step (Eq. probn) draws from the same law
    as rejection (Lemma 2), without retries."""
    n, src, dst, p, model = _tiny_graph(kind)
    g = oracle.OracleGraph(n, src, dst, weights=p, model=model, weight_seed=3)
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    dst_csr = np.repeat(np.arange(n), np.diff(a["off"])).tolist()
    law = iis_law(n, a["src"].tolist(), dst_csr, probs, a["w"].tolist(), g.W)
    T = 300_000
    out = g.sample_ids(0x4321 + len(kind), np.arange(T, dtype=np.uint64), bucket=True)
    assert (out["retries"] == 0).all() and (out["status"] == 0).all()
    deg = np.diff(a["off"])
    mo, mem = out["member_off"], out["members"]
    cnt = Counter()
    for t in range(T):
        cnt[(int(out["src"][t]), frozenset(mem[mo[t]:mo[t + 1]].tolist()))] += 1
    assert all(len(R) >= 2 for (_, R) in cnt) and set(cnt) <= set(law)
    for t in range(0, T, 1009):
        assert out["coins"][t] == deg[mem[mo[t]:mo[t + 1]]].sum()
    exp = {k: float(v) * T for k, v in law.items()}
    big = [k for k in exp if exp[k] >= 20]
    small = [k for k in exp if exp[k] < 20]
    obs = [cnt.get(k, 0) for k in big] + [sum(cnt.get(k, 0) for k in small)]
    ex = [exp[k] for k in big] + [sum(exp[k] for k in small)]
    if ex[-1] == 0:
        obs, ex = obs[:-1], ex[:-1]
    obs, ex = np.array(obs, float), np.array(ex, float)
    chi2 = ((obs - ex) ** 2 / ex).sum()
    dof = len(ex) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof)


def test_bucket_first_step_on_a_single_in_edge_row():
    # a source with one in-edge: the bucket is that edge, whatever its weight
    g = oracle.OracleGraph(3, [1, 2], [0, 1], weights=np.array([0.001, 0.5]), model=oracle.W_P)
    out = g.sample_ids(5, np.arange(2000, dtype=np.uint64), bucket=True)
    mo, mem = out["member_off"], out["members"]
    for t in range(2000):
        R = mem[mo[t]:mo[t + 1]].tolist()
        assert R[:2] == [out["src"][t], out["src"][t] + 1]
