"""Pins of the oracle's greedy max-coverage (Alg. 3) against brute force on
tiny sketches (the (1 - (1 - 1/k)^k) guarantee of Lemma 9 and the exact
optimum for k = 1), monotonicity and submodularity (Lemma 8), and agreement
with the oracle's own estimator on every prefix."""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import oracle
import synth


def _queries(sets):
    off = np.concatenate([[0], np.cumsum([len(s) for s in sets])]).astype(np.int64)
    seeds = np.array([v for s in sets for v in s], np.int32)
    return off, seeds


def _exact_est(sketch_sets, w, W, f, T, S):
    cov = sum(1 for R in sketch_sets if R & S)
    return Fraction(cov, T) * Fraction(W, 2**f) + sum(1 - Fraction(int(w[v]), 2**f) for v in S)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_greedy_guarantee_and_k1_optimum_by_brute_force(seed):
    n, m = 11, 30
    src, dst = synth.er(n, m, seed)
    g = oracle.OracleGraph(n, src, dst, weights=synth.uniform_p(m, seed, 0.05, 0.6), model=oracle.W_P)
    T = 60
    sk = oracle.OracleSketch(g, seed, T)
    a = sk.arrays()
    sets = [set(a["mem"][a["off"][j]:a["off"][j + 1]].tolist()) for j in range(T)]
    w = g.arrays()["w"]
    for k in (1, 2, 3, 4):
        seeds, cov, est = sk.greedy(k)
        assert len(set(seeds.tolist())) == k
        got = _exact_est(sets, w, g.W, g.f, T, set(seeds.tolist()))
        opt = max(_exact_est(sets, w, g.W, g.f, T, set(S)) for S in combinations(range(n), k))
        assert got >= (1 - Fraction(k - 1, k) ** k) * opt
        if k == 1:
            assert got == opt
            # ties are broken towards the lowest vertex id
            best = [v for v in range(n) if _exact_est(sets, w, g.W, g.f, T, {v}) == opt]
            assert seeds[0] == min(best)
        assert abs(est[-1] - float(got)) <= 1e-15 * float(got)


def test_greedy_prefixes_agree_with_estimator_and_are_monotone():
    n, m = 2000, 16000
    src, dst = synth.chunglu(n, m, 2.1, 7)
    g = oracle.OracleGraph(n, src, dst, weights=synth.tri(m, 7), model=oracle.W_P)
    T = 20_000
    sk = oracle.OracleSketch(g, 11, T)
    k = 40
    seeds, cov, est = sk.greedy(k)
    prefixes = [seeds[: i + 1].tolist() for i in range(k)]
    c2, e2 = sk.coverage(*_queries(prefixes))
    assert np.array_equal(cov, c2)
    assert np.array_equal(est, e2)
    assert (np.diff(cov) >= 0).all() and (np.diff(est) > 0).all()
    # diminishing returns along the greedy order (submodularity, Lemma 8)
    gains = np.diff(np.concatenate([[0.0], est]))
    assert (np.diff(gains) <= 1e-12).all()


def test_submodularity_on_random_sets():
    n, m = 500, 3000
    src, dst = synth.er(n, m, 8)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    sk = oracle.OracleSketch(g, 4, 5000)
    rng = np.random.default_rng(2)
    for _ in range(30):
        B = rng.choice(n, size=12, replace=False)
        A = B[:5]
        v = int(rng.choice(np.setdiff1d(np.arange(n), B)))
        sets = [A.tolist(), A.tolist() + [v], B.tolist(), B.tolist() + [v]]
        _, est = sk.coverage(*_queries(sets))
        gA, gB = est[1] - est[0], est[3] - est[2]
        assert gA >= gB - 1e-12 and gB >= -1e-12 and est[2] >= est[0] - 1e-12


def test_greedy_edge_cases():
    # k = n selects every vertex and covers every sample; k > n is rejected
    n, m = 9, 20
    src, dst = synth.er(n, m, 5)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    sk = oracle.OracleSketch(g, 1, 100)
    seeds, cov, est = sk.greedy(n)
    assert sorted(seeds.tolist()) == list(range(n)) and cov[-1] == 100
    with pytest.raises(oracle.OracleError):
        sk.greedy(n + 1)
    # vertices that appear in no sample still carry gain 1 - gamma_v (Alg. 3's
    # marginal gain). Edge 1 -> 0 plus isolated vertices 2, 3, 4: every sample is
    # {0, 1}; greedy takes 1 (I = 1 + p'), then the isolated vertices (gain 1
    # each, lowest id first) ahead of 0 (gain 1 - gamma_0).
    g = oracle.OracleGraph(5, [1], [0], weights=np.array([0.25]), model=oracle.W_P)
    T = 1000
    sk = oracle.OracleSketch(g, 2, T)
    seeds, cov, est = sk.greedy(4)
    assert seeds.tolist() == [1, 2, 3, 4] and cov.tolist() == [T] * 4
    G = g.W / 2**g.f
    assert np.allclose(est, [1 + G, 2 + G, 3 + G, 4 + G], rtol=1e-15)
    seeds, cov, est = sk.greedy(5)
    assert seeds.tolist()[-1] == 0 and abs(est[-1] - (4 + 1.0)) < 1e-12
