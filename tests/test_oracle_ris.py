"""Pins of the oracle's plain-RIS variant (Borgs et al.; Sec. II-C): the law
of a RIS sample from world enumeration (singular samples included), Lemma 1
unbiasedness, the variance comparison with SKIS samples (Lemmas 4-5 against
the Bernoulli variance of RIS), and coverage-only greedy."""
from collections import Counter
from fractions import Fraction
from itertools import combinations

import numpy as np

import oracle
import synth
from exact import gamma, influence, p_eff, rr_law


def _tiny():
    src = [1, 2, 3, 0, 4, 2, 3, 3, 4, 1]
    dst = [0, 0, 1, 2, 2, 3, 4, 4, 0, 3]
    p = np.array([0.5, 0.3, 0.7, 0.2, 1.0, 0.45, 0.6, 0.25, 0.15, 0.35])
    n = 6  # vertex 5 has no edges: every RIS sample from it is {5}
    return n, src, dst, p


def _csr(g):
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    dst_csr = np.repeat(np.arange(g.n), np.diff(a["off"])).tolist()
    return a, probs, a["src"].tolist(), dst_csr


def test_ris_law_matches_exact_enumeration():
    n, src, dst, p = _tiny()
    g = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    a, probs, sc, dc = _csr(g)
    law = rr_law(n, sc, dc, probs)
    exp = {(v, R): Fraction(1, n) * pr for v in range(n) for R, pr in law[v].items()}
    T = 300_000
    out = g.sample_ids(9, np.arange(T, dtype=np.uint64), ris=True)
    assert (out["retries"] == 0).all() and (out["status"] == 0).all()
    mo, mem = out["member_off"], out["members"]
    cnt = Counter((int(out["src"][t]), frozenset(mem[mo[t]:mo[t + 1]].tolist())) for t in range(T))
    assert set(cnt) <= set(exp)
    assert any(len(R) == 1 for (_, R) in cnt)  # singular samples occur
    keys = [k for k in exp if float(exp[k]) * T >= 20]
    rest = [k for k in exp if float(exp[k]) * T < 20]
    obs = np.array([cnt.get(k, 0) for k in keys] + [sum(cnt.get(k, 0) for k in rest)], float)
    ex = np.array([float(exp[k]) * T for k in keys] + [sum(float(exp[k]) * T for k in rest)])
    if ex[-1] == 0:
        obs, ex = obs[:-1], ex[:-1]
    chi2 = ((obs - ex) ** 2 / ex).sum()
    dof = len(ex) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof)


def test_lemma1_and_ris_estimate_unbiased():
    n, src, dst, p = _tiny()
    g = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    a, probs, sc, dc = _csr(g)
    law = rr_law(n, sc, dc, probs)
    T = 300_000
    sk = oracle.OracleSketch(g, 3, T, ris=True)
    sets = [list(S) for k in (1, 2) for S in combinations(range(n), k)]
    off = np.concatenate([[0], np.cumsum([len(S) for S in sets])]).astype(np.int64)
    cov, est = sk.coverage(off, np.array([v for S in sets for v in S], np.int32))
    for b, S in enumerate(sets):
        hit = sum(pr for v in range(n) for R, pr in law[v].items() if R & set(S)) / n
        I = influence(n, sc, dc, probs, S)
        assert n * hit == I  # Lemma 1, exactly
        x = float(hit)
        assert abs(est[b] - float(I)) <= 5 * n * np.sqrt(x * (1 - x) / T) + 1e-12
        assert est[b] == cov[b] * n / T


def test_skis_variance_is_below_ris_variance():
    # Lemma 4 (exact Var[Z]) against the Bernoulli variance of the RIS
    # variable Y, and Lemma 5's bound, for every S with |S| <= 2
    n, src, dst, p = _tiny()
    g = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    a, probs, sc, dc = _csr(g)
    gam = gamma(n, dc, probs)
    G = sum(gam)
    for k in (1, 2):
        for S in combinations(range(n), k):
            I = influence(n, sc, dc, probs, S)
            A = sum(1 - gam[v] for v in S)
            var_y = I / n * (1 - I / n)
            var_z = I / n * G / n - I * I / (n * n) - A / (n * n) * (G + A - 2 * I)
            x = (I - A) / G
            assert var_z == (G / n) ** 2 * x * (1 - x)  # Lemma 4 equals the Bernoulli form
            assert var_z <= I / n * G / n                # Lemma 5
            assert var_z <= var_y                        # SKIS never worse here


def test_ris_greedy_maximises_coverage():
    n, m = 12, 40
    src, dst = synth.er(n, m, 3)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    T = 500
    sk = oracle.OracleSketch(g, 4, T, ris=True)
    arr = sk.arrays()
    sets = [set(arr["mem"][arr["off"][j]:arr["off"][j + 1]].tolist()) for j in range(T)]
    seeds, cov, est = sk.greedy(2)
    counts = [sum(1 for R in sets if v in R) for v in range(n)]
    best = max(counts)
    assert seeds[0] == min(v for v in range(n) if counts[v] == best) and cov[0] == best
    assert est[1] == cov[1] * n / T


def test_skis_estimates_beat_ris_on_singletons():
    # the paper's headline (Sec. VI, Fig. 3): for single seeds, SKIS errors are
    # far smaller than RIS errors at the same number of samples
    n, m = 2000, 16000
    src, dst = synth.chunglu(n, m, 2.1, 8)
    p = synth.tri(m, 8)
    g = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    truth = oracle.OracleSketch(g, 99, 400_000)
    T = 20_000
    seeds = np.arange(0, n, 20, dtype=np.int32)
    off = np.arange(len(seeds) + 1, dtype=np.int64)
    _, ref = truth.coverage(off, seeds)
    err_skis, err_ris = [], []
    for rep in range(5):
        _, e1 = oracle.OracleSketch(g, 1000 + rep, T).coverage(off, seeds)
        _, e2 = oracle.OracleSketch(g, 2000 + rep, T, ris=True).coverage(off, seeds)
        err_skis.append(np.mean(np.abs(e1 - ref) / ref))
        err_ris.append(np.mean(np.abs(e2 - ref) / ref))
    assert np.mean(err_skis) * 3 < np.mean(err_ris)
