"""Pins of the oracle's coverage counts and SKIS estimator (Eq. 21) against
exact influence from world enumeration (Eq. 2, Lemma 3), the variance of
Lemma 4, closed forms on stars and paths, brute-force coverage, and forward
Monte-Carlo cascades (Sec. VI, ground truth)."""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import oracle
import synth
from exact import gamma, influence, p_eff, rr_law


def _csr_dst(a):
    return np.repeat(np.arange(len(a["off"]) - 1), np.diff(a["off"])).tolist()


def _queries(sets):
    off = np.concatenate([[0], np.cumsum([len(s) for s in sets])]).astype(np.int64)
    seeds = np.array([v for s in sets for v in s], np.int32)
    return off, seeds


def _graph_mixed():
    src = [1, 2, 3, 0, 4, 2, 3, 3, 4, 1, 0]
    dst = [0, 0, 1, 2, 2, 3, 4, 4, 0, 3, 4]
    p = np.array([0.5, 0.3, 0.7, 0.2, 1.0, 0.45, 0.6, 0.25, 0.15, 0.35, 0.05])
    return 5, src, dst, p


def test_lemma3_identity_by_enumeration():
    """I(S) = Pr[R ∩ S != {}] * Gamma + sum_{v in S} (1 - gamma_v), exactly."""
    n, src, dst, p = _graph_mixed()
    g = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    sc, dc = a["src"].tolist(), _csr_dst(a)
    gam = gamma(n, dc, probs)
    Gam = sum(gam)
    law = rr_law(n, sc, dc, probs)
    for k in (1, 2):
        for S in combinations(range(n), k):
            hit = Fraction(0)
            for v in range(n):
                for R, pr in law[v].items():
                    if R != frozenset([v]) and R & set(S):
                        hit += pr  # Pr[g non-singular at v and R meets S] = gamma_v Pr[hit | v]
            # Pr[R ∩ S != {}] for an IIS sample = sum_v (gamma_v / Gamma) * (hit_v / gamma_v)
            lhs = influence(n, sc, dc, probs, S)
            rhs = hit + sum(1 - gam[v] for v in S)
            assert lhs == rhs, S


def test_estimator_is_unbiased_within_lemma4_variance():
    n, src, dst, p = _graph_mixed()
    g = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    sc, dc = a["src"].tolist(), _csr_dst(a)
    gam = gamma(n, dc, probs)
    Gam = sum(gam)
    T = 400_000
    sk = oracle.OracleSketch(g, 777, T)
    sets = [list(S) for k in (1, 2, 3) for S in combinations(range(n), k)]
    off, seeds = _queries(sets)
    cov, est = sk.coverage(off, seeds)
    for b, S in enumerate(sets):
        I = influence(n, sc, dc, probs, S)
        A = sum(1 - gam[v] for v in S)
        x = (I - A) / Gam  # E[X_j(S)], Eq. xvar
        # Lemma 4: Var[Z_j] = (Gamma/n)^2 Var[X_j]; Var[I_R] = n^2 Var[Z_j] / T
        var_est = float(Gam) ** 2 * float(x * (1 - x)) / T
        fixed_point_slack = n * 2.0 ** -g.f * 4
        assert abs(est[b] - float(I)) <= 5 * np.sqrt(var_est) + fixed_point_slack, (S, est[b], float(I))
        # Lemma 5 bound on the variance holds
        assert float(Gam) ** 2 * float(x * (1 - x)) <= float(I) * float(Gam) + 1e-12


def test_in_star_centre_has_influence_one_exactly():
    # leaves -> centre: every sample has source c and contains c, so
    # I_R({c}) = Gamma + (1 - gamma_c) = 1 with zero variance
    d = 7
    for p in (0.3, 0.01):
        g = oracle.OracleGraph(d + 1, list(range(1, d + 1)), [0] * d, weights=np.full(d, p),
                               model=oracle.W_P)
        sk = oracle.OracleSketch(g, 5, 5000)
        assert (sk.arrays()["src"] == 0).all()
        cov, est, N, D = sk.coverage(*_queries([[0]]), exact=True)
        assert cov[0] == 5000 and N[0] == D[0] and est[0] == 1.0
        # a leaf: I({leaf}) = 1 + p'
        pe = float(p_eff(g.arrays()["tau"][0]))
        T = 200_000
        sk = oracle.OracleSketch(g, 6, T)
        cov, est = sk.coverage(*_queries([[1]]))
        G = float(g.W) / 2**g.f
        x = pe / G
        assert abs(est[0] - (1 + pe)) <= 5 * G * np.sqrt(x * (1 - x) / T) + 1e-9


def test_out_star_centre_closed_form():
    # centre -> leaves, each with p: I({c}) = 1 + d p'. Every sample is
    # {leaf, c}, so Cov({c}) = T and the estimate is exact up to fixed point.
    d, p = 6, 0.2
    g = oracle.OracleGraph(d + 1, [0] * d, list(range(1, d + 1)), weights=np.full(d, p),
                           model=oracle.W_P)
    pe = p_eff(g.arrays()["tau"][0])
    sk = oracle.OracleSketch(g, 8, 3000)
    cov, est = sk.coverage(*_queries([[0]]))
    assert cov[0] == 3000
    assert abs(Fraction(est[0]) - (1 + d * pe)) <= d * Fraction(1, 2**g.f) + Fraction(1, 2**50)


@pytest.mark.parametrize("L,p", [(6, 0.5), (4, 0.9)])
def test_path_closed_form(L, p):
    # v0 -> v1 -> ... -> v_{L-1}: I({v0}) = sum_{i<L} p'^i
    g = oracle.OracleGraph(L, list(range(L - 1)), list(range(1, L)), weights=np.full(L - 1, p),
                           model=oracle.W_P)
    pe = float(p_eff(g.arrays()["tau"][0]))
    T = 300_000
    sk = oracle.OracleSketch(g, 9, T)
    cov, est = sk.coverage(*_queries([[0]]))
    want = sum(pe**i for i in range(L))
    G = float(g.W) / 2**g.f
    x = (want - 1 + 0.0) / G  # S = {v0} has gamma 0, so A = 1
    assert abs(est[0] - want) <= 5 * G * np.sqrt(x * (1 - x) / T) + 1e-9


def test_coverage_matches_brute_force_set_intersection():
    n, m = 300, 1500
    src, dst = synth.er(n, m, 21)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    sk = oracle.OracleSketch(g, 3, 2000)
    a = sk.arrays()
    samples = [set(a["mem"][a["off"][j]:a["off"][j + 1]].tolist()) for j in range(2000)]
    off, seeds = synth.seed_sets(n, [1, 2, 5, 17, 60, 300], 4)
    cov, est, N, D = sk.coverage(off, seeds, exact=True)
    w = g.arrays()["w"]
    for b in range(len(off) - 1):
        S = set(seeds[off[b]:off[b + 1]].tolist())
        want = sum(1 for R in samples if R & S)
        assert cov[b] == want
        # Eq. 21 in units of 2^-f: the ratio N / D is Cov/T*Gamma~ + sum(1-gamma~)
        assert Fraction(N[b], D[b]) == Fraction(want, 2000) * Fraction(g.W, 2**g.f) + sum(
            1 - Fraction(int(w[v]), 2**g.f) for v in S)
        assert est[b] == float(Fraction(N[b], D[b])) or abs(est[b] / float(Fraction(N[b], D[b])) - 1) < 1e-15
    assert cov[-1] == 2000  # S = V meets every sample


def test_bad_queries_are_rejected():
    g = oracle.OracleGraph(4, [1, 2, 3], [0, 0, 0], model=oracle.W_WC)
    sk = oracle.OracleSketch(g, 1, 10)
    for sets in ([[]], [[1, 1]], [[4]], [[-1]]):
        off = np.concatenate([[0], np.cumsum([len(s) for s in sets])]).astype(np.int64)
        seeds = np.array([v for s in sets for v in s], np.int32)
        with pytest.raises(oracle.OracleError):
            sk.coverage(off, seeds)


def _forward_ic(n, src, dst, p, S, runs, rng):
    """Mean cascade size of forward IC simulations (Sec. II-A), numpy RNG."""
    order = np.argsort(src, kind="stable")
    s_sorted, d_sorted, p_sorted = src[order], dst[order], p[order]
    off = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=n))])
    sizes = np.empty(runs)
    for r in range(runs):
        active = np.zeros(n, bool)
        active[list(S)] = True
        frontier = list(S)
        while frontier:
            nxt = []
            for u in frontier:
                lo, hi = off[u], off[u + 1]
                live = rng.random(hi - lo) < p_sorted[lo:hi]
                for v in d_sorted[lo:hi][live]:
                    if not active[v]:
                        active[v] = True
                        nxt.append(v)
            frontier = nxt
        sizes[r] = active.sum()
    return sizes.mean(), sizes.std() / np.sqrt(runs)


def test_estimate_agrees_with_forward_monte_carlo():
    n, m = 200, 900
    src, dst = synth.er(n, m, 31)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    a = g.arrays()
    # effective per-input-edge probabilities (WC thresholds)
    pe = np.empty(m)
    pe[a["perm"]] = [float(p_eff(t)) for t in a["tau"]]
    T = 200_000
    sk = oracle.OracleSketch(g, 17, T)
    rng = np.random.default_rng(123)
    for S in ([0], [5, 9, 77], list(range(0, 200, 20))):
        cov, est = sk.coverage(*_queries([S]))
        mc, mc_se = _forward_ic(n, src, dst, pe, S, 3000, rng)
        G = float(g.W) / 2**g.f
        x = cov[0] / T
        se = np.sqrt(mc_se**2 + G**2 * x * (1 - x) / T)
        assert abs(est[0] - mc) <= 5 * se, (S, est[0], mc, se)
