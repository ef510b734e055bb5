"""Pins of the oracle's DSSA-style doubling driver: the approximation
guarantee against the exact optimum by world enumeration on a tiny graph, the
sample cap, and agreement of its answer with greedy on the final sketch."""
from itertools import combinations

import numpy as np

import oracle
import synth
from exact import influence, p_eff
from oracle.dssa import INV_E, dssa_maxinf


def test_inv_e_constant():
    import math

    assert INV_E == math.exp(-1.0) or abs(INV_E - math.exp(-1.0)) <= 2 ** -53


def test_dssa_meets_the_guarantee_by_enumeration():
    # I(S_k) >= (1 - 1/e - eps) OPT_k with exact I from every live-edge world
    src = [0, 0, 1, 2, 3, 4, 5, 6, 1, 7]
    dst = [1, 2, 3, 3, 4, 5, 6, 7, 5, 0]
    p = np.array([0.6, 0.4, 0.5, 0.3, 0.7, 0.5, 0.4, 0.6, 0.2, 0.3])
    n, k, eps = 8, 2, 0.3
    g = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    dst_csr = np.repeat(np.arange(n), np.diff(a["off"])).tolist()
    sc = a["src"].tolist()
    infl = {S: influence(n, sc, dst_csr, probs, S) for S in combinations(range(n), k)}
    opt = max(infl.values())
    for seed in range(4):
        seeds, res = dssa_maxinf(g, 100 + seed, 200 + seed, k, eps, 0.1, n0=256, n_max=1 << 16)
        S = tuple(sorted(int(v) for v in seeds))
        assert float(infl[S]) >= (1 - INV_E - eps) * float(opt)
        assert res["stopped_by"] in (1, 2) and res["samples"] <= 1 << 16


def test_dssa_cap_and_final_greedy():
    n, m = 500, 4000
    src, dst = synth.er(n, m, 6)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    # an unreachable coverage threshold runs to the sample cap
    seeds, res = dssa_maxinf(g, 1, 2, 5, 0.2, 0.01, lambda2=1 << 40, n0=512, n_max=4096)
    assert res["stopped_by"] == 2 and res["samples"] == 4096 and res["rounds"] == 4
    # the answer is greedy on R at its final size
    gs, gc, ge = oracle.OracleSketch(g, 1, 4096).greedy(5)
    assert np.array_equal(seeds, gs) and res["coverage"] == gc[-1] and res["estimate"] == ge[-1]
