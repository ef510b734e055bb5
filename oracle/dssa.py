"""DSSA-style doubling influence maximisation over SKIS sketches, oracle side
(TEST INFRASTRUCTURE ONLY; plain Python over the oracle's sketch, greedy and
coverage). Follows the paper's appendix "Improvements of SSA/DSSA using SKIS
sketch": two independent sketches R and R^c double each round t; greedy
(Alg. 3) on R gives S_k, re-estimated on R^c; stop when Cov_R(S_k) >=
Lambda_2 and (e1 + e2 + e1 e2)(1 - 1/e - eps) + (1 - 1/e) e3 <= eps with
  e1 = I_R / I_Rc - 1,
  e2 = eps sqrt(n (1 + eps) / (2^(t-1) I_Rc)),
  e3 = eps sqrt(n (1 + eps)(1 - 1/e - eps) / ((1 + eps/3) 2^(t-1) I_Rc)),
or at n_max samples. Lambda_2 is given in the paper only up to a constant; the
reading used (lambda2 = 0) is Lemma 7's (2 Gamma/n + 2 eps/3) ln(2 t_max /
delta) / eps^2. Estimates are formed from exact integers with correctly
rounded conversions."""
from __future__ import annotations

import math

import numpy as np

from .oracle import OracleGraph, OracleSketch

INV_E = 0.36787944117144233  # e^-1 rounded to binary64


def dssa_maxinf(graph: OracleGraph, seed_r: int, seed_rc: int, k: int, eps: float, delta: float,
                lambda2: int = 0, n0: int = 1 << 12, n_max: int = 1 << 24):
    n = graph.n
    W, f = graph.W, graph.f
    gamma_n = (float(W) / float(1 << f)) / float(n)
    t_max = 1
    N = n0
    while N < n_max:
        N *= 2
        t_max += 1
    if lambda2 == 0:
        lambda2 = math.ceil((2.0 * gamma_n + 2.0 * eps / 3.0) * math.log(2.0 * float(t_max) / delta) / (eps * eps))
    w = graph.arrays()["w"]
    N, t = n0, 1
    while True:
        R = OracleSketch(graph, seed_r, N)
        Rc = OracleSketch(graph, seed_rc, N)
        seeds, cov, _ = R.greedy(k)
        sum_c = sum((1 << f) - int(w[v]) for v in seeds)
        cov_r = int(cov[-1])
        cov_c = int(Rc.coverage(np.array([0, k], np.int64), seeds)[0][0])
        D = float(N << f)
        i_r = float(cov_r * W + N * sum_c) / D
        i_c = float(cov_c * W + N * sum_c) / D
        scale = math.ldexp(1.0, t - 1)
        e1 = i_r / i_c - 1.0
        e2 = eps * math.sqrt(n * (1.0 + eps) / (scale * i_c))
        e3 = eps * math.sqrt(n * (1.0 + eps) * (1.0 - INV_E - eps) / ((1.0 + eps / 3.0) * scale * i_c))
        res = dict(rounds=t, samples=N, lambda2=lambda2, coverage=cov_r, coverage_c=cov_c, estimate=i_r,
                   estimate_c=i_c, eps1=e1, eps2=e2, eps3=e3, stopped_by=0)
        if cov_r >= lambda2:
            lhs = (e1 + e2 + e1 * e2) * (1.0 - INV_E - eps) + (1.0 - INV_E) * e3
            if lhs <= eps:
                res["stopped_by"] = 1
                return seeds, res
        if N >= n_max:
            res["stopped_by"] = 2
            return seeds, res
        N = min(N * 2, n_max)
        t += 1
