"""Pins of the oracle's Linear Threshold variant (Sec. "Extensions to other
diffusion models", LT): the law of its importance samples and of its plain
RIS samples against exact enumeration of LT live-edge worlds (every vertex
keeps at most one in-edge), the estimator's unbiasedness against the exact
LT influence, closed forms, and the model's row constraint."""
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import lt_influence, lt_iis_law, lt_rr_law, p_eff


def _lt_graph(kind):
    if kind == "mixed":
        # rows: 0 <- {1, 2, 4} (sum 0.9), 1 <- {3} (p = 1: sentinel), 2 <- {0, 4},
        # 3 <- {2, 1, 1} (a parallel pair), 4 <- {3} (sum 0.35)
        src = [1, 2, 3, 0, 4, 2, 4, 1, 1, 3]
        dst = [0, 0, 1, 2, 2, 3, 0, 3, 3, 4]
        p = np.array([0.5, 0.3, 1.0, 0.2, 0.6, 0.45, 0.1, 0.25, 0.15, 0.35])
        return 5, src, dst, p, oracle.W_P
    if kind == "wc":
        src = [1, 2, 3, 0, 4, 2, 3, 4, 0, 1, 4]
        dst = [0, 0, 1, 2, 2, 3, 4, 1, 4, 3, 3]
        return 5, src, dst, None, oracle.W_WC
    raise KeyError(kind)


def _exact_inputs(g, n):
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    dst_csr = np.repeat(np.arange(n), np.diff(a["off"])).tolist()
    return a, a["src"].tolist(), dst_csr, probs


def _chi2_ok(cnt, law, T):
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
    return chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof)


def _collect(g, seed, T, ris=False):
    out = g.sample_ids(seed, np.arange(T, dtype=np.uint64), ris=ris)
    mo, mem = out["member_off"], out["members"]
    cnt = Counter()
    for t in range(T):
        cnt[(int(out["src"][t]), frozenset(mem[mo[t]:mo[t + 1]].tolist()))] += 1
    return out, cnt


@pytest.mark.parametrize("kind", ["mixed", "wc"])
def test_lt_gamma_is_the_row_weight_sum(kind):
    n, src, dst, p, model = _lt_graph(kind)
    g = oracle.OracleGraph(n, src, dst, weights=p, model=model, lt=True)
    a, s_csr, d_csr, probs = _exact_inputs(g, n)
    assert g.f == 32
    for v in range(n):
        gam = sum((probs[e] for e in range(len(d_csr)) if d_csr[e] == v), Fraction(0))
        assert Fraction(int(a["w"][v]), 1 << 32) == gam
    assert g.W == int(a["w"].sum())


@pytest.mark.parametrize("kind", ["mixed", "wc"])
def test_lt_iis_law_matches_exact_enumeration(kind):
    n, src, dst, p, model = _lt_graph(kind)
    g = oracle.OracleGraph(n, src, dst, weights=p, model=model, lt=True)
    a, s_csr, d_csr, probs = _exact_inputs(g, n)
    law = lt_iis_law(n, s_csr, d_csr, probs, a["w"].tolist(), g.W)
    assert abs(float(sum(law.values())) - 1.0) < 1e-12
    T = 300_000
    out, cnt = _collect(g, 0x17 + len(kind), T)
    assert (out["retries"] == 0).all()
    assert all(len(R) >= 2 for (_, R) in cnt) and set(cnt) <= set(law)
    ok, info = _chi2_ok(cnt, law, T)
    assert ok, info
    # work counter: every member's in-row once
    deg = np.diff(a["off"])
    mo, mem = out["member_off"], out["members"]
    for t in range(0, T, 997):
        assert out["coins"][t] == deg[mem[mo[t]:mo[t + 1]]].sum()


def test_lt_ris_law_matches_exact_enumeration():
    n, src, dst, p, model = _lt_graph("mixed")
    g = oracle.OracleGraph(n, src, dst, weights=p, model=model, lt=True)
    a, s_csr, d_csr, probs = _exact_inputs(g, n)
    rr = lt_rr_law(n, s_csr, d_csr, probs)
    law = {(v, R): pr / n for v in range(n) for R, pr in rr[v].items()}
    T = 200_000
    out, cnt = _collect(g, 0x99, T, ris=True)
    assert any(len(R) == 1 for (_, R) in cnt)  # singular samples occur
    ok, info = _chi2_ok(cnt, law, T)
    assert ok, info


@pytest.mark.parametrize("S", [[0], [3], [1, 4], [0, 2, 3]])
def test_lt_estimator_is_unbiased(S):
    n, src, dst, p, model = _lt_graph("mixed")
    g = oracle.OracleGraph(n, src, dst, weights=p, model=model, lt=True)
    a, s_csr, d_csr, probs = _exact_inputs(g, n)
    I = lt_influence(n, s_csr, d_csr, probs, S)
    law = lt_iis_law(n, s_csr, d_csr, probs, a["w"].tolist(), g.W)
    hit = float(sum(pr for (v, R), pr in law.items() if R & set(S)))
    Gamma = g.W / 2**32
    T = 200_000
    sk = oracle.OracleSketch(g, 0x5A + len(S), T)
    cov, est = sk.coverage(np.array([0, len(S)]), np.array(S, np.int32))
    sigma = Gamma * np.sqrt(hit * (1 - hit) / T)
    assert abs(est[0] - float(I)) < 5 * sigma + 1e-12, (est[0], float(I), sigma)


def test_lt_wc_path_is_exact():
    # directed path 0 -> 1 -> ... -> L under WC: every in-row is one
    # always-kept edge, so each sample is {0, ..., src} and I({0}) = L + 1
    L = 9
    src, dst = list(range(L)), list(range(1, L + 1))
    g = oracle.OracleGraph(L + 1, src, dst, model=oracle.W_WC, lt=True)
    sk = oracle.OracleSketch(g, 3, 5000)
    a = sk.arrays()
    for t in range(5000):
        R = sorted(a["mem"][a["off"][t]:a["off"][t + 1]].tolist())
        assert R == list(range(a["src"][t] + 1))
    cov, est = sk.coverage(np.array([0, 1]), np.array([0], np.int32))
    assert cov[0] == 5000 and est[0] == L + 1


def test_lt_rejects_rows_above_one():
    with pytest.raises(oracle.OracleError):
        oracle.OracleGraph(3, [1, 2], [0, 0], weights=np.array([0.6, 0.5]), model=oracle.W_P, lt=True)
    # the same weights are a valid IC instance
    oracle.OracleGraph(3, [1, 2], [0, 0], weights=np.array([0.6, 0.5]), model=oracle.W_P)
