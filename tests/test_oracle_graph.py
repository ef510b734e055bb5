"""Pins of the oracle's Philox generator, thresholds, canonical in-CSR,
fixed-point gamma and alias table against values fixed outside the oracle:
published known-answer vectors, exact rational arithmetic, library sorts and
exact mass invariants."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from exact import SENT, gamma, p_eff, tau_from_p

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert oracle.philox4x32_10(ctr, key).tolist() == want


def _graph(n, src, dst, **kw):
    return oracle.OracleGraph(n, np.asarray(src), np.asarray(dst), **kw)


def test_csr_is_canonical_against_lexsort():
    n, m = 50, 400
    rng = np.random.default_rng(5)
    src = rng.integers(0, n, m)
    dst = (src + rng.integers(1, n, m)) % n  # no self-loops; parallel edges likely
    p = rng.uniform(0, 1, m)
    g = _graph(n, src, dst, weights=p, model=oracle.W_P)
    a = g.arrays()
    order = np.lexsort((np.arange(m), src, dst))  # by dst, then src, then input index
    assert np.array_equal(a["perm"], order)
    assert np.array_equal(a["src"], src[order])
    assert np.array_equal(a["off"], np.concatenate([[0], np.cumsum(np.bincount(dst, minlength=n))]))
    assert np.array_equal(a["tau"], np.array([tau_from_p(x) for x in p[order]], np.uint32))
    # the same graph in another input order gives the same offsets and, per
    # row, the same (source, threshold) multiset; parallel edges with
    # different p keep their input order, so only the multiset is invariant
    sh = rng.permutation(m)
    b = _graph(n, src[sh], dst[sh], weights=p[sh], model=oracle.W_P).arrays()
    assert np.array_equal(a["off"], b["off"])
    for v in range(n):
        lo, hi = a["off"][v], a["off"][v + 1]
        assert sorted(zip(a["src"][lo:hi], a["tau"][lo:hi])) == sorted(zip(b["src"][lo:hi], b["tau"][lo:hi]))


def test_thresholds_exact():
    # explicit p: floor(p * 2^32) from the exact binary value of the double
    ps = [0.0, 1e-12, 0.001, 0.01, 0.1, 0.25, 0.5, 0.999999, 1 - 2.0**-33, 1 - 2.0**-32, 1.0]
    n = len(ps) + 1
    src = list(range(1, n))
    dst = [0] * (n - 1)
    a = _graph(n, src, dst, weights=np.array(ps), model=oracle.W_P).arrays()
    want = [tau_from_p(p) for p in ps]
    assert a["tau"].tolist() == want
    assert want[-1] == SENT and want[-2] == SENT and want[0] == 0
    # WC: floor(2^32 / d_in) in integers, sentinel at d_in = 1
    for d in (1, 2, 3, 7, 1000, 65537):
        a = _graph(d + 1, list(range(1, d + 1)), [0] * d, model=oracle.W_WC).arrays()
        t = (1 << 32) // d if d > 1 else SENT
        assert set(a["tau"].tolist()) == {t}
    with pytest.raises(oracle.OracleError):
        _graph(3, [1, 2], [0, 0], model=oracle.W_P, weights=np.array([0.5, np.nan]))
    with pytest.raises(oracle.OracleError):
        _graph(3, [1, 2], [0, 0], model=oracle.W_P, weights=np.array([0.5, 1.5]))
    with pytest.raises(oracle.OracleError):
        _graph(3, [1, 2], [0, 2], model=oracle.W_WC)  # self-loop
    with pytest.raises(oracle.OracleError):
        _graph(3, [1, 3], [0, 0], model=oracle.W_WC)  # id out of range


def test_tri_thresholds_levels_and_balance():
    n, m = 2000, 30000
    src, dst = synth.er(n, m, 9)
    a = oracle.OracleGraph(n, src, dst, model=oracle.W_TRI, weight_seed=77).arrays()
    levels = [tau_from_p(p) for p in (0.1, 0.01, 0.001)]
    vals, cnt = np.unique(a["tau"], return_counts=True)
    assert sorted(vals.tolist()) == sorted(levels)
    # uniform over the three levels: chi-square with 2 degrees of freedom
    chi2 = ((cnt - m / 3) ** 2 / (m / 3)).sum()
    assert chi2 < 20.0


@pytest.mark.parametrize("model", ["wc", "p"])
def test_fixed_point_gamma_within_bound(model):
    n, m = 300, 2500
    src, dst = synth.er(n, m, 3)
    if model == "wc":
        g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    else:
        g = oracle.OracleGraph(n, src, dst, weights=synth.uniform_p(m, 4, 0.0, 0.2), model=oracle.W_P)
    a = g.arrays()
    probs = [p_eff(t) for t in a["tau"]]
    dst_csr = np.repeat(np.arange(n), np.diff(a["off"]))
    gam = gamma(n, dst_csr.tolist(), probs)
    deg = np.diff(a["off"])
    assert g.f == 62 - (int(np.ceil(np.log2(n))) + 1)
    for v in range(n):
        approx = Fraction(int(a["w"][v]), 1 << g.f)
        bound = Fraction(1, 1 << g.f) + Fraction(int(deg[v]), 1 << 62)
        assert abs(approx - gam[v]) <= bound, v
    assert int(a["w"].astype(object).sum()) == g.W
    assert g.W <= 1 << 61


def _alias_mass(a, n, W):
    """Mass each vertex receives over all columns of the alias table."""
    mass = [0] * n
    for c in range(n):
        pr = int(a["prob"][c])
        assert 0 <= pr <= W
        mass[c] += pr
        mass[int(a["alias"][c])] += W - pr
    return mass


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_alias_table_represents_source_law_exactly(seed):
    # Eq. probu: Pr[src = v] = gamma_v / Gamma. With the fixed-point values the
    # table must give vertex v exactly mass w_v * n out of n columns of W.
    n, m = 500, 3000
    src, dst = synth.chunglu(n, m, 2.1, seed)
    g = oracle.OracleGraph(n, src, dst, weights=synth.tri(m, seed), model=oracle.W_P)
    a = g.arrays()
    mass = _alias_mass(a, n, g.W)
    assert mass == [int(x) * n for x in a["w"]]


def test_alias_table_degenerate_cases():
    # all mass on one vertex (in-star): every column aliases the centre
    d = 9
    g = oracle.OracleGraph(d + 1, list(range(1, d + 1)), [0] * d, model=oracle.W_WC)
    a = g.arrays()
    assert _alias_mass(a, d + 1, g.W) == [int(x) * (d + 1) for x in a["w"]]
    assert a["w"][1:].sum() == 0 and a["w"][0] == g.W
    # equal masses everywhere (directed cycle, WC): all columns full, alias = self
    n = 8
    g = oracle.OracleGraph(n, list(range(n)), [(i + 1) % n for i in range(n)], model=oracle.W_WC)
    a = g.arrays()
    assert a["prob"].tolist() == [g.W] * n and a["alias"].tolist() == list(range(n))


def test_source_draw_follows_alias_law():
    # The draw from the table: empirical source frequencies of oracle samples
    # on a graph where every in-edge is always live (so no sample is rejected
    # and every vertex with an in-edge can be a source).
    n, m = 60, 240
    src, dst = synth.er(n, m, 12)
    tau = np.full(m, SENT, np.uint32)
    # mix in some finite thresholds so the masses differ
    tau[::3] = 1 << 30
    g = oracle.OracleGraph(n, src, dst, weights=tau, model=oracle.W_TAU)
    a = g.arrays()
    T = 200_000
    out = g.sample_ids(0xABC, np.arange(T, dtype=np.uint64))
    cnt = np.bincount(out["src"], minlength=n)
    expect = a["w"].astype(np.float64) / float(g.W) * T
    keep = expect > 0
    assert cnt[~keep].sum() == 0
    chi2 = ((cnt[keep] - expect[keep]) ** 2 / expect[keep]).sum()
    dof = keep.sum() - 1
    # 5-sigma upper bound on a chi-square with dof degrees of freedom
    assert chi2 < dof + 5 * np.sqrt(2 * dof)
