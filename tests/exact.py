"""Exact truths for tiny probabilistic graphs, by enumerating every live-edge
world (Sec. II-A, Eq. 1-2 of arXiv 1709.03565). Pure Python with Fractions;
independent of both the oracle and the CUDA library."""
from __future__ import annotations

from collections import deque
from fractions import Fraction

SENT = 0xFFFFFFFF
TWO32 = 1 << 32


def tau_from_p(p: float) -> int:
    """floor(p * 2^32) from the exact binary value of the double p, clamped
    to the always-live sentinel."""
    if p >= 1.0:
        return SENT
    return min((Fraction(p) * TWO32).__floor__(), SENT)


def p_eff(tau: int) -> Fraction:
    """Effective edge probability of a threshold: tau / 2^32, 1 for the sentinel."""
    return Fraction(1) if int(tau) == SENT else Fraction(int(tau), TWO32)


def worlds(probs):
    """Every live-edge world (bitmask over edges) with its probability, Eq. 1."""
    m = len(probs)
    for mask in range(1 << m):
        pr = Fraction(1)
        for e in range(m):
            pr *= probs[e] if (mask >> e) & 1 else (1 - probs[e])
        if pr:
            yield mask, pr


def _reach(n, heads, tails, mask, start):
    """Vertices reachable from ``start`` along live edges tails[e] -> heads[e]."""
    adj = [[] for _ in range(n)]
    for e in range(len(heads)):
        if (mask >> e) & 1:
            adj[tails[e]].append(heads[e])
    seen = set(start)
    q = deque(start)
    while q:
        x = q.popleft()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                q.append(y)
    return seen


def influence(n, src, dst, probs, S) -> Fraction:
    """I(S) = sum_g |eta_g(S)| Pr[g] (Eq. 2)."""
    tot = Fraction(0)
    for mask, pr in worlds(probs):
        tot += pr * len(_reach(n, list(dst), list(src), mask, list(S)))
    return tot


def gamma(n, dst, probs):
    """gamma_v = 1 - prod over in-edges of (1 - w) (Eq. gamma_v), exactly."""
    g = [Fraction(1)] * n
    for e, v in enumerate(dst):
        g[v] *= 1 - probs[e]
    return [1 - x for x in g]


def rr_law(n, src, dst, probs):
    """Pr over worlds of the reverse-reachable set of each v:
    {v: {frozenset(R): Pr[eta^-_g(v) = R]}}."""
    law = {v: {} for v in range(n)}
    for mask, pr in worlds(probs):
        for v in range(n):
            R = frozenset(_reach(n, list(src), list(dst), mask, [v]))
            law[v][R] = law[v].get(R, Fraction(0)) + pr
    return law


def iis_law(n, src, dst, probs, w, W):
    """Law of one IIS sample (source, R) when the source is drawn with
    probability w_v / W and the first step is conditioned on a live in-edge
    (Lemma 2): Pr[(v, R)] = (w_v / W) * Pr[eta^-(v) = R] / gamma_v for R != {v}."""
    law = rr_law(n, src, dst, probs)
    gam = gamma(n, dst, probs)
    out = {}
    for v in range(n):
        if w[v] == 0:
            continue
        for R, pr in law[v].items():
            if R == frozenset([v]):
                continue
            out[(v, R)] = Fraction(int(w[v]), int(W)) * pr / gam[v]
    return out


# ------------------------------------------------------ Linear Threshold --
def lt_worlds(n, dst, probs):
    """Live-edge worlds of the Linear Threshold model (Kempe et al.): every
    vertex keeps at most one in-edge, edge e with probability w_e and none
    with probability 1 - sum of its row. Yields (kept edge per vertex or
    None, probability)."""
    import itertools

    options = []
    for v in range(n):
        row = [e for e in range(len(dst)) if dst[e] == v]
        rest = 1 - sum((probs[e] for e in row), Fraction(0))
        assert rest >= 0, "row weights above 1"
        options.append([(e, probs[e]) for e in row] + [(None, rest)])
    for combo in itertools.product(*options):
        pr = Fraction(1)
        for _, p in combo:
            pr *= p
        if pr:
            yield tuple(c for c, _ in combo), pr


def _lt_rr(src, kept, v):
    """Vertices that reach v in an LT world: the chain of kept in-edges back
    from v (each vertex keeps at most one), up to a repeat."""
    R = [v]
    x = v
    while kept[x] is not None:
        u = src[kept[x]]
        if u in R:
            break
        R.append(u)
        x = u
    return frozenset(R)


def lt_rr_law(n, src, dst, probs):
    """{v: {R: Pr[the LT reverse-reachable set of v is R]}}."""
    law = {v: {} for v in range(n)}
    for kept, pr in lt_worlds(n, dst, probs):
        for v in range(n):
            R = _lt_rr(src, kept, v)
            law[v][R] = law[v].get(R, Fraction(0)) + pr
    return law


def lt_iis_law(n, src, dst, probs, w, W):
    """Law of an LT importance sample: source v with probability w_v / W, then
    the reverse-reachable set of v conditioned on v keeping an in-edge
    (gamma_v = its row's weight sum): {(v, R): probability}."""
    law = {}
    gam = [sum((probs[e] for e in range(len(dst)) if dst[e] == v), Fraction(0)) for v in range(n)]
    rr = lt_rr_law(n, src, dst, probs)
    for v in range(n):
        if w[v] == 0:
            continue
        for R, pr in rr[v].items():
            if len(R) >= 2:
                law[(v, R)] = Fraction(int(w[v]), int(W)) * pr / gam[v]
    return law


def lt_influence(n, src, dst, probs, S) -> Fraction:
    """I(S) under LT: expected number of vertices whose reverse-reachable set
    meets S."""
    S = set(S)
    tot = Fraction(0)
    for kept, pr in lt_worlds(n, dst, probs):
        tot += pr * sum(1 for x in range(n) if _lt_rr(src, kept, x) & S)
    return tot
