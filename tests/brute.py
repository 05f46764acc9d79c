"""Brute-force link prediction straight from the definitions (test helper).

Scores every non-adjacent pair u < v by intersecting Python sets, with exact
rational arithmetic (fractions.Fraction) for the seven count measures of
Section 3.1 (Eq. 1-7) and FP64 sums for AA and RA (Eq. 8-9, read over the
common neighbours).  This is the naive baseline of Section 3.3, quadratic in
|V|, used only to pin the oracle on tiny graphs.  It shares no code with the
oracle.
"""
from __future__ import annotations

import math
from fractions import Fraction

MEASURES = ["CN", "JC", "SI", "SC", "HP", "HD", "LHN", "AA", "RA"]


def adjacency(g):
    return [set(int(x) for x in g.idx[g.off[i]:g.off[i + 1]]) for i in range(g.n)]


def exact_score(measure, cn, du, dv, union_size=None):
    """Exact ordering key of Eq. 1-7 (Salton through its square)."""
    if measure == "CN":
        return Fraction(cn)
    if measure == "JC":
        den = du + dv - cn
        if union_size is not None:
            assert den == union_size
        return Fraction(cn, den)
    if measure == "SI":
        return Fraction(cn, du + dv)
    if measure == "SC":
        return Fraction(cn * cn, du * dv)
    if measure == "HP":
        return Fraction(cn, min(du, dv))
    if measure == "HD":
        return Fraction(cn, max(du, dv))
    if measure == "LHN":
        return Fraction(cn, du * dv)
    raise ValueError(measure)


def float_score(measure, key):
    if measure == "SC":
        return math.sqrt(key.numerator / key.denominator) if key else 0.0
    return key.numerator / key.denominator


def pair_score(adj, deg, measure, u, v, cap=None):
    """(cn, key, value) for one pair; key is a Fraction (count measures) or
    the FP64 sum in increasing order of the common neighbour (AA/RA)."""
    common = sorted(b for b in (adj[u] & adj[v]) if cap is None or deg[b] <= cap)
    cn = len(common)
    if measure in ("AA", "RA"):
        s = 0.0
        for b in common:
            s += (1.0 / math.log(deg[b])) if measure == "AA" else (1.0 / deg[b])
        return cn, s, s
    if cn == 0:
        return 0, Fraction(0), 0.0
    union = len(adj[u] | adj[v]) if cap is None else None
    key = exact_score(measure, cn, deg[u], deg[v], union)
    return cn, key, float_score(measure, key)


def predict(g, measure, cap=None, k=0, threshold=0.0):
    """All pairs u < v, not adjacent, with cn > 0 and value > threshold,
    sorted by (key desc, u asc, v asc); first k (k = 0: all).
    Returns a list of (u, v, cn, key, value)."""
    adj = adjacency(g)
    deg = [len(a) for a in adj]
    out = []
    for u in range(g.n):
        for v in range(u + 1, g.n):
            if v in adj[u]:
                continue
            cn, key, value = pair_score(adj, deg, measure, u, v, cap)
            if cn == 0 or not value > threshold:
                continue
            out.append((u, v, cn, key, value))
    out.sort(key=lambda t: (-t[3], t[0], t[1]))
    return out[:k] if k else out


def predict_source(g, measure, a, k, cap=None, threshold=0.0):
    """Per-source form: partners c != a, not adjacent, cn > 0, value > threshold,
    sorted by (key desc, c asc), first k."""
    adj = adjacency(g)
    deg = [len(x) for x in adj]
    out = []
    for c in range(g.n):
        if c == a or c in adj[a]:
            continue
        cn, key, value = pair_score(adj, deg, measure, a, c, cap)
        if cn == 0 or not value > threshold:
            continue
        out.append((a, c, cn, key, value))
    out.sort(key=lambda t: (-t[3], t[1]))
    return out[:k]
