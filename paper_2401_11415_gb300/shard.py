"""Source sharding of the global mode across GPUs.

Sources are independent units (Section 4.1.7): the pairs (u, v), u < v, of a
source u are found by the scan of u alone.  So the global mode shards by
source range: each GPU runs ``lp_predict_range`` over one contiguous range of
[0, n) and keeps its best k, and the best k of the union of those lists,
under the library's total order (score desc, u asc, v asc), is the unsharded
result.  The global mode needs exactly one exchange: the ranks' lists are
all-gathered and merged (``predict_distributed``).  The per-source mode needs
none (its rows just concatenate).

``shard_bounds`` balances the ranges by an upper bound of each source's wedge
work (the degrees of its intermediaries that pass the hub test).
``merge_topk`` orders the count measures exactly, by the rational key
recomputed from the common-neighbour count and the two degrees; AA and RA by
their FP32 score (the lists agree with the unsharded call up to pairs within
FP32 rounding of each other).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

COUNT_MEASURES = ("CN", "JC", "SI", "SC", "HP", "HD", "LHN")


def shard_bounds(off, idx, nshards: int, degree_cap=None) -> list[int]:
    """Split points 0 = b0 <= b1 <= ... <= b_nshards = n of contiguous source
    ranges with about equal work bound sum_{b in Gamma_a, |Gamma_b| <= L_H} |Gamma_b|."""
    off = np.asarray(off, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    n = off.size - 1
    if nshards < 1:
        raise ValueError("nshards must be >= 1")
    deg = np.diff(off)
    db = deg[idx] if idx.size else np.zeros(0, np.int64)
    if degree_cap is not None and degree_cap >= 0:
        db = np.where(db <= degree_cap, db, 0)
    csum = np.concatenate([[0], np.cumsum(db)])
    work = csum[off]  # work before each source (prefix over arcs), n + 1 entries
    total = work[-1]
    bounds = [0]
    for s in range(1, nshards):
        bounds.append(int(np.searchsorted(work, total * s / nshards, side="left")))
    bounds.append(n)
    for i in range(1, len(bounds)):
        bounds[i] = max(bounds[i], bounds[i - 1])
    return bounds


def _key(measure: str, cn: int, du: int, dv: int):
    """The exact ordering key of a count measure (Eq. 1-7, Salton through its
    square), as the library defines it."""
    if measure == "CN":
        return Fraction(cn)
    if measure == "JC":
        return Fraction(cn, du + dv - cn)
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


def merge_topk(parts, k: int, measure: str, deg) -> np.ndarray:
    """The best k links of the union of the sorted lists in `parts` (arrays of
    the library's link dtype) under (score desc, u asc, v asc); `deg` is the
    degree array of the graph."""
    given = [p for p in parts if p is not None]
    nonempty = [p for p in given if len(p)]
    if not nonempty:
        return np.zeros(0, dtype=given[0].dtype) if given else np.zeros(0)
    allp = np.concatenate(nonempty)
    u = allp["u"].astype(np.int64)
    v = allp["v"].astype(np.int64)
    if measure in COUNT_MEASURES:
        deg = np.asarray(deg, dtype=np.int64)
        keys = [_key(measure, int(c), int(deg[a]), int(deg[b]))
                for c, a, b in zip(allp["cn"].tolist(), u.tolist(), v.tolist())]
        order = sorted(range(len(allp)), key=lambda i: (-keys[i], u[i], v[i]))
        order = np.asarray(order, dtype=np.int64)
    else:
        order = np.lexsort((v, u, -allp["score"].astype(np.float64)))
    return allp[order[: max(k, 0)]].copy()


def predict_sharded(predict_range, n: int, bounds, measure: str, degree_cap, k: int, deg,
                    threshold: float = 0.0) -> np.ndarray:
    """Run every range in turn (one process, e.g. one GPU standing in for
    several) and merge.  predict_range(measure, cap, k, begin, end, threshold)
    returns a range's sorted best k (Graph.predict_range)."""
    parts = [predict_range(measure, degree_cap, k, bounds[i], bounds[i + 1], threshold)
             for i in range(len(bounds) - 1)]
    return merge_topk(parts, k, measure, deg)


def predict_distributed(predict_range, bounds, measure: str, degree_cap, k: int, deg,
                        threshold: float = 0.0, group=None) -> np.ndarray:
    """One range per rank of the default torch.distributed group (len(bounds)
    = world size + 1): the rank's best k, one all_gather of the lists, and the
    same merge on every rank."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    if len(bounds) != world + 1:
        raise ValueError("need one range per rank")
    mine = predict_range(measure, degree_cap, k, bounds[rank], bounds[rank + 1], threshold)
    parts = [None] * world
    dist.all_gather_object(parts, mine, group=group)
    return merge_topk(parts, k, measure, deg)
