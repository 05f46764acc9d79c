"""Source sharding of the global mode across GPUs.

Sources are independent units (Section 4.1.7): the pairs (u, v), u < v, of a
source u are found by the scan of u alone.  So the global mode shards by
source range: each GPU runs ``lp_predict_range`` over one contiguous range of
[0, n) and keeps its best k, and the best k of the union of those lists,
under the library's total order (score desc, u asc, v asc), is the unsharded
result.  The global mode needs exactly one exchange: the ranks' lists are
all-gathered and merged (``predict_distributed``).  The per-source mode needs
none (its rows just concatenate).

This module only partitions, gathers and hands the lists to a merge.  The
merge is the library's ``lp_merge_links`` (``library_merge``): it orders the
links by the exact keys of the library's own selection (rebuilt on the
device), so the merged list equals one ``lp_predict`` call bit for bit.

``shard_bounds`` balances the ranges by an upper bound of each source's wedge
work (the degrees of its intermediaries that pass the hub test).
"""
from __future__ import annotations

import numpy as np


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


def gather_parts(parts):
    """One array of the links of every non-empty part (the merge input)."""
    given = [p for p in parts if p is not None]
    nonempty = [p for p in given if len(p)]
    if nonempty:
        return np.concatenate(nonempty)
    if given:
        return np.zeros(0, dtype=given[0].dtype)
    from . import LINK_DTYPE
    return np.zeros(0, dtype=LINK_DTYPE)


def library_merge(graph, measure: str, degree_cap):
    """merge(parts, k) through lp_merge_links on `graph` (a Graph whose
    lp_predict_range produced the parts)."""
    def merge(parts, k):
        return graph.merge(measure, degree_cap, gather_parts(parts), k)
    return merge


def predict_sharded(predict_range, merge, bounds, measure: str, degree_cap, k: int,
                    threshold: float = 0.0) -> np.ndarray:
    """Run every range in turn (one process, e.g. one GPU standing in for
    several) and merge.  predict_range(measure, cap, k, begin, end, threshold)
    returns a range's sorted best k (Graph.predict_range); merge(parts, k)
    returns the best k of their union (library_merge)."""
    parts = [predict_range(measure, degree_cap, k, bounds[i], bounds[i + 1], threshold)
             for i in range(len(bounds) - 1)]
    return merge(parts, k)


def predict_distributed(predict_range, merge, bounds, measure: str, degree_cap, k: int,
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
    return merge(parts, k)
