"""The expand-and-count large tier of the global mode (needs a GPU).

Large sources whose wedges would be cut into several id-range items are
instead expanded once into records grouped by bucket and counted bucket by
bucket (dense counters or a hash table per bucket).  The tier is forced on a
graph small enough for the oracle, with small tier limits (so that many
sources take it), small batches (several expand batches per call), a small
selection buffer (count items fail and are re-queued across compactions) and
64-slot hash tables (buckets overflow and are re-split).  Every result must
match the oracle (parity tolerance) and equal, byte for byte, the same call
without the tier: options change speed, never results.
"""
import numpy as np
import pytest

import lp_inputs as L
import oracle
from parity import compare_global

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_11415_gb300 import _build
    _build.build()
    import paper_2401_11415_gb300 as m
    torch.cuda.init()
    return m


@pytest.fixture(scope="module")
def graph():
    # hubs of a few thousand neighbours: multi-bucket dense units; mid-degree
    # sources with wide, sparse second-order ranges: hash units
    return L.chung_lu(200000, 8.0, 2.1, dmax=3000, seed=12)


def with_options(lp, opts, fn):
    saved = {o: lp.lp_get_option(o) for o in opts}
    try:
        for o, v in opts.items():
            lp.lp_set_option(o, v)
        return fn()
    finally:
        for o, v in saved.items():
            lp.lp_set_option(o, v)


def tier_opts(lp, extra):
    o = {lp.LP_OPT_WARP_MAX_WEDGES: 64, lp.LP_OPT_MED_MAX_WEDGES: 128,
         lp.LP_OPT_CTA_MAX_WEDGES: 257}
    o.update(extra)
    return o


@pytest.mark.parametrize("measure", ["JC", "CN", "SC", "HP", "AA", "RA"])
@pytest.mark.parametrize("cap", [None, 64])
def test_expand_tier_matches_oracle(lp, graph, measure, cap):
    g = graph
    k = 20000
    with lp.Graph.from_csr(g) as G:
        base = with_options(lp, tier_opts(lp, {lp.LP_OPT_EXPAND: 0}),
                            lambda: G.predict(measure, cap, k))
        got, st = with_options(lp, tier_opts(lp, {lp.LP_OPT_EXPAND: 1,
                                                  lp.LP_OPT_EXPAND_BATCH: 1 << 16}),
                               lambda: (G.predict(measure, cap, k), lp.lp_last_stats()))
    assert st["exp_units"] > 0 and st["exp_batches"] > 1 and st["tier_launches"][3] > 0
    assert got.tobytes() == base.tobytes()
    exp = oracle.predict(g.n, g.off, g.idx, measure, cap, k=k)
    compare_global(got, exp, measure, g, cap)


@pytest.mark.parametrize("measure", ["JC", "RA"])
def test_expand_tier_overflow_and_compaction(lp, graph, measure):
    """64-slot hash tables (every hash bucket overflows and is re-split) and a
    selection buffer a little above 2k (count items fail when it fills and
    are re-queued after the compaction)."""
    g = graph
    k = 20000
    with lp.Graph.from_csr(g) as G:
        base = with_options(lp, {lp.LP_OPT_EXPAND: 0}, lambda: G.predict(measure, None, k))
        opts = tier_opts(lp, {lp.LP_OPT_EXPAND: 1, lp.LP_OPT_EXPAND_BATCH: 1 << 17,
                              lp.LP_OPT_EXPAND_HASH_LOGCAP: 6, lp.LP_OPT_SELECT_BUFFER: 4096})
        got, st = with_options(lp, opts, lambda: (G.predict(measure, None, k), lp.lp_last_stats()))
    assert st["exp_units"] > 0 and st["splits"] > 0 and st["compactions"] > 1
    assert got.tobytes() == base.tobytes()
