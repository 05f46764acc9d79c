"""Batched multi-graph mode (lp_batch_*, needs a GPU).

Graphs of uneven sizes (and an edgeless one) are packed into one
block-diagonal graph; the recorded per-source query over every vertex must
give, for each graph, exactly what lp_predict_sources gives on that graph
alone (ids shifted by the graph's base), call after call (CUDA-graph
replays), and after the autotuner has changed the binning options.  Sampled
rows are also checked against the oracle.
"""
import numpy as np
import pytest

import lp_inputs as L
import oracle
from parity import compare_sources

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
def graphs():
    rng = np.random.default_rng(2024)
    gs = []
    for i in range(12):
        n = int(np.exp(rng.uniform(np.log(150), np.log(4000))))
        deg = float(rng.uniform(4, 16))
        gamma = float(rng.uniform(2.0, 2.8))
        gs.append(L.chung_lu(n, deg, gamma, dmax=n ** 0.6 * 4, seed=1000 + i))
    gs.insert(5, L.from_edges(7, np.array([], np.int32), np.array([], np.int32)))  # no edges
    return gs


def _rows(lp, out, cnt, n_total, k):
    links = out.cpu().numpy().view(lp.LINK_DTYPE)[: n_total * k].reshape(n_total, k)
    return links, cnt.cpu().numpy()[:n_total]


@pytest.mark.parametrize("measure,cap", [("JC", None), ("AA", 32), ("RA", 256)])
def test_batch_equals_each_graph_alone(lp, graphs, measure, cap):
    k = 10
    with lp.Batch(graphs) as B:
        assert B.n_graphs == len(graphs) and B.n_total == sum(g.n for g in graphs)
        out, cnt = B.predict_all(measure, cap, k)
        links, counts = _rows(lp, out, cnt, B.n_total, k)
        first = out.clone()
        out2, _ = B.predict_all(measure, cap, k)          # a replay
        assert np.array_equal(out2.cpu().numpy(), first.cpu().numpy())
        for i, g in enumerate(graphs):
            b0, b1 = int(B.bases[i]), int(B.bases[i + 1])
            assert b1 - b0 == g.n
            if g.n == 0:
                continue
            gl, gc = links[b0:b1].copy(), counts[b0:b1]
            live = gl["u"] >= 0
            gl["u"][live] -= b0
            gl["v"][live] -= b0
            with lp.Graph.from_csr(g) as G:
                el, ec = G.predict_sources(measure, np.arange(g.n, dtype=np.int32), k, cap)
            assert np.array_equal(gc, ec), (measure, i)
            if measure in ("AA", "RA"):
                # the packed graph's larger max degree may pick another
                # fixed-point scale, so near-equal sums can swap: every row
                # is checked against the oracle within the AA/RA tolerance
                every = np.arange(g.n, dtype=np.int32)
                ol, oc = oracle.predict_sources(g.n, g.off, g.idx, measure, every, k, cap)
                compare_sources(gl, gc, ol, oc, measure, g, every, cap)
            else:
                assert gl.tobytes() == el.tobytes(), (measure, i)
            if i in (0, 3):
                rng = np.random.default_rng(i)
                pick = np.sort(rng.choice(g.n, min(40, g.n), replace=False)).astype(np.int32)
                ol, oc = oracle.predict_sources(g.n, g.off, g.idx, measure, pick, k, cap)
                compare_sources(gl[pick], gc[pick], ol, oc, measure, g, pick, cap)


def test_autotune_keeps_results(lp, graphs):
    k = 8
    with lp.Batch(graphs) as B:
        out, cnt = B.predict_all("JC", 256, k)
        ref = out.clone().cpu().numpy()
        d, b, opts = B.autotune("JC", 256, k, repeats=1)
        assert d > 0 and 0 < b <= d
        assert set(opts) == {"warp_max", "med_max", "cta_max", "item_wedges", "big_threads"}
        assert opts["big_threads"] in (512, 1024)
        out2, _ = B.predict_all("JC", 256, k)
        assert np.array_equal(out2.cpu().numpy(), ref)


def test_batch_rejects_bad_input(lp):
    bad = L.Graph(3, np.array([0, 1, 2, 2], np.int32), np.array([1, 5], np.int32))
    with pytest.raises(lp.LPError) as e:
        lp.Batch([L.gnp(20, 0.2, 1), bad])
    assert e.value.status == lp.LP_EINVAL
    with lp.Batch([L.gnp(30, 0.2, 2)]) as B:
        with pytest.raises(lp.LPError) as e:
            B.predict_all("JC", None, 0)
        assert e.value.status == lp.LP_EINVAL


def test_overflowing_split_items_fall_back(lp, graphs):
    """Tiny split tables make split hash items overflow on the first replay;
    the plan is recorded again with dense items and the rows stay exact."""
    keys = (lp.LP_OPT_CTA_MAX_WEDGES, lp.LP_OPT_SPLIT_TARGET, lp.LP_OPT_SPLIT_LOGCAP)
    old = [lp.lp_get_option(x) for x in keys]
    try:
        for x, v in zip(keys, (257, 256, 6)):
            lp.lp_set_option(x, v)
        with lp.Batch(graphs) as B:
            out, cnt = B.predict_all("CN", None, 6)
            links, counts = _rows(lp, out, cnt, B.n_total, 6)
    finally:
        for x, v in zip(keys, old):
            lp.lp_set_option(x, v)
    for i in (0, 4, 8):
        g = graphs[i]
        b0, b1 = int(B.bases[i]), int(B.bases[i + 1])
        gl = links[b0:b1].copy()
        live = gl["u"] >= 0
        gl["u"][live] -= b0
        gl["v"][live] -= b0
        with lp.Graph.from_csr(g) as G:
            el, ec = G.predict_sources("CN", np.arange(g.n, dtype=np.int32), 6, None)
        assert np.array_equal(counts[b0:b1], ec)
        assert gl.tobytes() == el.tobytes()
