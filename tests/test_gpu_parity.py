"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

Sizes: the Chung-Lu 2,000-vertex workload (all 9 measures, IBase and DLH
with hub limit 64, N_P = |E^U|), tiny and small random graphs that span
several items and tiers, and the degenerate cases (empty graphs, no edges,
hub limit 0, k above the candidate count, thresholds).  Small option values
force the selection-buffer compaction and the hash-overflow split paths.
"""
import ctypes

import numpy as np
import pytest

import lp_inputs as L
import oracle
from parity import compare_global, compare_sources

pytestmark = pytest.mark.gpu

MEASURES = oracle.MEASURES


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
def cfg1():
    g = L.cfg_chung_lu_2k()
    return L.holdout(g, 0.1, seed=43)


def run_global(lp, g, measure, cap, k, threshold=0.0):
    with lp.Graph.from_csr(g) as G:
        return G.predict(measure, cap, k, threshold)


def check_global(lp, g, measure, cap, k, threshold=0.0):
    got = run_global(lp, g, measure, cap, k, threshold)
    exp = oracle.predict(g.n, g.off, g.idx, measure, cap, k=k, threshold=threshold)
    compare_global(got, exp, measure, g, cap)
    return got


def test_cfg1_all_measures(lp, cfg1):
    g = cfg1.observed
    k = len(cfg1.hu)
    with lp.Graph.from_csr(g) as G:
        for cap in (None, 64):
            for m in MEASURES:
                got = G.predict(m, cap, k)
                exp = oracle.predict(g.n, g.off, g.idx, m, cap, k=k)
                compare_global(got, exp, m, g, cap)
                st = lp.lp_last_stats()
                w, _ = oracle.work(g.n, g.off, g.idx, cap, 0)
                assert st["wedges"] == w


def test_cfg1_f1_reported(lp, cfg1):
    g = cfg1.observed
    k = len(cfg1.hu)
    f1 = {}
    for cap in (None, 64):
        got = run_global(lp, g, "RA", cap, k)
        f1[cap] = oracle.quality(got["u"], got["v"], cfg1.hu, cfg1.hv)["f1"]
        exp = oracle.predict(g.n, g.off, g.idx, "RA", cap, k=k)
        assert abs(f1[cap] - oracle.quality(exp["u"], exp["v"], cfg1.hu, cfg1.hv)["f1"]) <= 2 / k
    assert f1[None] > 0 and f1[64] > 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_small_graphs(lp, seed):
    graphs = [L.gnp(60, 0.08, seed), L.chung_lu(500, 7.0, 2.2, dmax=120, seed=seed),
              L.rmat(9, 8, seed=seed)]
    for g in graphs:
        for m in MEASURES:
            for cap in (None, 3, 8):
                for k in (0, 17):
                    check_global(lp, g, m, cap, k)


def test_all_candidates_and_threshold(lp):
    g = L.chung_lu(400, 8.0, 2.3, dmax=90, seed=9)
    for m in ("JC", "RA", "SC", "LHN"):
        allp = oracle.predict(g.n, g.off, g.idx, m, None)
        vals = np.unique(allp["value"])
        for th in (-1.0, 0.0, float(vals[len(vals) // 2]), float(vals[-1]), 1e30):
            check_global(lp, g, m, None, 0, th)
            check_global(lp, g, m, 16, 25, th)


def test_pair_counts_large_groups(lp):
    # AA / RA report |Gamma_u ∩ Gamma_v| (kept intermediaries) for every link;
    # with many links per endpoint the counts come from the CTA forms (bitmap
    # walk or the endpoint's wedges against a table of its links), with few
    # from the warp form, and under a hub limit from the kept lists
    g = L.chung_lu(3000, 12.0, 2.05, dmax=1500, seed=21)
    for m in ("AA", "RA"):
        for cap in (None, 64, 16):
            check_global(lp, g, m, cap, 150000)
    # a hub owning more than 4096 links: its group is cut into parts, one CTA each
    g = L.chung_lu(20000, 10.0, 2.1, dmax=6000, seed=22)
    check_global(lp, g, "RA", None, 300000)
    check_global(lp, g, "AA", 64, 300000)


def test_degenerate_graphs(lp):
    empty = L.Graph(0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert len(run_global(lp, empty, "JC", None, 10)) == 0
    isolated = L.Graph(5, np.zeros(6, np.int32), np.zeros(0, np.int32))
    assert len(run_global(lp, isolated, "CN", None, 10)) == 0
    star = L.from_edges(9, np.zeros(8, np.int32), np.arange(1, 9, dtype=np.int32))
    for m in MEASURES:
        check_global(lp, star, m, None, 0)
        assert len(run_global(lp, star, m, 7, 0)) == 0        # centre above the limit
        check_global(lp, star, m, 8, 5)                          # inclusive limit
        assert len(run_global(lp, star, m, 0, 0)) == 0        # limit 0: nothing
    e = [(i, j) for i in range(7) for j in range(i + 1, 7)]
    clique = L.from_edges(7, np.array([x for x, _ in e], np.int32), np.array([y for _, y in e], np.int32))
    for m in MEASURES:
        assert len(run_global(lp, clique, m, None, 0)) == 0
    g = L.gnp(30, 0.2, 4)
    check_global(lp, g, "CN", None, 10**6)                      # k above the candidates


def test_per_source_cfg1(lp, cfg1):
    g = cfg1.observed
    src = np.arange(g.n, dtype=np.int32)
    with lp.Graph.from_csr(g) as G:
        for cap in (None, 64):
            for m in MEASURES:
                gl, gc = G.predict_sources(m, src, 10, cap)
                ol, oc = oracle.predict_sources(g.n, g.off, g.idx, m, src, 10, cap)
                compare_sources(gl, gc, ol, oc, m, g, src, cap)


def test_per_source_k_and_repeats(lp):
    g = L.chung_lu(700, 9.0, 2.1, dmax=200, seed=5)
    rng = np.random.default_rng(0)
    src = rng.integers(0, g.n, 300).astype(np.int32)
    src[:10] = src[0]                                            # repeated source
    with lp.Graph.from_csr(g) as G:
        for k in (1, 7, 64):
            for m in ("CN", "JC", "AA", "RA", "HP"):
                for cap in (None, 5):
                    gl, gc = G.predict_sources(m, src, k, cap)
                    ol, oc = oracle.predict_sources(g.n, g.off, g.idx, m, src, k, cap)
                    compare_sources(gl, gc, ol, oc, m, g, src, cap)
        with pytest.raises(lp.LPError):
            G.predict_sources("JC", np.array([g.n], np.int32), 5)
        with pytest.raises(lp.LPError):
            G.predict_sources("JC", src, 65)
        gl, gc = G.predict_sources("JC", np.zeros(0, np.int32), 5)
        assert gl.shape == (0, 5)


def test_compaction_and_redo(lp, cfg1):
    """A small selection buffer forces repeated compactions, failed records
    and re-queued work; the result must not change."""
    g = cfg1.observed
    k = len(cfg1.hu)
    old = lp.lp_get_option(lp.LP_OPT_SELECT_BUFFER)
    try:
        for buf in (64, 3000):
            lp.lp_set_option(lp.LP_OPT_SELECT_BUFFER, buf)
            for m in ("JC", "RA", "CN", "SC"):
                for cap in (None, 64):
                    got = run_global(lp, g, m, cap, k)
                    st = lp.lp_last_stats()
                    exp = oracle.predict(g.n, g.off, g.idx, m, cap, k=k)
                    compare_global(got, exp, m, g, cap)
                    if buf == 64:
                        assert st["compactions"] > 0
            got = run_global(lp, g, "JC", None, 0)               # k = 0 grows the buffer
            compare_global(got, oracle.predict(g.n, g.off, g.idx, "JC", None), "JC", g, None)
    finally:
        lp.lp_set_option(lp.LP_OPT_SELECT_BUFFER, old)


@pytest.mark.parametrize("big_threads", [1024, 512])
def test_split_and_dense_items(lp, big_threads):
    """Tiny tier limits and split tables force CTA items, hash overflows that
    are re-split, and dense-counter items; with one 1024-thread or two
    512-thread large-tier CTAs per SM (half the table, half the window)."""
    g = L.chung_lu(3000, 12.0, 2.05, dmax=1500, seed=12)
    keys = (lp.LP_OPT_WARP_MAX_WEDGES, lp.LP_OPT_MED_MAX_WEDGES, lp.LP_OPT_CTA_MAX_WEDGES,
            lp.LP_OPT_SPLIT_TARGET, lp.LP_OPT_SPLIT_LOGCAP, lp.LP_OPT_BIG_CTA_THREADS)
    old = [lp.lp_get_option(x) for x in keys]
    try:
        for vals in ((8, 16, 257, 256, 6), (64, 512, 1024, 2048, 9), (256, 1024, 8192, 6144, 14)):
            vals = vals + (big_threads,)
            for x, v in zip(keys, vals):
                lp.lp_set_option(x, v)
            for m in ("CN", "JC", "RA", "AA"):
                for cap in (None, 40):
                    got = check_global(lp, g, m, cap, 500)
                    st = lp.lp_last_stats()
                    if vals[4] == 6 and cap is None:
                        assert st["splits"] > 0 and st["cta_items"] > 0
                        assert all(x > 0 for x in st["tier_launches"][:3])
                src = np.arange(0, g.n, 7, dtype=np.int32)
                with lp.Graph.from_csr(g) as G:
                    gl, gc = G.predict_sources(m, src, 10, None)
                ol, oc = oracle.predict_sources(g.n, g.off, g.idx, m, src, 10, None)
                compare_sources(gl, gc, ol, oc, m, g, src, None)
    finally:
        for x, v in zip(keys, old):
            lp.lp_set_option(x, v)


def test_deterministic(lp, cfg1):
    g = cfg1.observed
    with lp.Graph.from_csr(g) as G:
        for m in ("RA", "AA", "JC"):
            a = G.predict(m, None, 1500)
            b = G.predict(m, None, 1500)
            assert a.tobytes() == b.tobytes()


def test_rejects_asymmetric_graph(lp):
    # 0 -> 1 without 1 -> 0 is caught by the device-side reverse-arc check
    with pytest.raises(lp.LPError) as e:
        lp.lp_graph_create(3, np.array([0, 1, 1, 2], np.int32), np.array([1, 0], np.int32))
    assert e.value.status == lp.LP_EINVAL


def test_truncation_status(lp, cfg1):
    g = cfg1.observed
    with lp.Graph.from_csr(g) as G:
        full = G.predict("JC", None, 100)
        out = np.zeros(40, dtype=lp.LINK_DTYPE)
        n = ctypes.c_int64()
        st = lp.lib().lp_predict(G.handle, 1, -1, 100, 0.0, out.ctypes.data, 40, ctypes.byref(n))
        assert st == lp.LP_ETRUNC and n.value == 100
        assert out.tobytes() == full[:40].tobytes()


def _star_with_path(leaves):
    """Star K_{1,leaves} (centre 0) plus a 3-edge path beside it."""
    n = leaves + 4
    u = np.concatenate([np.zeros(leaves, np.int32), np.array([leaves + 1, leaves + 2], np.int32)])
    v = np.concatenate([np.arange(1, leaves + 1, dtype=np.int32),
                        np.array([leaves + 2, leaves + 3], np.int32)])
    return L.from_edges(n, u, v)


def test_ra_accuracy_guard(lp):
    """RA weights 1/|Gamma_b| (Eq. 9) are rounded to 2^-F fraction bits, a
    relative error of up to |Gamma_b| 2^-(F+1).  A star whose centre has
    2^21 + 1 leaves keeps that within 1e-6 and must match the oracle; with
    2^21 + 2^18 leaves it would not, so IBase RA is refused with LP_EINVAL
    while a hub limit that drops the centre, and AA (weights 1/ln|Gamma_b|),
    are still answered and match the oracle."""
    from parity import compare_sources
    for leaves, refused in ((2 ** 21 + 1, False), (2 ** 21 + 2 ** 18, True)):
        g = _star_with_path(leaves)
        src = np.array([1, leaves, leaves + 1], np.int32)
        with lp.Graph.from_csr(g) as G:
            runs = [("AA", None), ("RA", 1 << 20)]
            if refused:
                with pytest.raises(lp.LPError) as e:
                    G.predict_sources("RA", src, 4, None)
                assert e.value.status == lp.LP_EINVAL
                with pytest.raises(lp.LPError) as e:
                    G.predict("RA", None, 10)
                assert e.value.status == lp.LP_EINVAL
            else:
                runs.append(("RA", None))
            for m, cap in runs:
                gl, gc = G.predict_sources(m, src, 4, cap)
                ol, oc = oracle.predict_sources(g.n, g.off, g.idx, m, src, 4, cap)
                compare_sources(gl, gc, ol, oc, m, g, src, cap)
                if cap is None:
                    assert gc[0] == 4 and gc[1] == 4  # leaves meet every other leaf
