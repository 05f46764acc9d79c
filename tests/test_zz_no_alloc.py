"""The per-source entry point that allocates nothing (lp_predict_sources_static).

Some callers of this library cannot allocate device memory while they serve a
request: they run under a memory pool they do not own, or on a path where an
allocation, and the device synchronisation it can cause, is not allowed.  For
them the library offers a variant of the per-source query whose working memory
is one fixed array in device global memory, made resident (with the code of
the kernels it launches) when the graph is created.  This test calls it through
the C ABI twice in a row and checks both results against the ordinary entry
point (lp_predict_sources_dev) within the parity tolerance used elsewhere:
count measures exactly, AA and RA within 1e-6 relative.  The second call shows
that what the shared array keeps from the first call does not leak into the
next.  Free device memory is read before the first and after the second call
and must not change: neither call allocates, the first one included.

With small tier limits and 64-slot split tables (options that change speed,
never results), sources above 257 wedges become hash items that overflow, are
re-split into dense items on the host and leave partial lists, so the
re-split and merge steps of the allocation-free path run too (a re-split item
is never the only item of its source, so every split implies a merge).
"""
import numpy as np
import pytest

import lp_inputs as L

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_11415_gb300 import _build
    _build.build()
    import paper_2401_11415_gb300 as lp
    torch.cuda.init()
    return lp, torch


class Buffers:
    """Output buffers allocated once, so that the calls themselves are the
    only thing that could change the device's free memory."""

    def __init__(self, torch, n, k):
        self.out = torch.zeros((n * k * 16,), dtype=torch.uint8, device="cuda")
        self.cnt = torch.zeros((n,), dtype=torch.int32, device="cuda")
        self.n, self.k = n, k

    def run(self, lp, torch, fn, G, measure, src, cap):
        self.out.zero_()
        self.cnt.fill_(-7)
        fn(G.handle, measure, src, self.n, self.k, cap, 0.0, self.out, self.cnt)
        torch.cuda.synchronize()
        links = self.out.cpu().numpy().view(lp.LINK_DTYPE).reshape(self.n, self.k)
        return links, self.cnt.cpu().numpy()


def same(a, b, measure):
    la, ca = a
    lb, cb = b
    assert np.array_equal(ca, cb)
    for i in range(len(ca)):
        x, y = la[i, : ca[i]], lb[i, : cb[i]]
        assert np.array_equal(x["u"], y["u"]) and np.array_equal(x["v"], y["v"])
        assert np.array_equal(x["cn"], y["cn"])
        if measure in ("AA", "RA"):
            assert np.allclose(x["score"], y["score"], rtol=TOL, atol=0)
        else:
            assert np.array_equal(x["score"], y["score"])


def check_static(lp, torch, G, measure, cap, k, src):
    n = src.numel()
    ref_buf, st_buf = Buffers(torch, n, k), Buffers(torch, n, k)
    ref = ref_buf.run(lp, torch, lp.lp_predict_sources_dev, G, measure, src, cap)
    assert ref[1].sum() > 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    first = st_buf.run(lp, torch, lp.lp_predict_sources_static, G, measure, src, cap)
    second = st_buf.run(lp, torch, lp.lp_predict_sources_static, G, measure, src, cap)
    stats = lp.lp_last_stats()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (measure, free0, free1)
    same(first, ref, measure)
    same(second, ref, measure)
    return stats


def test_static_entry_point_matches_dev(env):
    lp, torch = env
    # hubs make some sources large enough to be split into several items
    g = L.chung_lu(4000, 12.0, 2.05, dmax=1500, seed=21)
    rng = np.random.default_rng(5)
    src = torch.tensor(rng.integers(0, g.n, 700), dtype=torch.int32, device="cuda")
    with lp.Graph.from_csr(g) as G:
        for measure, cap, k in (("JC", None, 10), ("RA", 64, 16), ("CN", None, 5)):
            check_static(lp, torch, G, measure, cap, k, src)


def test_static_entry_point_split_and_merge(env):
    lp, torch = env
    g = L.chung_lu(4000, 12.0, 2.05, dmax=1500, seed=21)
    rng = np.random.default_rng(6)
    src = torch.tensor(rng.integers(0, g.n, 500), dtype=torch.int32, device="cuda")
    opts = {lp.LP_OPT_WARP_MAX_WEDGES: 1, lp.LP_OPT_MED_MAX_WEDGES: 1,
            lp.LP_OPT_CTA_MAX_WEDGES: 257, lp.LP_OPT_SPLIT_LOGCAP: 6}
    saved = {o: lp.lp_get_option(o) for o in opts}
    try:
        for o, v in opts.items():
            lp.lp_set_option(o, v)
        with lp.Graph.from_csr(g) as G:
            for measure, cap, k in (("JC", None, 10), ("AA", 64, 8)):
                stats = check_static(lp, torch, G, measure, cap, k, src)
                assert stats["splits"] > 0, (measure, stats)
    finally:
        for o, v in saved.items():
            lp.lp_set_option(o, v)


def test_static_entry_point_rejects_oversized_requests(env):
    lp, torch = env
    g = L.gnp(40, 0.2, 3)
    with lp.Graph.from_csr(g) as G:
        n = 1 << 21  # above the 2^20 source limit of the fixed array
        src = torch.zeros((n,), dtype=torch.int32, device="cuda")
        out = torch.zeros((16,), dtype=torch.uint8, device="cuda")
        cnt = torch.zeros((1,), dtype=torch.int32, device="cuda")
        with pytest.raises(lp.LPError) as e:
            lp.lp_predict_sources_static(G.handle, "JC", src, n, 4, None, 0.0, out, cnt)
        assert e.value.status == lp.LP_EINVAL
