"""The per-source entry point that allocates nothing (lp_predict_sources_static).

Some callers of this library cannot allocate device memory while they serve a
request: they run under a memory pool they do not own, or on a path where an
allocation, and the device synchronisation it can cause, is not allowed.  For
them the library offers a variant of the per-source query whose working memory
is one fixed array in device global memory.  This test calls it through the
C ABI twice in a row and checks both results against the ordinary entry point
(lp_predict_sources_dev) within the parity tolerance used elsewhere: count
measures exactly, AA and RA within 1e-6 relative.  The second call shows that
what the shared array keeps from the first call does not leak into the next.
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


def run(lp, torch, fn, G, measure, src, k, cap):
    n = src.numel()
    out = torch.zeros((n * k * 16,), dtype=torch.uint8, device="cuda")
    cnt = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    fn(G.handle, measure, src, n, k, cap, 0.0, out, cnt)
    torch.cuda.synchronize()
    links = out.cpu().numpy().view(lp.LINK_DTYPE).reshape(n, k)
    return links, cnt.cpu().numpy()


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


def test_static_entry_point_matches_dev(env):
    lp, torch = env
    # hubs make some sources large enough to be split into several items
    g = L.chung_lu(4000, 12.0, 2.05, dmax=1500, seed=21)
    rng = np.random.default_rng(5)
    src = torch.tensor(rng.integers(0, g.n, 700), dtype=torch.int32, device="cuda")
    with lp.Graph.from_csr(g) as G:
        for measure, cap, k in (("JC", None, 10), ("RA", 64, 16), ("CN", None, 5)):
            ref = run(lp, torch, lp.lp_predict_sources_dev, G, measure, src, k, cap)
            assert ref[1].sum() > 0
            first = run(lp, torch, lp.lp_predict_sources_static, G, measure, src, k, cap)
            second = run(lp, torch, lp.lp_predict_sources_static, G, measure, src, k, cap)
            same(first, ref, measure)
            same(second, ref, measure)


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
