"""lp_serve_*: continuous batching of per-source queries (needs a GPU).

Mode 0 (the default) runs batches from host worker threads; mode 1 serves
requests with a resident kernel that claims one source at a time from a ring
in mapped host memory.  Both modes are checked the same way.

Each served result must equal lp_predict_sources on the same sources alone,
whatever else is in the batch, and a quarter of the served requests (all four
kinds of query) are checked row by row against the CPU oracle; requests of uneven sizes and different
(measure, hub limit, k) arrive from several threads.  Bounded waits, a full
queue and bad requests are made on the host side (a paused server), never by
stalling the GPU.
"""
import threading

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
def graph():
    return L.chung_lu(6000, 12.0, 2.1, dmax=1200, seed=31)


KINDS = [("JC", 64, 10), ("RA", None, 5), ("CN", 16, 8), ("AA", 256, 10)]


@pytest.mark.parametrize("mode", [0, 1])
def test_served_equals_alone(lp, graph, mode):
    g = graph
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(160):
        n = int(np.exp(rng.uniform(0, np.log(400))))
        reqs.append((rng.integers(0, g.n, n).astype(np.int32), KINDS[i % len(KINDS)]))
    with lp.Graph.from_csr(g) as G:
        expect = [G.predict_sources(kind[0], src, kind[2], kind[1]) for src, kind in reqs]
        with lp.Server(G, slots=3, max_batch_sources=2000, max_k=16, mode=mode) as S:
            ids = [None] * len(reqs)

            def submit(lo, hi):
                for i in range(lo, hi):
                    src, (m, cap, k) = reqs[i]
                    ids[i] = S.submit(src, m, k, cap)

            th = [threading.Thread(target=submit, args=(j * 40, (j + 1) * 40)) for j in range(4)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            got = [S.wait(ids[i], 60_000_000) for i in range(len(reqs))]
            st = S.stats()
        assert st["submitted"] == st["completed"] == len(reqs)
        assert st["max_batch_requests"] > 1        # requests were merged into batches
        for (gl, gc), (el, ec) in zip(got, expect):
            assert np.array_equal(gc, ec)
            assert gl.tobytes() == el.tobytes()
        # the served rows themselves against the oracle: a quarter of the
        # requests (j % 16 in {0, 5, 10, 15} covers all four kinds of query)
        for j in range(len(reqs)):
            if j % 16 not in (0, 5, 10, 15):
                continue
            src, (m, cap, k) = reqs[j]
            ol, oc = oracle.predict_sources(g.n, g.off, g.idx, m, src, k, cap)
            compare_sources(got[j][0], got[j][1], ol, oc, m, g, src, cap)


@pytest.mark.parametrize("mode", [0, 1])
def test_paused_timeout_full_queue_and_errors(lp, graph, mode):
    g = graph
    src = np.arange(50, dtype=np.int32)
    with lp.Graph.from_csr(g) as G:
        with lp.Server(G, slots=1, max_pending=3, max_batch_sources=100, paused=True,
                       mode=mode) as S:
            a = S.submit(src, "JC", 10, 64)
            b = S.submit(src[:7], "JC", 10, 64)
            c = S.submit(src[:3], "RA", 5, None)
            with pytest.raises(lp.LPError) as e:
                S.submit(src, "JC", 10, 64)                 # fourth queued request
            assert e.value.status == lp.LP_EBUSY
            with pytest.raises(lp.LPError) as e:
                S.wait(a, 2000)                              # paused: cannot finish
            assert e.value.status == lp.LP_ETIMEOUT
            assert not S.poll(a)
            for bad in (dict(sources=np.array([g.n], np.int32), measure="JC", k=5),
                        dict(sources=src, measure="JC", k=17),
                        dict(sources=np.arange(101, dtype=np.int32), measure="JC", k=5)):
                with pytest.raises(lp.LPError) as e:
                    S.submit(bad["sources"], bad["measure"], bad["k"])
                assert e.value.status == lp.LP_EINVAL
            S.resume()
            ra = S.wait(a, 60_000_000)
            rb = S.wait(b, 60_000_000)
            rc = S.wait(c, 60_000_000)
            with pytest.raises(lp.LPError) as e:
                S.wait(a, 1000)                              # already released
            assert e.value.status == lp.LP_EINVAL
            assert S.stats()["max_batch_requests"] >= 2      # a and b shared a batch
        ea = G.predict_sources("JC", src, 10, 64)
        assert ra[0].tobytes() == ea[0].tobytes()
        eb = G.predict_sources("JC", src[:7], 10, 64)
        assert rb[0].tobytes() == eb[0].tobytes()
        ec = G.predict_sources("RA", src[:3], 5, None)
        assert rc[0].tobytes() == ec[0].tobytes()


@pytest.mark.parametrize("mode", [0, 1])
def test_close_finishes_queued_requests(lp, graph, mode):
    g = graph
    with lp.Graph.from_csr(g) as G:
        S = lp.Server(G, slots=2, paused=True, mode=mode)
        for i in range(10):
            S.submit(np.arange(i * 10, i * 10 + 10, dtype=np.int32), "CN", 4)
        S.close()                                            # resumes, drains, frees


def test_resident_kernel_leaves_when_idle_and_is_relaunched(lp, graph):
    """The resident kernel's wait for work is bounded: with idle_polls = 20
    (about 0.1 ms) it leaves between requests, and the next submitted request
    launches it again; every result still equals the plain call."""
    import time
    g = graph
    rng = np.random.default_rng(3)
    with lp.Graph.from_csr(g) as G:
        with lp.Server(G, slots=1, max_batch_sources=500, mode=1, idle_polls=20) as S:
            for i in range(4):
                src = rng.integers(0, g.n, 50 + 40 * i).astype(np.int32)
                rid = S.submit(src, "RA", 10, 64)
                got = S.wait(rid, 60_000_000)
                exp = G.predict_sources("RA", src, 10, 64)
                assert got[0].tobytes() == exp[0].tobytes()
                assert np.array_equal(got[1], exp[1])
                time.sleep(0.05)  # far longer than the kernel waits for work
            st = S.stats()
        assert st["kernel_launches"] >= 4 and st["completed"] == 4


def test_resident_kernel_admits_by_memory(lp, graph):
    """Room for 64 sources in flight (max_batch_sources 64, one slot): requests
    of 40 sources are admitted one at a time as memory frees up, all finish
    and equal the plain call."""
    g = graph
    rng = np.random.default_rng(4)
    reqs = [rng.integers(0, g.n, 40).astype(np.int32) for _ in range(12)]
    with lp.Graph.from_csr(g) as G:
        with lp.Server(G, slots=1, max_batch_sources=64, max_k=8, mode=1) as S:
            ids = [S.submit(r, "JC", 8, 64) for r in reqs]
            got = [S.wait(i, 60_000_000) for i in ids]
            st = S.stats()
        assert st["max_batch_requests"] == 1  # two never fit at once
        for r, (gl, gc) in zip(reqs, got):
            el, ec = G.predict_sources("JC", r, 8, 64)
            assert np.array_equal(gc, ec) and gl.tobytes() == el.tobytes()


@pytest.mark.parametrize("measure,cap", [("RA", None), ("JC", 64)])
def test_resident_kernel_defers_large_sources(lp, graph, measure, cap):
    """Sources with more wedges than defer_wedges (here 200, so many of them)
    are left by the resident kernel to the tiered per-source pipeline when the
    request is collected; the rows are the plain call's either way."""
    g = graph
    rng = np.random.default_rng(9)
    reqs = [rng.integers(0, g.n, m).astype(np.int32) for m in (1, 17, 300, 900)]
    with lp.Graph.from_csr(g) as G:
        with lp.Server(G, slots=2, max_batch_sources=1000, max_k=10, mode=1,
                       defer_wedges=200) as S:
            ids = [S.submit(r, measure, 10, cap) for r in reqs]
            got = [S.wait(i, 60_000_000) for i in ids]
            st = S.stats()
        assert 0 < st["deferred_sources"] < sum(len(r) for r in reqs)
        for r, (gl, gc) in zip(reqs, got):
            el, ec = G.predict_sources(measure, r, 10, cap)
            assert np.array_equal(gc, ec) and gl.tobytes() == el.tobytes()
