"""Source sharding of the global mode (paper_2401_11415_gb300.shard).

Sources are independent (Section 4.1.7), so the best k of the union of the
best-k lists of a partition of the sources into ranges is the unsharded best
k.  CPU tests check the range split, the gather and the exchange with the
oracle standing in for each range's device call and for the merge,
sequentially and as two gloo ranks (JC and RA); the GPU test merges
lp_predict_range shards with the library's exact merge (lp_merge_links) and
compares with one lp_predict call byte for byte, AA and RA included.
"""
import os
import socket

import numpy as np
import pytest

import lp_inputs as L
import oracle
from paper_2401_11415_gb300 import LINK_DTYPE, shard

COUNT = set(oracle.COUNT_MEASURES)


def oracle_range(g):
    """A range's best k from the oracle's per-source lists (c > a only)."""
    def run(measure, cap, k, begin, end, threshold=0.0):
        src = np.arange(begin, end, dtype=np.int32)
        if src.size == 0:
            return np.zeros(0, dtype=LINK_DTYPE)
        rows, cnt = oracle.predict_sources(g.n, g.off, g.idx, measure, src, g.n, cap, threshold)
        picks = []
        for i, a in enumerate(src.tolist()):
            for x in rows[i, : cnt[i]]:
                if int(x["v"]) > a:
                    picks.append((a, x))
        if measure in COUNT:
            from fractions import Fraction
            picks.sort(key=lambda t: (-Fraction(int(t[1]["num"]), int(t[1]["den"])), t[0],
                                      int(t[1]["v"])))
        else:
            picks.sort(key=lambda t: (-float(t[1]["value"]), t[0], int(t[1]["v"])))
        picks = picks[:k]
        out = np.zeros(len(picks), dtype=LINK_DTYPE)
        for j, (a, x) in enumerate(picks):
            out[j] = (a, int(x["v"]), np.float32(x["value"]), int(x["cn"]))
        return out
    return run


def test_shard_bounds_partition_and_balance():
    g = L.chung_lu(3000, 10.0, 2.2, dmax=300, seed=5)
    for ns in (1, 2, 3, 7):
        for cap in (None, 16):
            b = shard.shard_bounds(g.off, g.idx, ns, cap)
            assert b[0] == 0 and b[-1] == g.n and len(b) == ns + 1
            assert all(x <= y for x, y in zip(b, b[1:]))
            deg = np.diff(g.off)
            db = deg[g.idx]
            if cap is not None:
                db = np.where(db <= cap, db, 0)
            per = np.add.reduceat(np.concatenate([db, [0]]), g.off[:-1]) * (deg > 0)
            work = [int(per[b[i]:b[i + 1]].sum()) for i in range(ns)]
            assert max(work) <= sum(work) / ns + per.max()


def oracle_merge(g, measure, cap):
    """A test-side merge (the library's needs a GPU): the best k of the union
    of the parts by the oracle's exact key of each pair."""
    from fractions import Fraction

    def merge(parts, k):
        allp = shard.gather_parts(parts)
        keyed = []
        for x in allp:
            r, adj = oracle.pair(g.n, g.off, g.idx, measure, int(x["u"]), int(x["v"]), cap)
            assert not adj
            key = Fraction(int(r["num"]), int(r["den"])) if measure in COUNT else float(r["value"])
            keyed.append((-key, int(x["u"]), int(x["v"]), x))
        keyed.sort(key=lambda t: t[:3])
        out = np.zeros(min(k, len(keyed)), dtype=LINK_DTYPE)
        for j, t in enumerate(keyed[:k]):
            out[j] = t[3]
        return out
    return merge


def check_against_oracle(got, exp, measure, g, cap):
    assert len(got) == len(exp)
    if measure in COUNT:
        assert np.array_equal(got["u"], exp["u"]) and np.array_equal(got["v"], exp["v"])
        assert np.array_equal(got["cn"], exp["cn"])
    else:
        from parity import compare_global
        compare_global(got, exp, measure, g, cap)


@pytest.mark.parametrize("measure,cap", [("JC", None), ("CN", 8), ("SC", None), ("RA", 8),
                                         ("AA", None)])
def test_sharded_merge_equals_unsharded(measure, cap):
    g = L.chung_lu(400, 8.0, 2.1, dmax=60, seed=9)
    k = 300
    exp = oracle.predict(g.n, g.off, g.idx, measure, cap, k=k)
    for ns in (2, 5):
        b = shard.shard_bounds(g.off, g.idx, ns, cap)
        got = shard.predict_sharded(oracle_range(g), oracle_merge(g, measure, cap), b, measure,
                                    cap, k)
        check_against_oracle(got, exp, measure, g, cap)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir, measure):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = L.chung_lu(400, 8.0, 2.1, dmax=60, seed=9)
        b = shard.shard_bounds(g.off, g.idx, world, None)
        got = shard.predict_distributed(oracle_range(g), oracle_merge(g, measure, None), b,
                                        measure, None, 300)
        np.save(os.path.join(outdir, f"rank{rank}.npy"), got)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("measure", ["JC", "RA"])
def test_two_gloo_ranks_merge_equals_unsharded(tmp_path, measure):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path), measure), nprocs=2, join=True)
    g = L.chung_lu(400, 8.0, 2.1, dmax=60, seed=9)
    exp = oracle.predict(g.n, g.off, g.idx, measure, None, k=300)
    got0 = np.load(tmp_path / "rank0.npy")
    got1 = np.load(tmp_path / "rank1.npy")
    assert got0.tobytes() == got1.tobytes()  # every rank holds the same merged list
    check_against_oracle(got0, exp, measure, g, None)


@pytest.mark.gpu
@pytest.mark.parametrize("measure", ["JC", "RA", "AA", "SC"])
def test_gpu_range_shards_merge_to_predict(measure):
    """lp_predict_range over 2 and 4 balanced ranges, merged by lp_merge_links,
    must be the lp_predict list byte for byte (AA and RA too: the merge orders
    them by the fixed-point sums the selection uses)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_11415_gb300 import _build
    _build.build()
    import paper_2401_11415_gb300 as lp
    for g, cap in ((L.cfg_chung_lu_2k(), None), (L.rmat(16, 16, seed=3), 256)):
        k = 5000
        with lp.Graph.from_csr(g) as G:
            whole = G.predict(measure, cap, k)
            for ns in (2, 4):
                b = shard.shard_bounds(g.off, g.idx, ns, cap)
                got = shard.predict_sharded(G.predict_range, shard.library_merge(G, measure, cap),
                                            b, measure, cap, k)
                assert got.tobytes() == whole.tobytes(), (measure, ns)
            # k = 0 keeps every link; a merge of one whole list is itself
            assert G.merge(measure, cap, whole[::-1].copy(), 0).tobytes() == whole.tobytes()
            bad = whole[:3].copy()
            bad["u"][0], bad["v"][0] = bad["v"][0], bad["u"][0]  # u > v
            with pytest.raises(lp.LPError) as e:
                G.merge(measure, cap, bad, 10)
            assert e.value.status == lp.LP_EINVAL
            with pytest.raises(lp.LPError) as e:
                G.predict_range(measure, cap, 10, 5, 3)
            assert e.value.status == lp.LP_EINVAL
