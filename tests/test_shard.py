"""Source sharding of the global mode (paper_2401_11415_gb300.shard).

Sources are independent (Section 4.1.7), so the best k of the union of the
best-k lists of a partition of the sources into ranges is the unsharded best
k.  CPU tests check the range split and the merge with the oracle standing in
for each range's device call, sequentially and as two gloo ranks; the GPU test
merges lp_predict_range shards and compares with one lp_predict call.
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


@pytest.mark.parametrize("measure,cap", [("JC", None), ("CN", 8), ("SC", None), ("RA", 8)])
def test_sharded_merge_equals_unsharded(measure, cap):
    g = L.chung_lu(400, 8.0, 2.1, dmax=60, seed=9)
    k = 300
    deg = np.diff(g.off)
    exp = oracle.predict(g.n, g.off, g.idx, measure, cap, k=k)
    for ns in (2, 5):
        b = shard.shard_bounds(g.off, g.idx, ns, cap)
        got = shard.predict_sharded(oracle_range(g), g.n, b, measure, cap, k, deg)
        assert len(got) == len(exp)
        if measure in COUNT:
            assert np.array_equal(got["u"], exp["u"]) and np.array_equal(got["v"], exp["v"])
            assert np.array_equal(got["cn"], exp["cn"])
        else:
            assert np.allclose(got["score"], exp["value"], rtol=1e-6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = L.chung_lu(400, 8.0, 2.1, dmax=60, seed=9)
        b = shard.shard_bounds(g.off, g.idx, world, None)
        got = shard.predict_distributed(oracle_range(g), b, "JC", None, 300, np.diff(g.off))
        np.save(os.path.join(outdir, f"rank{rank}.npy"), got)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_merge_equals_unsharded(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    g = L.chung_lu(400, 8.0, 2.1, dmax=60, seed=9)
    exp = oracle.predict(g.n, g.off, g.idx, "JC", None, k=300)
    for r in range(2):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert np.array_equal(got["u"], exp["u"]) and np.array_equal(got["v"], exp["v"])
        assert np.array_equal(got["cn"], exp["cn"])


@pytest.mark.gpu
@pytest.mark.parametrize("measure", ["JC", "RA"])
def test_gpu_range_shards_merge_to_predict(measure):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_11415_gb300 import _build
    _build.build()
    import paper_2401_11415_gb300 as lp
    for g, cap in ((L.cfg_chung_lu_2k(), None), (L.rmat(16, 16, seed=3), 256)):
        k = 5000
        deg = np.diff(g.off)
        with lp.Graph.from_csr(g) as G:
            whole = G.predict(measure, cap, k)
            for ns in (2, 4):
                b = shard.shard_bounds(g.off, g.idx, ns, cap)
                got = shard.predict_sharded(G.predict_range, g.n, b, measure, cap, k, deg)
                assert len(got) == len(whole)
                if measure == "JC":
                    assert got.tobytes() == whole.tobytes()
                else:  # order within equal FP32 scores may differ; sets only at the cutoff
                    assert np.allclose(got["score"], whole["score"], rtol=1e-6)
                    diff = set(zip(got["u"].tolist(), got["v"].tolist())) ^ \
                        set(zip(whole["u"].tolist(), whole["v"].tolist()))
                    cut = float(whole["score"][-1])
                    for a, c in diff:
                        r, _ = oracle.pair(g.n, g.off, g.idx, measure, a, c, cap)
                        assert abs(float(r["value"]) - cut) <= 1e-6 * cut
            with pytest.raises(lp.LPError) as e:
                G.predict_range(measure, cap, 10, 5, 3)
            assert e.value.status == lp.LP_EINVAL
