"""The evaluation harness (paper_2401_11415_gb300.evaluate): held-out-edge
precision, recall and F1 (Eq. 10-12) and the hub-limit sweep (Section 4.4).

CPU tests pin ``quality`` to the definitions (set arithmetic written out here)
and to special cases; the GPU test runs the sweep on the 2,000-vertex
Chung-Lu split and checks every row's F1 against the oracle's predictions.
"""
import numpy as np
import pytest

import lp_inputs as L
import oracle
from paper_2401_11415_gb300 import evaluate


def _sets(pu, pv, hu, hv):
    p = {(min(a, b), max(a, b)) for a, b in zip(pu.tolist(), pv.tolist())}
    h = {(min(a, b), max(a, b)) for a, b in zip(hu.tolist(), hv.tolist())}
    return p, h


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_quality_matches_definitions(seed):
    rng = np.random.default_rng(seed)
    n = 60
    pu, pv = rng.integers(0, n, 400), rng.integers(0, n, 400)
    keep = pu != pv
    pu, pv = pu[keep], pv[keep]
    hu, hv = rng.integers(0, n, 300), rng.integers(0, n, 300)
    keep = hu != hv
    hu, hv = hu[keep], hv[keep]
    q = evaluate.quality(pu, pv, hu, hv)
    p, h = _sets(pu, pv, hu, hv)
    hits = len(p & h)
    assert q["hits"] == hits
    assert q["precision"] == pytest.approx(hits / len(p))
    assert q["recall"] == pytest.approx(hits / len(h))
    pr, rc = hits / len(p), hits / len(h)
    assert q["f1"] == pytest.approx(2 * pr * rc / (pr + rc))
    o = oracle.quality(pu, pv, hu, hv)
    assert o["hits"] == q["hits"] and o["f1"] == pytest.approx(q["f1"])


def test_quality_special_cases():
    hu = np.array([0, 2, 4]), np.array([1, 3, 5])
    # P = E^U (reversed orientation): everything right
    q = evaluate.quality(hu[1], hu[0], hu[0], hu[1])
    assert q == {"hits": 3, "precision": 1.0, "recall": 1.0, "f1": 1.0}
    # nothing predicted
    q = evaluate.quality(np.array([], int), np.array([], int), hu[0], hu[1])
    assert q["precision"] == 0.0 and q["recall"] == 0.0 and q["f1"] == 0.0
    # |P| = |E^U|: precision equals recall, so F1 equals both
    q = evaluate.quality(np.array([0, 2, 7]), np.array([1, 9, 8]), hu[0], hu[1])
    assert q["precision"] == q["recall"] == q["f1"] == pytest.approx(1 / 3)


@pytest.mark.gpu
def test_cap_sweep_matches_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_11415_gb300 import _build
    _build.build()
    split = L.holdout(L.cfg_chung_lu_2k(), 0.1, seed=43)
    g = split.observed
    k = len(split.hu)
    rows = evaluate.cap_sweep(split, ("JC", "RA"), (4, 64, None), repeats=1)
    assert len(rows) == 6
    for r in rows:
        exp = oracle.predict(g.n, g.off, g.idx, r["measure"], r["cap"], k=k)
        qo = oracle.quality(exp["u"], exp["v"], split.hu, split.hv)
        if r["measure"] == "JC":   # identical link sets
            assert r["hits"] == qo["hits"] and r["f1"] == pytest.approx(qo["f1"])
        else:                      # RA: sets may differ only at the cutoff
            assert abs(r["f1"] - qo["f1"]) <= 2 / k
        assert r["ms"] > 0
        assert r["speedup"] is not None
    ibase = [r for r in rows if r["cap"] is None]
    assert all(r["speedup"] == pytest.approx(1.0) for r in ibase)
    assert "| JC | 4 |" in evaluate.table(rows)
