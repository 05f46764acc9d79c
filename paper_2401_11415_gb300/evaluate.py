"""Evaluation harness: held-out-edge quality and the hub-limit sweep.

The predicted links of a call are compared with the edges held out of the
graph (Section 5.1.4): precision |P ∩ E^U| / |P| (Eq. 10), recall
|P ∩ E^U| / |E^U| (Eq. 11) and their harmonic mean F1 (Eq. 12), pairs taken
unordered.  ``cap_sweep`` repeats the study of Section 4.4 on a split: for
every measure and hub limit L_H (None = IBase) it predicts N_P = |E^U| links
with the CUDA library, times the call on the device and reports F1 and the
speedup over IBase.

Command line (prints a markdown table)::

    python -m paper_2401_11415_gb300.evaluate --graph rmat --scale 20 \\
        --measures JC RA --caps 4 32 256 1024 none
"""
from __future__ import annotations

import argparse
import time

import numpy as np


def _pair_keys(u, v) -> np.ndarray:
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    return (lo << 32) | hi


def quality(pred_u, pred_v, held_u, held_v) -> dict:
    """Precision (Eq. 10), recall (Eq. 11) and F1 (Eq. 12) of the predicted
    pairs against the held-out edges, both as sets of unordered pairs."""
    p = np.unique(_pair_keys(pred_u, pred_v))
    h = np.unique(_pair_keys(held_u, held_v))
    hits = int(np.isin(p, h, assume_unique=True).sum())
    precision = hits / p.size if p.size else 0.0
    recall = hits / h.size if h.size else 0.0
    f1 = 2 * precision * recall / (precision + recall) if hits else 0.0
    return {"hits": hits, "precision": precision, "recall": recall, "f1": f1}


def cap_sweep(split, measures=("JC", "RA"), caps=(4, 32, 256, 1024, None), n_p=None,
              repeats=1) -> list[dict]:
    """One row per (measure, hub limit): device time of the predict call (the
    best of `repeats`), links returned, precision, recall, F1 and the speedup
    over the IBase row of the same measure (when IBase is among `caps`)."""
    import paper_2401_11415_gb300 as lp

    g = split.observed
    k = len(split.hu) if n_p is None else int(n_p)
    rows = []
    lp.lp_set_timing(True)
    try:
        with lp.Graph.from_csr(g) as G:
            for m in measures:
                base = None
                mrows = []
                for cap in caps:
                    best = None
                    for _ in range(max(1, repeats)):
                        t0 = time.perf_counter()
                        links = G.predict(m, cap, k)
                        wall = (time.perf_counter() - t0) * 1e3
                        ms = float(lp.lp_last_stats()["ms_total"]) or wall
                        best = ms if best is None else min(best, ms)
                    q = quality(links["u"], links["v"], split.hu, split.hv)
                    row = {"measure": m, "cap": cap, "ms": best, "links": int(len(links)), **q}
                    if cap is None:
                        base = best
                    mrows.append(row)
                for row in mrows:
                    row["speedup"] = (base / row["ms"]) if base and row["ms"] > 0 else None
                rows.extend(mrows)
    finally:
        lp.lp_set_timing(False)
    return rows


def table(rows: list[dict]) -> str:
    out = ["| measure | L_H | ms | links | precision | recall | F1 | speedup vs IBase |",
           "|---|---:|---:|---:|---:|---:|---:|---:|"]
    for r in rows:
        cap = "none" if r["cap"] is None else str(r["cap"])
        sp = "" if r["speedup"] is None else f"{r['speedup']:.1f}x"
        out.append(f"| {r['measure']} | {cap} | {r['ms']:.2f} | {r['links']} | {r['precision']:.4f} "
                   f"| {r['recall']:.4f} | {r['f1']:.4f} | {sp} |")
    return "\n".join(out)


def main(argv=None) -> None:
    import lp_inputs as L

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--graph", default="rmat", choices=["rmat", "chunglu", "chunglu2k"])
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale")
    ap.add_argument("--n", type=int, default=1 << 20, help="Chung-Lu vertices")
    ap.add_argument("--holdout", type=float, default=0.1)
    ap.add_argument("--measures", nargs="+", default=["JC", "RA"])
    ap.add_argument("--caps", nargs="+", default=["4", "32", "256", "1024", "none"])
    ap.add_argument("--repeats", type=int, default=2)
    a = ap.parse_args(argv)
    if a.graph == "rmat":
        g = L.rmat(a.scale, 16, seed=1)
    elif a.graph == "chunglu":
        g = L.chung_lu(a.n, 16.0, 2.3, dmax=a.n ** 0.5 * 10, seed=7)
    else:
        g = L.cfg_chung_lu_2k()
    split = L.holdout(g, a.holdout, seed=43)
    caps = [None if c.lower() in ("none", "inf") else int(c) for c in a.caps]
    rows = cap_sweep(split, a.measures, caps, repeats=a.repeats)
    obs = split.observed
    print(f"graph {g.name}: n={g.n}, observed edges={len(obs.idx) // 2}, held out={len(split.hu)}")
    print(table(rows))


if __name__ == "__main__":
    main()
