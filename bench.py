#!/usr/bin/env python3
"""Benchmark: predicted edges/s of DLH link prediction on one GB300.

Workload (one step): the R-MAT scale-20 web-like graph (edge factor 16,
(a, b, c) = (0.57, 0.19, 0.19), symmetrised, deduplicated, self-loops removed,
ids permuted; 10% of the edges held out), predicted in global mode with
N_P = |E^U| for the DLH hub-limit sweep {16, 64, 256, 1024, none (IBase)}
with Jaccard and Resource Allocation: ten lp_predict calls.

value: sum of |P| over the step / step time, graph resident on the device,
       outputs written to device memory (lp_predict_dev), CUDA events on the
       library's stream.
e2e:   the same step through the host-buffer API: lp_graph_create from the
       host CSR (pinned), ten lp_predict calls into host buffers,
       lp_graph_destroy.
roofline: the dominant scan kernel, algorithmic bytes (Gamma_a ids, degree of
       each b, the b offset of kept arcs, 4 bytes per scanned wedge) / its
       event-timed duration.
rmat24_dlh256: the same measurements for R-MAT scale 24 (16,777,216 vertices,
       10% held out), DLH hub limit 256, JC and RA, N_P = |E^U|.
cpu_baseline: the CPU oracle on all host cores over the ten calls of the
       step, run once outside the timed region (about 4 minutes on 16 cores;
       --cpu-baseline sample times only the cap-16 pair), plus the cap-16 pair
       on one thread.

--impl reference runs the CPU oracle (the only reference this method has)
on a bounded sample of the same workload (the cap-16 JC and RA calls per
step); our line reports its own edges/s on that sample too (matched_sample).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CAPS = [16, 64, 256, 1024, None]
MEASURES = ["JC", "RA"]
METRIC = "predicted edges/s (DLH, JC & RA)"
WORKLOAD = ("R-MAT scale 20 (1,048,576 vertices, edge factor 16, a,b,c=0.57,0.19,0.19), "
            "10% held out; global top-|E^U| for DLH caps {16,64,256,1024,inf} x {JC,RA}")
SAMPLE_CAPS = [(16, "JC"), (16, "RA")]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources each measured kernel and its launches are built from
KERNEL_SOURCES = {
    "k_scan_big": ["lp_internal.cuh", "lp_scan_dev.cuh", "lp_scan.cu", "lp_api.cu"],
    "k_exp_tiles+k_exp_count": ["lp_internal.cuh", "lp_scan_dev.cuh", "lp_scan.cu",
                                "lp_expand.cu", "lp_api.cu"],
}


def kernel_hash(kernel: str = "k_scan_big") -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2401_11415_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, KERNEL_SOURCES["k_exp_tiles+k_exp_count"]):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources: the measured DRAM bytes per algorithmic byte
    of the captured launches (every launch of the kernel in one call) times
    this run's algorithmic bytes per launch.  (None, None) otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None, None
    ent = rec.get(kernel)
    if not ent or ent.get("kernel_hash") != kernel_hash(kernel):
        return None, None
    ratio = ent.get("dram_bytes_per_alg_byte")
    if ratio is None:
        return None, None
    return int(ratio * alg_bytes_per_launch), (
        f"{ratio:.4f} DRAM bytes per algorithmic byte, measured by ncu on {ent.get('workload')}")


_ARGS = None


def make_workload():
    import lp_inputs as L
    scale = _ARGS.scale if _ARGS is not None else 20
    g = L.rmat(scale, 16, seed=1)
    split = L.holdout(g, 0.1, seed=43)
    return split


def step_calls():
    calls = [(m, c) for c in CAPS for m in MEASURES]
    if _ARGS is not None and _ARGS.only:
        want = set(_ARGS.only.split(","))
        calls = [(m, c) for m, c in calls if f"{m}@{'inf' if c is None else c}" in want]
    return calls


# ------------------------------------------------------------- our arm ----

def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    import paper_2401_11415_gb300 as lp
    from paper_2401_11415_gb300 import _build
    _build.build()

    if args.select_buffer:
        lp.lp_set_option(lp.LP_OPT_SELECT_BUFFER, args.select_buffer)
    split = make_workload()
    obs = split.observed
    k = len(split.hu)
    G = lp.Graph.from_csr(obs)
    stream = torch.cuda.ExternalStream(G.stream)
    d_out = torch.empty((k * 16,), dtype=torch.uint8, device="cuda")
    calls = step_calls()

    def one_step(collect=None):
        tot = 0
        for m, c in calls:
            n = lp.lp_predict_dev(G.handle, m, c, k, 0.0, d_out, k)
            tot += n
            if collect is not None:
                collect.append(lp.lp_last_stats())
        return tot

    for _ in range(args.warmup):
        one_step()
    dist_barrier(world)
    torch.cuda.synchronize()
    lp.lp_set_timing(True)
    stats = []
    with ClockSampler(local_rank) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        total = 0
        for _ in range(args.steps):
            total += one_step(stats)
        ev1.record(stream)
        torch.cuda.synchronize()
    lp.lp_set_timing(False)
    ms = ev0.elapsed_time(ev1)
    ms_max = dist_max(ms, world)
    dist_barrier(world)

    # e2e through the host-buffer API (graph upload + host outputs)
    e2e = None if args.no_e2e else run_e2e(lp, torch, obs, k, max(1, min(args.steps, 3)))

    roof = roofline(stats)
    wedges = sum(s["wedges"] for s in stats)
    gpu_launches = sum(s["launches"] for s in stats)
    value = (total * world) / (ms_max / 1e3)
    per_cap = {}
    for (m, c), s in zip(calls * args.steps, stats):
        key = f"{m}@{'inf' if c is None else c}"
        per_cap[key] = per_cap.get(key, 0.0) + s["ms_total"]
    # our rate on the reference arm's sample (the cap-16 JC and RA calls)
    samp = [f"{m}@{c}" for c, m in SAMPLE_CAPS]
    samp_ms = sum(per_cap.get(x, 0.0) for x in samp) / args.steps
    samp_edges = k * len(samp)
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "edges/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32+u64 (exact integer counts; fixed-point AA/RA)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "edges_undirected": int(obs.edges),
                   "vertices": int(obs.n), "N_P": k, "calls_per_step": len(calls),
                   "l2": "no flush: graph arrays 0.6 GB > 129 MB L2, re-read every call",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "gpu_launches": int(gpu_launches),
        "roofline": roof,
        "wedges_per_s": round(wedges / (ms / 1e3), 1),
        "per_call_ms": {k_: round(v / args.steps, 3) for k_, v in per_cap.items()},
        "matched_sample": {"calls": samp, "value": round(samp_edges / (samp_ms / 1e3), 1)
                           if samp_ms > 0 else None, "unit": "edges/s",
                           "note": "device time of the calls the reference arm times per step"},
        "clocks": clk.summary(),
    }
    if args.scale != 20 or args.only:
        line["config"]["workload"] += f" [subset: scale {args.scale}, calls {args.only or 'all'}]"
    G.close()
    if not args.no_rmat24 and args.scale == 20 and not args.only and world == 1:
        line["rmat24_dlh256"] = run_rmat24(lp, torch, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(split, args.cpu_baseline)
    return line


TIER_KERNELS = ["k_scan_warp", "k_scan_cta", "k_scan_big", "k_exp_tiles+k_exp_count"]


def roofline(stats):
    """The dominant scan kernel (by summed device time): its algorithmic
    bytes per launch -- 4 B per Gamma_a id and per degree of b over the
    arcs of the sources binned to it, 4 B per kept arc (the b offset), 4 B
    per wedge -- over its average event-timed launch.  The expand-and-count
    tier is one unit here: its time is that of its arc, expand and count
    passes together, its launches the count-pass launches."""
    nt = len(stats[0]["tier_ms"]) if stats else 3
    tier_ms = [sum(s["tier_ms"][i] for s in stats) for i in range(nt)]
    tier_launch = [sum(s["tier_launches"][i] for s in stats) for i in range(nt)]
    dom = max(range(nt), key=lambda i: tier_ms[i])
    name = TIER_KERNELS[dom]
    alg_bytes = 0
    for s in stats:
        alg_bytes += (4 * s["tier_arcs"][dom] + 4 * s["tier_arcs"][dom] + 4 * s["tier_kept"][dom]
                      + 4 * s["tier_wedges"][dom])
    launches = max(1, tier_launch[dom])
    bytes_per_launch = alg_bytes / launches
    avg_ms = tier_ms[dom] / launches
    peak, peak_kind = peaks()
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    traffic, basis = traffic_record(name, bytes_per_launch)
    return {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "traffic": traffic, "traffic_basis": basis,
            "alg_bytes_per_launch": int(bytes_per_launch),
            "avg_launch_ms": round(avg_ms, 4), "launches": int(launches),
            "share_of_scan_ms": round(tier_ms[dom] / max(1e-9, sum(tier_ms)), 4)}


def run_rmat24(lp, torch, args):
    """R-MAT scale 24 (10% held out), DLH(256) JC and RA with N_P = |E^U|: a
    graph whose index array is far larger than the L2, where the
    expand-and-count tier runs.  Graph resident, outputs in device memory,
    CUDA events on the library's stream."""
    import lp_inputs as L
    t0 = time.perf_counter()
    split = L.holdout(L.cfg_rmat24(), 0.1, seed=43)
    t_gen = time.perf_counter() - t0
    obs = split.observed
    k = len(split.hu)
    G = lp.Graph.from_csr(obs)
    stream = torch.cuda.ExternalStream(G.stream)
    d_out = torch.empty((k * 16,), dtype=torch.uint8, device="cuda")
    calls = [("JC", 256), ("RA", 256)]
    for _ in range(args.r24_warmup):
        for m, c in calls:
            lp.lp_predict_dev(G.handle, m, c, k, 0.0, d_out, k)
    torch.cuda.synchronize()
    lp.lp_set_timing(True)
    stats, total, per = [], 0, {}
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.r24_steps):
            for m, c in calls:
                total += lp.lp_predict_dev(G.handle, m, c, k, 0.0, d_out, k)
                st = lp.lp_last_stats()
                stats.append(st)
                per[f"{m}@{c}"] = per.get(f"{m}@{c}", 0.0) + st["ms_total"]
        ev1.record(stream)
        torch.cuda.synchronize()
    lp.lp_set_timing(False)
    ms = ev0.elapsed_time(ev1)
    G.close()
    # whole-call algorithmic bytes of the survey's formula B_L (every wedge of
    # every source, 16 B per output link) over the call time
    b_l = sum(4 * (obs.n + 1) + 8 * obs.arcs + 4 * s["kept_arcs"] + 4 * s["wedges"] + 16 * k
              for s in stats)
    peak, peak_kind = peaks()
    path_gbs = b_l / (ms * 1e-3) / 1e9
    return {"workload": "R-MAT scale 24 (16,777,216 vertices, edge factor 16, "
                        "a,b,c=0.57,0.19,0.19), 10% held out; global top-|E^U| for DLH(256) "
                        "JC and RA",
            "edges_undirected": int(obs.edges), "N_P": k, "steps": args.r24_steps,
            "warmup": args.r24_warmup, "ms_per_step": round(ms / args.r24_steps, 3),
            "ms_per_call": {x: round(v / args.r24_steps, 3) for x, v in per.items()},
            "edges_per_s": round(total / (ms / 1e3), 1), "unit": "edges/s",
            "wedges_per_s": round(sum(s["wedges"] for s in stats) / (ms / 1e3), 1),
            "roofline": roofline(stats),
            "path_roofline": {"bytes": "B_L of every call (4(N+1) + 8A + 4 kept + 4 W + 16 |P|)",
                              "achieved": round(path_gbs, 1), "peak": peak, "unit": "GB/s",
                              "frac": round(path_gbs / peak, 4), "peak_source": peak_kind},
            "parity": "tests/test_gpu_fullsize.py::test_rmat24_global_sampled",
            "graph_generate_s": round(t_gen, 1), "clocks": clk.summary()}


def run_e2e(lp, torch, obs, k, steps):
    """Host-buffer path: create from pinned host CSR, predict into host
    buffers, destroy; timed per step on the host around synchronous calls."""
    off = torch.from_numpy(obs.off).pin_memory()
    idx = torch.from_numpy(obs.idx).pin_memory()
    out = torch.empty((k * 16,), dtype=torch.uint8).pin_memory()
    import ctypes
    cnt = ctypes.c_int64()
    calls = step_calls()
    lib = lp.lib()
    t_best = None
    total = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        h = ctypes.c_void_p()
        st = lib.lp_graph_create(obs.n, off.data_ptr(), idx.data_ptr(), 0, ctypes.byref(h))
        assert st == 0, lp.lp_last_error()
        for m, c in calls:
            st = lib.lp_predict(h, lp.MEASURES.index(m), -1 if c is None else c, k, 0.0,
                                out.data_ptr(), k, ctypes.byref(cnt))
            assert st == 0, lp.lp_last_error()
            total += cnt.value
        lib.lp_graph_destroy(h)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    return {"value": round(total / t, 1), "unit": "edges/s",
            "h2d_bytes_per_step": int(4 * (obs.n + 1) + 4 * obs.arcs),
            "d2h_bytes_per_step": int(16 * total / steps)}


def cpu_baseline(split, which="full"):
    """The oracle on all host cores, once: over the ten calls of the step
    ("full", the same work as the timed step) or the cap-16 pair ("sample");
    and the cap-16 pair on one thread."""
    import oracle
    obs = split.observed
    k = len(split.hu)
    cores = os.cpu_count() or 1
    t = 0.0
    tot = 0
    pairs = [(c, m) for c in CAPS for m in MEASURES] if which == "full" else SAMPLE_CAPS
    for c, m in pairs:
        t0 = time.perf_counter()
        r = oracle.predict(obs.n, obs.off, obs.idx, m, c, k=k, nthreads=cores)
        t += time.perf_counter() - t0
        tot += len(r)
    t1 = 0.0
    n1 = 0
    for c, m in SAMPLE_CAPS:
        t0 = time.perf_counter()
        n1 += len(oracle.predict(obs.n, obs.off, obs.idx, m, c, k=k, nthreads=1))
        t1 += time.perf_counter() - t0
    what = ("all ten calls of the step (DLH caps 16, 64, 256, 1024, none x JC, RA), full "
            "graph, once" if which == "full" else
            "the DLH cap-16 JC and RA calls of the step, full graph; caps 64-inf left out")
    return {"value": round(tot / t, 1), "unit": "edges/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{what} ({tot} predicted edges in {t:.1f} s)",
            "one_thread": {"value": round(n1 / t1, 1), "unit": "edges/s", "cores": 1,
                           "sample": f"the same calls on one thread ({n1} predicted edges in "
                                     f"{t1:.1f} s)"}}


# ------------------------------------------------------------ serving ----

def run_serve(args):
    """Per-source serving on R-MAT scale 24 (requests of 1-4096 sources, top-10
    DLH(256) RA, Poisson arrivals): one plain lp_predict_sources call per
    request in FIFO order versus lp_serve_* continuous batching."""
    import threading
    import torch
    import lp_inputs as L
    import paper_2401_11415_gb300 as lp
    from paper_2401_11415_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    scale = args.scale if args.scale != 20 else 24
    t0 = time.perf_counter()
    g = L.rmat(scale, 16, seed=1)
    t_gen = time.perf_counter() - t0
    rng = np.random.default_rng(11)
    live_v = np.nonzero(np.diff(g.off) > 0)[0].astype(np.int32)
    R = args.requests
    sizes = np.exp(rng.uniform(0, np.log(4096), R)).astype(np.int64).clip(1, 4096)
    reqs = [live_v[rng.integers(0, live_v.size, int(m))] for m in sizes]
    measure, cap, k = "RA", 256, 10
    t0 = time.perf_counter()
    G = lp.Graph.from_csr(g)
    t_create = time.perf_counter() - t0
    for r in reqs[:5]:
        G.predict_sources(measure, r, k, cap)
    # plain service times, serialised
    plain_res, svc = [], []
    for r in reqs:
        t = time.perf_counter()
        plain_res.append(G.predict_sources(measure, r, k, cap))
        svc.append(time.perf_counter() - t)
    svc = np.array(svc)
    mu = R / svc.sum()
    edges = int(sum(int(c.sum()) for _, c in plain_res))
    out = {"metric": "served per-source top-10 DLH(256) RA: p50/p99 latency and edges/s",
           "workload": f"R-MAT scale {scale} (n={g.n}, {g.edges} undirected edges), {R} requests "
                       "of 1-4096 sources (log-uniform), Poisson arrivals",
           "graph_generate_s": round(t_gen, 1), "graph_create_s": round(t_create, 2),
           "plain_capacity_req_per_s": round(mu, 1), "predicted_edges": edges, "loads": []}
    for rho in args.loads:
        lam = rho * mu
        arr = np.cumsum(rng.exponential(1.0 / lam, R))
        # plain: FIFO, one call per request, real time
        t_start = time.perf_counter()
        lat_p = np.zeros(R)
        for i, r in enumerate(reqs):
            now = time.perf_counter() - t_start
            if now < arr[i]:
                time.sleep(arr[i] - now)
            G.predict_sources(measure, r, k, cap)
            lat_p[i] = (time.perf_counter() - t_start) - arr[i]
        span_p = time.perf_counter() - t_start
        entry = {"load": rho, "arrival_req_per_s": round(lam, 1),
                 "plain": {"p50_ms": round(1e3 * float(np.percentile(lat_p, 50)), 2),
                           "p99_ms": round(1e3 * float(np.percentile(lat_p, 99)), 2),
                           "edges_per_s": round(edges / span_p, 1)}}
        for mode in (0, 1):
            entry["served" if mode == 0 else "served_resident_kernel"] = serve_once(
                lp, G, reqs, arr, plain_res, measure, k, cap, mode, args.slots, edges)
        out["loads"].append(entry)
    G.close()
    return out


def serve_once(lp, G, reqs, arr, plain_res, measure, k, cap, mode, slots, edges):
    """Submit every request at its arrival time to a server of the given mode
    (0: host batches, the default; 1: resident kernel), wait from several
    threads; latency is completion minus arrival."""
    import threading
    R = len(reqs)
    S = lp.Server(G, slots=slots, max_batch_sources=65536, max_k=16, mode=mode)
    ids = [None] * R
    lat_s = np.zeros(R)
    got = [None] * R
    ready = [threading.Event() for _ in range(R)]
    t_start = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            now = time.perf_counter() - t_start
            if now < arr[i]:
                time.sleep(arr[i] - now)
            ids[i] = S.submit(r, measure, k, cap)
            ready[i].set()

    def waiter(j, nw):
        for i in range(j, R, nw):
            ready[i].wait()
            got[i] = S.wait(ids[i], -1)
            lat_s[i] = (time.perf_counter() - t_start) - arr[i]

    nw = 8
    th = [threading.Thread(target=submitter)] + \
         [threading.Thread(target=waiter, args=(j, nw)) for j in range(nw)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    span_s = time.perf_counter() - t_start
    st = S.stats()
    S.close()
    same = all(got[i][0].tobytes() == plain_res[i][0].tobytes() and
               np.array_equal(got[i][1], plain_res[i][1]) for i in range(R))
    return {"p50_ms": round(1e3 * float(np.percentile(lat_s, 50)), 2),
            "p99_ms": round(1e3 * float(np.percentile(lat_s, 99)), 2),
            "edges_per_s": round(edges / span_s, 1),
            "batches": st["batches"], "max_batch_requests": st["max_batch_requests"],
            "kernel_launches": st["kernel_launches"],
            "identical_to_plain": bool(same)}


# ------------------------------------------------------- reference arm ----

def run_batch(args):
    """Batched multi-graph study: many Chung-Lu graphs (vertex counts
    log-uniform in [1k, 500k], mean degree 8-32, exponent 2.0-2.8, seeds
    1000 + i) packed into one lp_batch; per-source top-10 of every vertex for
    JC (hub limit 256) and AA (hub limit 32), each query recorded once and
    replayed, with autotuned binning; versus one plain lp_predict_sources_dev
    call per graph on the same GPU."""
    import torch
    import lp_inputs as L
    import paper_2401_11415_gb300 as lp
    from paper_2401_11415_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(4)
    t0 = time.perf_counter()
    graphs = []
    for i in range(args.graphs):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(500000))))
        deg = float(rng.uniform(8, 32))
        gamma = float(rng.uniform(2.0, 2.8))
        graphs.append(L.chung_lu(n, deg, gamma, dmax=8.0 * n ** 0.5, seed=1000 + i))
    t_gen = time.perf_counter() - t0
    k = 10
    queries = [("JC", 256), ("AA", 32)]
    t0 = time.perf_counter()
    B = lp.Batch(graphs)
    t_pack = time.perf_counter() - t0
    singles = [lp.Graph.from_csr(g) for g in graphs]
    st = torch.cuda.Stream()
    rows = []
    for m, cap in queries:
        default_ms, tuned_ms, opts = B.autotune(m, cap, k, repeats=2)
        for _ in range(args.warmup):
            B.predict_all(m, cap, k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            out, cnt = B.predict_all(m, cap, k)
        torch.cuda.synchronize()
        batched_s = (time.perf_counter() - t0) / args.steps
        links = int(cnt[: B.n_total].sum().item())
        # one plain call per graph, every vertex as a source
        bufs = []
        for g in graphs:
            src = torch.arange(g.n, dtype=torch.int32, device="cuda")
            bufs.append((src, torch.empty((max(g.n, 1) * k * 16,), dtype=torch.uint8, device="cuda"),
                         torch.empty((max(g.n, 1),), dtype=torch.int32, device="cuda")))
        for _ in range(max(1, args.warmup // 2)):
            for G, g, (src, o, c) in zip(singles, graphs, bufs):
                lp.lp_predict_sources_dev(G.handle, m, src, g.n, k, cap, 0.0, o, c)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for G, g, (src, o, c) in zip(singles, graphs, bufs):
                lp.lp_predict_sources_dev(G.handle, m, src, g.n, k, cap, 0.0, o, c)
        torch.cuda.synchronize()
        plain_s = (time.perf_counter() - t0) / args.steps
        same = all(
            np.array_equal(bufs[i][2].cpu().numpy(),
                           cnt[int(B.bases[i]):int(B.bases[i + 1])].cpu().numpy())
            for i in range(len(graphs)))
        rows.append({"query": f"{m}@{cap}", "links": links, "batched_ms": round(batched_s * 1e3, 3),
                     "plain_ms": round(plain_s * 1e3, 3),
                     "batched_edges_per_s": round(links / batched_s, 1),
                     "plain_edges_per_s": round(links / plain_s, 1),
                     "speedup": round(plain_s / batched_s, 2), "counts_identical": bool(same),
                     "autotune": {"default_ms": round(default_ms, 3), "tuned_ms": round(tuned_ms, 3),
                                  "options": opts}})
    for G in singles:
        G.close()
    B.close()
    tot_links = sum(r["links"] for r in rows)
    tot_b = sum(r["batched_ms"] for r in rows) / 1e3
    tot_p = sum(r["plain_ms"] for r in rows) / 1e3
    return {"metric": "predicted edges/s (batched per-source top-10, JC(256) + AA(32))",
            "value": round(tot_links / tot_b, 1), "unit": "edges/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "plain_value": round(tot_links / tot_p, 1), "speedup_vs_plain": round(tot_p / tot_b, 2),
            "data": "synthetic",
            "config": {"workload": f"{len(graphs)} Chung-Lu graphs, n log-uniform in [1k, 500k], "
                                   "mean degree U[8, 32], exponent U[2.0, 2.8], seeds 1000+i",
                       "vertices": int(sum(g.n for g in graphs)),
                       "edges_undirected": int(sum(g.edges for g in graphs)),
                       "generation_s": round(t_gen, 1), "pack_s": round(t_pack, 2)},
            "queries": rows}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    split = make_workload()
    obs = split.observed
    k = len(split.hu)

    cores = os.cpu_count() or 1

    def one():
        tot = 0
        for c, m in SAMPLE_CAPS:
            tot += len(oracle.predict(obs.n, obs.off, obs.idx, m, c, k=k, nthreads=cores))
        return tot

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        total += one()
    t = time.perf_counter() - t0
    value = total / t
    sample = ("oracle (CPU, OpenMP, all host cores): per step the DLH cap-16 JC and RA "
              "calls of the workload on the full graph")
    return {"metric": METRIC, "value": round(value, 1), "unit": "edges/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t * 1e3 / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + (f" [subset: scale {args.scale}]"
                                               if args.scale != 20 else ""), "sample": sample},
            "cpu_baseline": {"value": round(value, 1), "unit": "edges/s",
                             "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 1), "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------- distributed ----

_pg = None


def dist_init():
    global _pg
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        _pg = dist
    return rank, world, local


def dist_barrier(world):
    if world > 1 and _pg is not None:
        _pg.barrier()


def dist_max(x, world):
    if world > 1 and _pg is not None:
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        _pg.all_reduce(t, op=_pg.ReduceOp.MAX)
        return float(t.item())
    return x


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-baseline", default="full", choices=["full", "sample"],
                    help="oracle over all ten calls (full) or the cap-16 pair (sample)")
    ap.add_argument("--no-rmat24", action="store_true",
                    help="skip the R-MAT scale-24 DLH(256) record")
    ap.add_argument("--r24-steps", type=int, default=3, help="rmat24_dlh256: timed steps")
    ap.add_argument("--r24-warmup", type=int, default=1, help="rmat24_dlh256: warm-up steps")
    ap.add_argument("--only", default="", help="subset of calls, e.g. JC@inf,RA@256")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale (20 = the workload)")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "serve", "batch"],
                    help="sweep: the DLH cap sweep (the benchmark line); serve: serving study; "
                         "batch: batched multi-graph study")
    ap.add_argument("--graphs", type=int, default=256, help="batch: number of graphs")
    ap.add_argument("--requests", type=int, default=1500, help="serve: number of requests")
    ap.add_argument("--loads", type=float, nargs="+", default=[0.5, 0.9, 2.0],
                    help="serve: arrival rates as multiples of the plain capacity")
    ap.add_argument("--slots", type=int, default=2, help="serve: server slots")
    ap.add_argument("--select-buffer", type=int, default=0,
                    help="minimum selection-buffer capacity (candidates); 0 = library default")
    args = ap.parse_args()
    global _ARGS
    _ARGS = args
    rank, world, local = dist_init()
    if args.workload == "serve":
        line = run_serve(args) if rank == 0 else None
    elif args.workload == "batch":
        line = run_batch(args) if rank == 0 else None
    elif args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and _pg is not None:
        _pg.destroy_process_group()


if __name__ == "__main__":
    main()
