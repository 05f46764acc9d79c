"""The benchmark's JSON contract on the host (no GPU): the reference arm (the
oracle on the host cores) prints one JSON line with the benchmark's keys,
and the DRAM-traffic record is used only while the kernel sources hash to
the value stored with it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--scale", "10", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True).stdout
    d = json.loads(out.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert "[subset: scale 10]" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_traffic_record_follows_kernel_hash(tmp_path, monkeypatch):
    b = _bench_module()
    h = b.kernel_hash()
    assert h == b.kernel_hash() and len(h) == 16
    (tmp_path / "profiles").mkdir()
    rec = {"k_scan_big": {"kernel_hash": h, "dram_bytes_per_alg_byte": 0.25,
                          "workload": "a test"}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    # the hash is taken over the sources under ROOT: point it back at the repository's
    monkeypatch.setattr(b, "kernel_hash", lambda kernel="k_scan_big": h)
    t, basis = b.traffic_record("k_scan_big", 4000)
    assert t == 1000 and "a test" in basis
    assert b.traffic_record("k_scan_cta", 4000) == (None, None)
    monkeypatch.setattr(b, "kernel_hash", lambda kernel="k_scan_big": "0" * 16)
    assert b.traffic_record("k_scan_big", 4000) == (None, None)


def test_roofline_picks_dominant_tier_and_counts_its_bytes():
    b = _bench_module()
    st = {"tier_ms": [1.0, 2.0, 3.0, 10.0], "tier_launches": [1, 1, 2, 4],
          "tier_arcs": [10, 20, 30, 1000], "tier_kept": [5, 5, 5, 500],
          "tier_wedges": [7, 7, 7, 100000]}
    r = b.roofline([st, st])
    assert r["kernel"] == "k_exp_tiles+k_exp_count"
    alg = 2 * (8 * 1000 + 4 * 500 + 4 * 100000)
    assert r["launches"] == 8 and r["alg_bytes_per_launch"] == alg // 8
    assert abs(r["avg_launch_ms"] - 20.0 / 8) < 1e-9
    gbs = (alg / 8) / (20.0 / 8 * 1e-3) / 1e9
    assert abs(r["achieved"] - round(gbs, 1)) < 0.11
    assert abs(r["frac"] - round(gbs / r["peak"], 4)) < 1e-4
    assert abs(r["share_of_scan_ms"] - 10.0 / 16.0) < 1e-4
    old = {k: v[:3] for k, v in st.items()}  # three tiers (per-source statistics)
    assert b.roofline([old])["kernel"] == "k_scan_big"
