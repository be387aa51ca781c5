"""Host logic of bench.py's measurement (no GPU): captured counters go stale with their kernel
sources, and a form's roofline fraction is the larger of its HBM and pipe fractions."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_every_counter_names_known_sources():
    for (path, key), e in bench.COUNTERS.items():
        assert key in ("flops", "dram")
        assert path.split(":")[0] in bench.PATH_SOURCES
        assert len(e["source_hash"]) == 16 and e["capture"].startswith("ncu")
        for f in bench.PATH_SOURCES[path.split(":")[0]]:
            assert os.path.exists(os.path.join(bench.CSRC, f)), f


def test_counter_is_null_once_sources_change(monkeypatch):
    path = "d3q27:f32"
    e = bench.COUNTERS[(path, "flops")]
    monkeypatch.setattr(bench, "source_hash", lambda files: e["source_hash"])
    assert bench.counter(path, "flops")[0] == e["value"]
    monkeypatch.setattr(bench, "source_hash", lambda files: "0" * 16)
    v, note = bench.counter(path, "flops")
    assert v is None and "changed" in note
    assert bench.counter("d3q27:nonexistent", "flops") == (None, "not captured")


def test_roofline_takes_the_slower_limit(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "pipe_peaks", lambda device: {"fp32x2": 60.0, "fp64": 1.0})
    monkeypatch.setattr(bench, "counter", lambda path, key: (500.0, "test"))
    # 1e9 updates in 100 ms: 200 B -> 2000 GB/s (1/3 of HBM); 500 flops -> 5 TFLOP/s of 60
    r = bench.roofline(1e9, 100.0, 200, "fp32", "d3q27:f32", 0)
    assert abs(r["hbm_frac"] - 1 / 3) < 1e-12 and abs(r["pipe_frac"] - 5 / 60) < 1e-12
    assert r["bound"] == "hbm" and r["frac"] == r["hbm_frac"]
    r = bench.roofline(1e9, 100.0, 200, "fp64", "d3q27:f64", 0)     # 5 TFLOP/s of 1: pipe-bound
    assert r["bound"] == "fp64" and abs(r["frac"] - 5.0) < 1e-12
    r = bench.roofline(1e9, 100.0, 200, None, None, 0)
    assert r["bound"] == "hbm" and "pipe_frac" not in r
