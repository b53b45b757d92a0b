"""Host-side logic of bench.py on CPU: the roofline block's arithmetic, and the rule that
captured DRAM traffic is reported only while the kernel sources hash to the captured
version (a kernel change cannot keep stale counters: the line then reports null)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_block_arithmetic():
    rb = bench.roofline_block("k", 20, 1_000_000, 2.0, traffic=123)
    # 20 B x 1e6 nodes in 2 ms = 10 GB/s
    assert rb["achieved"] == pytest.approx(10.0)
    peak, kind = bench.measured_peaks()
    assert rb["peak"] == peak and rb["peak_kind"] == kind
    assert rb["frac"] == pytest.approx(10.0 / peak)
    assert rb["traffic"] == 123 and rb["unit"] == "GB/s" and rb["bound"] == "hbm"


def test_captured_traffic_needs_the_captured_sources(monkeypatch):
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {"w": {"hash": h, "bytes": 42},
                                                    "stale": {"hash": "0" * 16, "bytes": 7}})
    assert bench.captured_traffic("w") == 42
    assert bench.captured_traffic("stale") is None
    assert bench.captured_traffic("absent") is None
    # the adjoint's counters are keyed on the adjoint's sources as well
    assert bench.captured_traffic("w", bench.ADJOINT_SOURCES) is None


def test_measured_peak_is_used_when_present():
    peak, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000.0
    else:
        assert kind == "fallback" and peak == bench.FALLBACK_HBM_GBS


def test_captured_traffic_needs_the_captured_options(monkeypatch):
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {
        "default": {"hash": h, "bytes": 1},
        "tuned": {"hash": h, "bytes": 2, "opts": {"tile": "8x8x8", "order": 0.0, "converge": "sweep"}}})
    assert bench.captured_traffic("default") == 1
    assert bench.captured_traffic("default", opts={"tile": "8x8x8", "order": 0.0, "schedule": "persistent"}) == 1
    assert bench.captured_traffic("default", opts={"tile": "8x8x4"}) is None
    assert bench.captured_traffic("tuned", opts={"tile": "8x8x8", "order": 0.0, "schedule": "persistent",
                                                 "converge": "sweep"}) == 2
    assert bench.captured_traffic("tuned", opts={"tile": "8x8x8", "order": 0.0}) is None


def test_source_hash_ignores_comments_but_not_code():
    a = "int f(int x) { return x + 1; }  // one\n/* two */"
    b = "int  f(int x)\n{ return x + 1; }   // another comment"
    c = "int f(int x) { return x + 2; }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
