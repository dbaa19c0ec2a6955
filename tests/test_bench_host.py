"""Host-side arithmetic of bench.py (no GPU): the lower bounds reported beside the roofline
and the algorithmic byte and flop counts of a workload."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_bounds_pick_the_tightest():
    # 100 hops of 1 us; 6.782 GB at 6782.1 GB/s is 1 ms; 2.5 GFLOP at 1.25 TFLOP/s is 2 ms
    r = bench.roofline_bounds(100, 1000.0, 6.7821e9, 6782.1, 2.5e9, "f64", 4.0)
    assert r["latency_bound_ms"] == pytest.approx(0.1)
    assert r["hbm_bound_ms"] == pytest.approx(1.0)
    assert r["fp64_bound_ms"] == pytest.approx(2.0)
    assert r["tightest_bound"] == "fp64"
    assert r["frac_of_tightest_bound"] == pytest.approx(0.5)
    r = bench.roofline_bounds(10 ** 5, 1000.0, 6.7821e9, 6782.1, 2.5e9, "f64", 400.0)
    assert r["tightest_bound"] == "latency" and r["frac_of_tightest_bound"] == pytest.approx(0.25)


def test_no_fp64_bound_for_fp32():
    r = bench.roofline_bounds(10, 1000.0, 6.7821e9, 6782.1, 2.5e9, "f32", 2.0)
    assert r["fp64_bound_ms"] is None and r["fp64_peak_tflops"] is None
    assert r["tightest_bound"] == "hbm"


def test_lap2d64_counts():
    # 64 x 64 grid: L has n + (n - 64) + (n - 64) entries (diagonal, west, south), M the
    # full 5-point pattern; FP64 CSR costs 12 bytes per entry plus the row pointers
    wl = bench.make_workload("lap2d64", "f64")
    n = 4096
    nnzL = n + 2 * (n - 64)
    nnzM = n + 4 * (n - 64)
    assert (wl["nnzL"], wl["nnzM"]) == (nnzL, nnzM)
    csr = lambda z: 12 * z + 4 * (n + 1)
    assert wl["fwd_bytes"] == csr(nnzL) + csr(nnzM) + 3 * 8 * n
    assert wl["fwd_flops"] == 2 * (nnzL + nnzM) + n


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    # a record counts only while the files it lists are unchanged; other sources may change
    csrc = tmp_path / "paper_2111_12238_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cuh").write_text("kernel v1")
    (csrc / "other.cu").write_text("launcher v1")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench._csrc_hash(["k.cuh"])
    rec = {"w": {"fwd": {"kernel": "k", "bytes_per_launch": 1234, "sources": ["k.cuh"], "csrc_hash": h}}}
    (tmp_path / "profiles" / "traffic.json").write_text(__import__("json").dumps(rec))
    assert bench._recorded_traffic("w", "fwd") == 1234
    (csrc / "other.cu").write_text("launcher v2")
    assert bench._recorded_traffic("w", "fwd") == 1234
    (csrc / "k.cuh").write_text("kernel v2")
    assert bench._recorded_traffic("w", "fwd") is None
    assert bench._recorded_traffic("w", "adj") is None
