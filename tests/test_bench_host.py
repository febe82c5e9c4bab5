"""bench.py host logic (no GPU): the roofline object of the JSON line.

The fraction is the sector model's bytes over the measured step time and the
measured copy peak; the ncu traffic figure is attached only while the round
kernels' sources hash to the value the capture was keyed to, so a kernel
changed since the capture reports no traffic instead of a stale one.
"""
import importlib

import pytest

bench = importlib.import_module("bench")

N, M = 1_000_000, 1_230_000
STATS = {"first_layer": 240_000, "n_peeled": N, "frontier": 860_000, "hinge_moves": 18_000}


def _prof(rounds_ms=100.0, steps=10):
    # name -> [launches, total ms] over `steps` steps, as profile_read gives it
    return {"records_bucket": [steps, 10.0 * steps], "rounds": [steps, rounds_ms * steps],
            "emit_scatter": [steps, 3.0 * steps]}


def test_roofline_is_the_largest_step_against_the_measured_peak():
    r = bench.roofline_of(_prof(), 10, N, M, STATS, "graph")
    assert r["kernel"] == "rounds"
    model = bench.byte_model("rounds", N, M, STATS)
    assert r["algorithmic_bytes_per_step"] == model["sector"]
    assert r["achieved"] == pytest.approx(model["sector"] / 0.1 / 1e9)
    peak, _ = bench.measured_peaks()
    assert r["peak"] == peak
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["launches_per_step"] == 1  # the graph loop is one launch
    assert model["word"] < model["sector"]


def test_host_loop_folds_round_zero_and_sorted_rounds_into_the_rounds():
    prof = _prof(rounds_ms=60.0)
    prof["round0"] = [10, 80.0]
    prof["rounds_sorted"] = [30, 300.0]
    r = bench.roofline_of(prof, 10, N, M, STATS, "host")
    assert r["kernel"] == "rounds"
    assert r["ms_per_step"] == pytest.approx(60.0 + 8.0 + 30.0)
    assert r["launches_per_step"] == pytest.approx((10 + 10 + 30) / 10)


def test_traffic_only_while_the_sources_match_the_capture(monkeypatch):
    src, _, per_unit, where = bench.NCU_TRAFFIC["rounds"]
    # keyed to the present sources: the figure is scaled by the units
    monkeypatch.setitem(bench.NCU_TRAFFIC, "rounds", (src, bench.src_hash(src), per_unit, where))
    r = bench.roofline_of(_prof(), 10, N, M, STATS, "graph")
    assert r["traffic_per_step"] == pytest.approx(per_unit * N)
    assert r["traffic"] == pytest.approx(per_unit * N)
    assert r["traffic_source"].startswith("ncu dram__bytes")
    # keyed to other sources: no traffic rather than a stale one
    monkeypatch.setitem(bench.NCU_TRAFFIC, "rounds", (src, "0" * 16, per_unit, where))
    r = bench.roofline_of(_prof(), 10, N, M, STATS, "graph")
    assert r["traffic"] is None and r["traffic_per_step"] is None


def test_source_hash_covers_every_listed_file(tmp_path, monkeypatch):
    a, b = tmp_path / "a.cu", tmp_path / "b.cu"
    a.write_text("x")
    b.write_text("y")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.src_hash(("a.cu", "b.cu"))
    b.write_text("z")
    assert bench.src_hash(("a.cu", "b.cu")) != h
    assert len(h) == 16
