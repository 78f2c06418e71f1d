"""Host logic of bench.py without a GPU: which schedule an arm runs, the L2
fetch granularity it runs with, and when the committed ncu traffic figure
applies (same kernel sources, same fetch granularity)."""
import json

import bench


def test_effective_schedule():
    # 16-bit storage runs the two-pass schedule unless tiled is asked for;
    # AUTO is tiled for 4- and 8-byte storage
    for k in ("auto", "two_pass", "fused", "tiled"):
        for st in ("fp16", "bf16"):
            assert bench.effective_schedule(k, st) == ("tiled" if k == "tiled" else "two_pass")
    for st in ("fp32", "fp64"):
        assert bench.effective_schedule("auto", st) == "tiled"
        for k in ("two_pass", "fused", "tiled"):
            assert bench.effective_schedule(k, st) == k


def test_l2_fetch_per_schedule():
    assert bench.l2_fetch_for("auto", "fp32", -1) == 128
    assert bench.l2_fetch_for("tiled", "fp64", -1) == 128
    assert bench.l2_fetch_for("two_pass", "fp32", -1) == 32
    assert bench.l2_fetch_for("auto", "fp16", -1) == 32
    assert bench.l2_fetch_for("tiled", "fp16", -1) == 128
    assert bench.l2_fetch_for("fused", "fp32", -1) == 32
    for req in (0, 32, 64, 128):  # an explicit request wins
        assert bench.l2_fetch_for("auto", "fp32", req) == req


def test_traffic_applies_only_to_matching_captures(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.source_hash()
    (prof / "traffic.json").write_text(json.dumps({
        "tile/fp32": {"bytes_per_launch_full": 8.0e9, "source_hash": h, "l2_fetch_granularity_bytes": 128},
        "collide/fp32": {"bytes_per_launch_full": 7.0e9, "source_hash": "stale", "l2_fetch_granularity_bytes": 32},
    }))
    # measured_traffic reads profiles/ under bench.ROOT; point it at the copy
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: h)
    assert bench.measured_traffic("tile", "fp32", 128) == 8.0e9
    assert bench.measured_traffic("tile", "fp32", 32) is None      # other fetch granularity
    assert bench.measured_traffic("collide", "fp32", 32) is None   # taken on other sources
    assert bench.measured_traffic("march", "fp32", 32) is None     # never captured

