"""Host-side pieces of bench.py that need no GPU: the stored DRAM-traffic
figure is used only for its own workload and kernel sources, and the config
object both arms print."""
from __future__ import annotations

import json

import bench


def test_traffic_figure_only_for_its_workload_and_sources(monkeypatch, tmp_path):
    with open(bench.TRAFFIC_FILE) as f:
        stored = json.load(f)
    fresh = stored["source_sha256"] == bench.decide_sources_sha()
    assert bench.measured_traffic(stored["scale"]) == (float(stored["dram_bytes_per_launch"]) if fresh else None)
    assert bench.measured_traffic(stored["scale"] - 2) is None
    monkeypatch.setattr(bench, "decide_sources_sha", lambda: "0" * 64)
    assert bench.measured_traffic(stored["scale"]) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_traffic(stored["scale"]) is None


def test_traffic_figure_against_algorithmic_bytes():
    with open(bench.TRAFFIC_FILE) as f:
        d = json.load(f)
    ratio = d["dram_bytes_per_launch"] / d["algorithmic_bytes_per_launch"]
    assert 1.0 <= ratio < 4.0
    assert d["dram_bytes_per_launch"] * d["sub_sweeps"] == d["dram_read_bytes"] + d["dram_write_bytes"]


def test_config_object():
    c = bench.workload_config(22, 4194304, 128312380, "det", 2)
    assert c["parallelism"] == "replicas x2" and c["schedule"] == "det"
    assert c["batch_fracs"] == list(bench.BATCH_FRACS)
    assert c["l2"].startswith("inputs larger than L2 (CSR 1.1 GB)")
    assert bench.l2_note(50e6).startswith("inputs smaller than L2")
