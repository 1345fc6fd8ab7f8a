"""Host-side pieces of bench.py that need no GPU: the stored DRAM-traffic
figure is used only for its own workload and kernel sources (scaled to the
run's entries per launch when taken on a smaller case), the stored figures
are consistent with their capture, and the config object both arms print."""
from __future__ import annotations

import json
import os

import pytest

import bench


def _write(tmp_path, **d):
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(d))
    return str(p)


def test_traffic_figure_only_for_its_workload_and_sources(monkeypatch, tmp_path):
    sha = bench.decide_sources_sha()
    path = _write(tmp_path, source_sha256=sha, dram_bytes_per_launch=1000.0,
                  dram_bytes_per_scanned_entry=2.5)
    monkeypatch.setitem(bench.TRAFFIC_FILES, "cl", path)
    # a figure per scanned entry scales to the run's entries per launch
    assert bench.measured_traffic("cl", 400) == 1000.0
    assert bench.measured_traffic("cl", 800) == 2000.0
    path2 = _write(tmp_path, source_sha256=sha, dram_bytes_per_launch=1234.0)
    monkeypatch.setitem(bench.TRAFFIC_FILES, "cl", path2)
    assert bench.measured_traffic("cl", 400) == 1234.0
    monkeypatch.setattr(bench, "decide_sources_sha", lambda: "0" * 64)
    assert bench.measured_traffic("cl", 400) is None              # the kernels changed since
    monkeypatch.setitem(bench.TRAFFIC_FILES, "cl", str(tmp_path / "missing.json"))
    assert bench.measured_traffic("cl", 400) is None
    assert bench.measured_traffic("lowdeg", 400) is None


@pytest.mark.parametrize("key", sorted(bench.TRAFFIC_FILES))
def test_stored_traffic_figures_against_algorithmic_bytes(key):
    path = bench.TRAFFIC_FILES[key]
    if not os.path.exists(path):
        pytest.skip("no capture stored for this workload")
    with open(path) as f:
        d = json.load(f)
    ratio = d["dram_bytes_per_launch"] / d["algorithmic_bytes_per_launch"]
    assert 0.5 <= ratio < 4.0
    assert abs(d["dram_bytes_per_launch"] * d["sub_sweeps"] - (d["dram_read_bytes"] + d["dram_write_bytes"])) <= d["sub_sweeps"]


def test_config_objects():
    c = bench.RmatWorkload(22).config(4194304, 128312380, "det", 2)
    assert c["parallelism"] == "replicas x2" and c["schedule"] == "det"
    assert c["batch_fracs"] == list(bench.RMAT_FRACS)
    assert c["l2"].startswith("inputs larger than L2 (CSR 1.1 GB)")
    c = bench.ChungLuWorkload().config(bench.CL_N, 2 * bench.CL_M, "det", 1)
    assert c["workload"].startswith("chung-lu") and c["batch_fracs"] == list(bench.CL_FRACS)
    assert c["l2"].startswith("inputs larger than L2 (CSR 16.4 GB)")
    assert bench.l2_note(50e6).startswith("inputs smaller than L2")


def test_host_info_names_the_cores():
    h = bench.host_info()
    assert h["nproc"] == os.cpu_count()
