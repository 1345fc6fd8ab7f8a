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


def test_record_traffic_reads_an_ncu_capture(monkeypatch, tmp_path):
    hdr = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
          '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"'
    rows = []
    for k, (name, rd, wr) in enumerate([("void decide_group<16, 5, 0, 0, int, long>(MoveArgs<T5>)", 100.0, 10.0),
                                        ("void hub_insert_k<int, unsigned int>(MoveArgs<T1>, bool, HubWork)", 2.0, 1.0),
                                        ("apply_moves_k(const int *, long *)", 999.0, 999.0)]):
        for metric, unit, v in (("dram__bytes_read.sum", "Mbyte", rd), ("dram__bytes_write.sum", "Mbyte", wr),
                                ("gpu__time_duration.sum", "usecond", 5.0)):
            rows.append(f'"{k}","1","python","h","{name}","1","13","(256, 1, 1)","(9, 1, 1)","0","10.3",'
                        f'"Command line profiler metrics","{metric}","{unit}","{v}"')
    csv_path = tmp_path / "cap.csv"
    csv_path.write_text("==PROF== noise\n" + hdr + "\n" + "\n".join(rows) + "\n")
    prof = tmp_path / "prof.log"
    prof.write_text('log line\n{"workload": "w", "move0_kernel_launches": 2, "move0_bytes": 500e6, '
                    '"move0_scanned_entries": 1000000}\n')
    out = tmp_path / "traffic.json"
    monkeypatch.setitem(bench.TRAFFIC_FILES, "cl", str(out))

    class A:
        record_traffic, profile_json, workload = str(csv_path), str(prof), "cl"
    assert bench.record_traffic(A) == 0
    d = json.loads(out.read_text())
    assert d["dram_read_bytes"] == 102e6 and d["dram_write_bytes"] == 11e6   # apply kernel left out
    assert d["dram_bytes_per_launch"] == 113e6 / 2 and d["algorithmic_bytes_per_launch"] == 250e6
    assert d["dram_bytes_per_scanned_entry"] == 113.0
    assert bench.measured_traffic("cl", 1000) == 113000.0
