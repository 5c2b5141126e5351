"""Host-side pieces of bench.py that need no GPU: the defaults of the
command line, the summary of the nvidia-smi clock samples, the measured-peak
lookup and the gate on the committed DRAM-traffic figures (a figure counts
only for the render source and workload it was captured on)."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_defaults_one_gpu_and_enough_warmup(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    assert a.impl == "ours" and a.config == "cfg2" and a.attr == "f32" and a.tile == 16
    assert a.batch == 0 and a.ppt == 0 and a.persistent == 0


def test_clock_rows_median_max_and_reasons():
    rows = [
        "0, 1965, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1180.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "index, clocks.sm, clocks.max.sm",  # a header line: skipped
        "0, 2010, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.summarise_clock_rows(rows)
    assert c["samples"] == 3 and c["sm_mhz"] == 1980.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    hot = rows + ["0, 1500, 2070, 1300.0, 0x48, Active, Active, Not Active, Not Active"]
    assert bench.summarise_clock_rows(hot)["reasons"] == [
        "hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    assert bench.summarise_clock_rows([]) is None
    assert bench.summarise_clock_rows(["garbage"]) is None


def _fake_root(tmp_path, src=b"// kernels\n", entry=None):
    csrc = tmp_path / "paper_2603_09277_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "render.cu").write_bytes(src)
    (tmp_path / "profiles").mkdir()
    h = hashlib.sha256(src).hexdigest()[:16]
    ent = {"bytes_per_launch": 4.5e7, "render_cu_sha256_16": h, "config": "cfg2"}
    ent.update(entry or {})
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"render_bwd_kernel": ent}))
    return h


def test_traffic_counts_only_for_its_source_and_workload(tmp_path, monkeypatch):
    _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg2") == 4.5e7
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg3") is None
    assert bench.traffic_from_profiles("render_fwd_kernel", "cfg2") is None
    # the source changed after the capture: no figure
    (tmp_path / "paper_2603_09277_gb300" / "csrc" / "render.cu").write_bytes(b"// changed\n")
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg2") is None
    # unreadable or absent summary: no figure
    (tmp_path / "profiles" / "traffic.json").write_text("{not json")
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg2") is None
    (tmp_path / "profiles" / "traffic.json").unlink()
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg2") is None


def test_measured_peak_else_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_peak() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6681.5}))
    assert bench.measured_hbm_peak() == (6681.5, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops": 1900}))
    assert bench.measured_hbm_peak() == (6800.0, "fallback")


def test_committed_peaks_file_is_read_when_present():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("no measured peaks in this checkout")
    want = float(json.load(open(path))["hbm_gbs"])
    assert bench.measured_hbm_peak() == (want, "measured")
