"""Host-side pieces of bench.py that need no GPU: the defaults of the
command line, the summary of the nvidia-smi clock samples, the measured-peak
lookup, the gate on the committed DRAM-traffic figures (a figure counts only
for the render source and workload it was captured on), and the launch-form
autotuner's choice and cache with its timing replaced."""
import hashlib
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_defaults_one_gpu_and_enough_warmup(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    # the metric's configuration: the batched workload of 8 views of uneven size
    assert a.impl == "ours" and a.config == "cfg3" and a.attr == "f32" and a.tile == 16
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
    ent = {"kernel": "render_bwd_kernel", "bytes_per_launch": 4.5e7, "source": "render.cu",
           "source_sha256_16": h, "config": "cfg2"}
    ent.update(entry or {})
    other = dict(ent, config="cfg3", bytes_per_launch=1.4e8)
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"entries": [ent, other]}))
    return h


def test_traffic_counts_only_for_its_source_and_workload(tmp_path, monkeypatch):
    _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg2") == 4.5e7
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg3") == 1.4e8
    assert bench.traffic_from_profiles("render_bwd_kernel", "cfg5") is None
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


def test_autotune_picks_the_fastest_form_and_caches_it(tmp_path, monkeypatch):
    """The autotuner's host logic with the timing replaced: the fastest
    candidate wins, the choice is cached per workload signature (candidate
    set included) and reused unless forced."""
    from paper_2603_09277_gb300 import autotune, scenes
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda *a: "GB300 (fake)")
    calls = []

    def fake_time(cams, prm, params, target, gamma, form, attr_dtype="f32", steps=5, warmup=2):
        calls.append(autotune.form_name(form))
        # 2 px/thread, 128-entry batch, one CTA per tile is the fastest here
        return 1.0 if autotune.form_name(form) == "ppt2_b128_per_tile" else 2.0 + len(calls)

    monkeypatch.setattr(autotune, "time_form", fake_time)
    cams = [scenes.camera(64, 48, 64.0)]
    prm = scenes.params()
    params = {"means": np.zeros((10, 3), np.float32)}
    best, ms = autotune.tune(cams, prm, params, None, 0.015)
    assert best == {"pixels_per_thread": 2, "persistent": 0, "batch": 128}
    assert sorted(ms) == sorted(calls) == sorted(autotune.form_name(f)
                                                 for f in autotune.candidates(16, "f32"))
    n = len(calls)
    assert autotune.tune(cams, prm, params, None, 0.015)[0] == best and len(calls) == n
    autotune.tune(cams, prm, params, None, 0.015, force=True)
    assert len(calls) == 2 * n
    # another staging dtype is another workload, without the 128-entry forms
    best16, ms16 = autotune.tune(cams, prm, params, None, 0.015, attr_dtype="bf16")
    assert best16["batch"] == 256 and not any("_b128_" in k for k in ms16)
    db = json.load(open(tmp_path / "autotune.json"))
    assert len(db) == 2 and all("GB300 (fake)" in k for k in db)


def test_view0_error_leaves_out_excluded_and_other_pixels():
    """The error a form states is the largest difference over the compared
    pixels of view 0 only: pixels outside the oracle's band, excluded pixels
    and pixels of later views do not count."""
    torch = pytest.importorskip("torch")
    H, W = 4, 5
    mask = np.zeros((H, W), bool)
    mask[1:3] = True
    excl = np.zeros((H, W), bool)
    excl[1, 0] = True
    ref = {"mask": mask, "excluded": excl, "image": np.zeros((H, W, 3)),
           "final_T": np.ones((H, W)), "entropy": np.zeros((H, W))}
    img = torch.zeros(H * W + 7, 3)
    img[W * 1 + 0] = 5.0          # excluded pixel
    img[0] = 3.0                  # outside the band
    img[H * W + 2] = 9.0          # a later view
    img[W * 2 + 3, 1] = 0.25      # compared
    T = torch.ones(H * W + 7)
    T[W * 1 + 1] = 0.5
    h = torch.zeros(H * W + 7)
    e = bench.view0_error(ref, img, T, h)
    assert e == {"image": 0.25, "final_T": 0.5, "entropy": 0.0}
