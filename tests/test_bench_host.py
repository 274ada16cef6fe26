"""Host-side pieces of bench.py that need no GPU: the clock-sample summary
(throttle reasons must be reported), the tie of the stored DRAM-traffic figure
to the blend kernel's source, and the oracle arm's bounded per-step timing."""
import json
import os

import numpy as np

import bench
from paper_2512_20927_gb300 import scenes


def _sampler_with(rows):
    s = bench.ClockSampler(0)
    s.proc = object()   # a sampler that ran
    s.path = os.path.join(os.environ.get("PYTEST_TMP", "/tmp"), f"qr_clock_test_{os.getpid()}.csv")
    with open(s.path, "w") as fh:
        for r in rows:
            fh.write(", ".join(r) + "\n")
    return s


def test_clock_summary_reports_median_and_throttle_reasons():
    idle = ["0", "2070", "2070", "900.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    capped = ["0", "1950", "2070", "1400.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"]
    hot = ["0", "1800", "2070", "1400.0", "0x40", "Not Active", "Active", "Not Active", "Not Active"]
    s = _sampler_with([idle, capped, idle])
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    out = _sampler_with([idle, hot]).summary()
    assert out["reasons"] == ["hw_thermal_slowdown"]
    assert _sampler_with([]).summary() is None


def test_traffic_figure_is_tied_to_the_kernel_source(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "blend_indoor_traffic.json")
    stored = json.load(open(path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: stored["kernel_source_hash"])
    assert bench._traffic_from_profile() == stored["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench._traffic_from_profile() is None


def test_oracle_arm_step_is_bounded_and_reuses_the_projection():
    g, f = scenes.tiny_scene(n=300, channels=8)
    cam = scenes.tiny_camera(32, 24)
    fps, cores, npx, secs = bench.oracle_frames_per_s(g, f, cam, 0.2, seed=0)
    assert fps > 0 and cores >= 1 and npx >= cores
    proj = bench.oracle_frames_per_s.last_proj
    fps2, _, _, secs2 = bench.oracle_frames_per_s(g, f, cam, 0.2, seed=1, proj=proj)
    assert fps2 > 0 and np.isfinite(secs2)
    assert bench.oracle_frames_per_s.last_proj[1] == proj[1]   # the projection time is reused
