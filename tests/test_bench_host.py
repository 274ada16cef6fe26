"""Host-side pieces of bench.py that need no GPU: the clock-sample summary
(throttle reasons must be reported), the tie of the stored DRAM-traffic figure
to the blend kernel's source, the oracle arm's bounded per-step timing, the
per-tile distinct-row count U_tile and the near-tie categories of the parity
sample."""
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


def test_tile_distinct_rows_counts_each_tile_s_set_once():
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(3)
    W, H, K = 37, 21, 5                      # ragged 16x16 tiles on both axes
    ids = rng.integers(-1, 40, (W * H, K)).astype(np.int32)
    got = bench.tile_distinct_rows(torch.from_numpy(ids), W, 16, 16)
    seen = set()
    for p in range(W * H):
        y, x = divmod(p, W)
        seen.update((y // 16, x // 16, int(v)) for v in ids[p] if v >= 0)
    assert got == len(seen)
    # one tile, every pixel listing the same rows: U_tile = U
    same = np.tile(np.array([[3, 7, -1, -1, -1]], np.int32), (16 * 16, 1))
    assert bench.tile_distinct_rows(torch.from_numpy(same), 16, 16, 16) == 2


def test_parity_sample_reports_tie_categories():
    class Ref:
        pass
    K, W = 2, 4
    pix = np.array([[0, 0], [1, 0], [2, 0], [3, 0]], np.int32)
    ref = Ref()
    ref.ids = np.array([[5, -1], [6, 7], [8, -1], [1, 2]], np.int32)
    ref.cnt = np.array([1, 2, 1, 2])
    ref.tie = np.array([0, 1, 2 | 4, 1 | 8])     # bit 8 (dense T_min) is not Algorithm 1's
    ref.wq = np.zeros((4, K))
    ref.out_q = np.zeros((4, 3))
    ref.scale_q = np.ones(4)
    ids = ref.ids.copy()
    ids[1] = [6, 9]                               # a mismatch on a flagged pixel only
    rep = bench.sample_parity(ids, ref.cnt.astype(np.uint8), np.zeros((4, 3)), W, pix, ref)
    assert rep["near_tie_pixels"] == 3 and rep["mismatch_nontie"] == 0
    assert rep["near_tie_by_category"] == {"boundary": 2, "alpha_min_border": 1, "equal_depth": 1}
