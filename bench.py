"""Benchmark of the Q-Render hot path on GB300 (one JSON line on stdout).

Workload (the metric's configuration): the synthetic indoor room -- 500,000
Gaussians, 60 % within 2 cm of the floor/walls and 40 % uniform in the
6 x 6 x 3 m box, 512-D L2-normalised FP32 features, one 640 x 480 camera with a
60 degree horizontal field of view at the room centre; Q-Render with K = 8
against the dense Eq. 1 blend on the same GPU.

A step is one Q-Render frame: projection, depth sort + binning + tile sort +
ranges, Algorithm 1 selection and the feature blend (all in this repo's
kernels).  `value` is frames/s with the inputs resident in HBM; `e2e` is the
same metric through qr_render_host with pinned host buffers (inputs copied in
and the 512-D map copied out every step).  The dense Eq. 1 frame rate, the
per-stage times and K = 4 / 16 are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
(under torchrun for N > 1: every rank renders its own frames, no collective
on the data path; the time is the max over ranks).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "indoor-room FP32: 500k Gaussians, 640x480, 512-D features, Q-Render K=8 vs dense"
N_GAUSS, WIDTH, HEIGHT, C, K = 500_000, 640, 480, 512, 8
METRIC = "512-D feature frames/s, Q-Render vs dense blend on 1 GB300; % HBM roofline"


def config_dict(n):
    """The workload's config (the same dict in both arms)."""
    return {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT,
            "channels": C, "K": K, "tile": "16x16",
            "l2": "inputs larger than L2 (1.0 GB feature table, 0.63 GB map per step)",
            "parallelism": f"{n} independent renderers" if n > 1 else "single GPU"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, ws, device=None):
    """Element-wise maximum over all ranks of this rank's timings (ms): the
    job is as slow as its slowest rank."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64)
    if ws > 1:
        import torch.distributed as dist
        if device is not None:
            t = t.to(device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t = t.cpu()
    return [float(x) for x in t]


def whole_job_rate(ws, ms_per_step):
    """Frames per second of the whole job when every rank renders one frame per
    step (weak scaling: the per-rank work is fixed as ranks are added)."""
    return ws * 1000.0 / ms_per_step


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"qr_clocks_{os.getpid()}.csv")

    def __enter__(self):
        self.fh = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is live (bounded wait)
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.fh is not None:
            self.fh.close()
            self.fh = None

    def summary(self):
        """Clock summary of the samples taken; removes the sample file."""
        if not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.remove(self.path)
        if self.proc is None:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def kernel_source_hash() -> str:
    """Hash of the blend kernel's source file (ties a stored ncu traffic figure to it)."""
    with open(os.path.join(ROOT, "paper_2512_20927_gb300", "csrc", "blend.cu"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def _traffic_from_profile():
    """DRAM bytes per launch of the blend kernel from the committed ncu summary,
    only if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "blend_indoor_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- CPU oracle
def oracle_frames_per_s(g, feat, cam, budget_s: float, seed: int = 0, proj=None):
    """FP64 oracle (test infrastructure) on a bounded sample of the workload's pixels.

    proj: (projection, its seconds) from an earlier call, reused so that a
    run of many steps times the full-frame projection once; every step's
    frame time still includes it."""
    import oracle
    feat = np.ascontiguousarray(feat, np.float64)   # converted once, outside the timed part
    if proj is None:
        t0 = time.perf_counter()
        pr = oracle.project(g, cam.as_array())
        t_proj = time.perf_counter() - t0
    else:
        pr, t_proj = proj
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    P = cam.width * cam.height
    # calibrate on a small sample, then size the sample to the budget
    npx = cores * 2
    pix = np.stack([rng.integers(0, cam.width, npx), rng.integers(0, cam.height, npx)], 1)
    t0 = time.perf_counter()
    oracle.render(pr, feat, K, pix.astype(np.int32), want_dense=False, threads=cores,
                  alpha_min=oracle.ALPHA_MIN_F32, alpha_max=oracle.ALPHA_MAX_F32)
    per_px = (time.perf_counter() - t0) / npx
    npx = int(max(cores, min(P, (budget_s - t_proj) / max(per_px, 1e-9))))
    pix = np.stack([rng.integers(0, cam.width, npx), rng.integers(0, cam.height, npx)], 1)
    t0 = time.perf_counter()
    ref = oracle.render(pr, feat, K, pix.astype(np.int32), want_dense=False, threads=cores,
                        alpha_min=oracle.ALPHA_MIN_F32, alpha_max=oracle.ALPHA_MAX_F32)
    t_px = (time.perf_counter() - t0) / npx
    frame_s = t_proj + t_px * P
    oracle_frames_per_s.last_proj = (pr, t_proj)
    oracle_frames_per_s.last_sample = (pix.astype(np.int32), ref)
    return 1.0 / frame_s, cores, npx, t_proj + t_px * npx


def sample_parity(ids, counts, out, width, pix, ref):
    """Selections and features of the GPU frame on the oracle's sampled pixels:
    near-tie pixels (oracle flags), per category (a test transmittance near a
    segment boundary, alpha * G near alpha_min, equal neighbouring depths),
    mismatches off them (must be 0) and the largest mixed relative feature
    error."""
    from oracle import compare
    idx = pix[:, 1].astype(np.int64) * width + pix[:, 0]
    rep = compare.selection_report(ids[idx], np.zeros(ids[idx].shape), counts[idx], ref)
    same, tie = rep["same"], rep["tie"]
    err = compare.feature_error(out[idx], ref.out_q, ref.scale_q)
    flags = np.asarray(ref.tie)
    return {"pixels": rep["pixels"], "near_tie_pixels": rep["tie_pixels"],
            "near_tie_by_category": {"boundary": int(((flags & 1) != 0).sum()),
                                     "alpha_min_border": int(((flags & 2) != 0).sum()),
                                     "equal_depth": int(((flags & 4) != 0).sum())},
            "mismatch_nontie": rep["mismatch_nontie"],
            "feat_err_max": float(err[same].max()) if same.any() else None}


def tile_distinct_rows(ids, width, tile_w, tile_h):
    """U_tile: the sum over screen tiles of the distinct Gaussians selected in
    the tile (each row read once per tile with perfect in-tile reuse), the
    reuse diagnostic beside U (each row read once per frame)."""
    import torch
    P, K = ids.shape
    pix = torch.arange(P, device=ids.device)
    tiles_x = (width + tile_w - 1) // tile_w
    tile = (pix // width // tile_h) * tiles_x + (pix % width) // tile_w
    key = tile[:, None].to(torch.int64) * (1 << 32) + ids.to(torch.int64)
    return int(torch.unique(key[ids >= 0]).numel())


# --------------------------------------------------------------------------- GPU arm
def run_gpu(args, ws, rank, local):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    g, feat = scenes.room_scene(seed=0, n=N_GAUSS, channels=C)
    cam = scenes.room_camera(WIDTH, HEIGHT)
    gdev = tuple(t.to(dev) for t in q.gaussians_to_device(g, device="cpu"))
    fdev = torch.from_numpy(feat).to(dev)

    def frame_for(k):
        res = q.render_frame(gdev, fdev, cam, K=k, dense=True)
        fr = res["frame"]
        return fr, res

    fr, res = frame_for(K)
    P = fr.pixels
    ids, w, cnt, out = res["ids"], res["weights"], res["counts"], res["out"]
    dout, tf = res["dense"], res["T_final"]
    U = int(torch.unique(ids[ids >= 0]).numel())
    U_tile = tile_distinct_rows(ids, WIDTH, 16, 16)
    sel_per_px = float(cnt.float().mean().item())

    def q_frame():
        q.qr_project(fr, *gdev)
        q.qr_sort(fr)
        q.qr_select(fr, ids, w, cnt)
        q.qr_blend(fdev, None, ids, w, cnt, out)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- eager steps with per-stage events (warm-up, then timed)
    for _ in range(args.warmup):
        q_frame()
    barrier()
    nev = 4
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(args.steps)]
    launches0 = q.qr_launch_count()
    # clocks are sampled from before the eager timed steps to after the graph-timed ones
    clk = ClockSampler(local)
    clk.__enter__()
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        e = evs[s]
        e[0].record(stream)
        q.qr_project(fr, *gdev)
        q.qr_sort(fr)
        e[1].record(stream)
        q.qr_select(fr, ids, w, cnt)
        e[2].record(stream)
        q.qr_blend(fdev, None, ids, w, cnt, out)
        e[3].record(stream)
    t_end.record(stream)
    barrier()
    launches = q.qr_launch_count() - launches0
    eager_ms = t_start.elapsed_time(t_end) / args.steps
    st = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(3)] for e in evs])
    stage_ms = st.mean(axis=0)
    blend_ms = float(stage_ms[2])
    if args.profile:
        clk.__exit__(None, None, None)
        return {"profile": True, "eager_ms_per_step": eager_ms, "stages_ms": stage_ms.tolist(),
                "gpu_launches": int(launches)}

    # ---- the same frame replayed from a captured CUDA graph
    graph_ms = None
    graph_repeats = 0
    try:
        gstream = torch.cuda.Stream()
        gstream.wait_stream(stream)
        with torch.cuda.stream(gstream):
            q_frame()
        stream.wait_stream(gstream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            q_frame()
        for _ in range(args.warmup):
            graph.replay()
        barrier()
        # the K timed steps are repeated (each repeat timed on its own) until the
        # repeats span about a second, so the clock sampler sees the timed region;
        # the step time is the median repeat
        reps, t_all = [], 0.0
        while t_all < 1000.0 and len(reps) < 200:
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record()
            for _ in range(args.steps):
                graph.replay()
            g1.record()
            barrier()
            r_ms = g0.elapsed_time(g1)
            reps.append(r_ms / args.steps)
            t_all += r_ms
        graph_ms = float(np.median(reps))
        graph_repeats = len(reps)
    except Exception as exc:  # noqa: BLE001 - report and keep the eager number
        print(f"# graph capture unavailable: {exc}", file=sys.stderr)
    clk.__exit__(None, None, None)

    step_ms = min(eager_ms, graph_ms) if graph_ms else eager_ms

    # ---- dense Eq. 1 frame on the same GPU
    def d_frame():
        q.qr_project(fr, *gdev)
        q.qr_sort(fr)
        q.qr_dense(fr, fdev, None, dout, tf)
    for _ in range(2):
        d_frame()
    torch.cuda.synchronize()
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    nd = max(3, args.steps // 4)
    d0.record()
    for _ in range(nd):
        d_frame()
    d1.record()
    torch.cuda.synchronize()
    dense_ms = d0.elapsed_time(d1) / nd
    # the dense kernel alone, and its work (useful: C multiply-adds per blended
    # (pixel, Gaussian) pair; executed: as the kernel counts them)
    dk_ms = _time_ms(lambda: q.qr_dense(fr, fdev, None, dout, tf), max(3, args.steps // 4))
    wc = q.qr_dense_work(fr, fdev, None, dout, tf).cpu().numpy()
    props = torch.cuda.get_device_properties(dev)
    sm_clock_mhz = 2070.0
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_clock_mhz * 1e6 / 1e12
    useful = 2.0 * C * float(wc[0])
    executed = 2.0 * float(wc[1])
    dense_info = {"kernel_ms": round(dk_ms, 4), "frame_ms": round(dense_ms, 4),
                  "blended_pairs": int(wc[0]),
                  "useful_tflop": round(useful / 1e12, 4),
                  "executed_tflop": round(executed / 1e12, 4),
                  "useful_TFLOP_per_s": round(useful / dk_ms / 1e9, 2),
                  "roofline": {"bound": "alu", "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                               "frac_useful": round(useful / dk_ms / 1e9 / fp32_peak, 4),
                               "frac_executed": round(executed / dk_ms / 1e9 / fp32_peak, 4),
                               "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 "
                                              f"lanes x 2 flops x {sm_clock_mhz:.0f} MHz"}}

    # ---- K = 4 and 16
    per_k = {}
    for k2 in (4, 16):
        fr2, r2 = frame_for(k2)
        a = (r2["ids"], r2["weights"], r2["counts"], r2["out"])

        def f2():
            q.qr_project(fr2, *gdev)
            q.qr_sort(fr2)
            q.qr_select(fr2, a[0], a[1], a[2])
            q.qr_blend(fdev, None, a[0], a[1], a[2], a[3])
        for _ in range(2):
            f2()
        torch.cuda.synchronize()
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record()
        for _ in range(max(3, args.steps // 4)):
            f2()
        k1.record()
        torch.cuda.synchronize()
        per_k[str(k2)] = round(1000.0 / (k0.elapsed_time(k1) / max(3, args.steps // 4)), 2)
        del fr2, r2, a
    per_k[str(K)] = round(1000.0 / step_ms, 2)

    # ---- end to end through the host-buffer C-ABI call: every step uploads the
    # Gaussians and the feature table from pinned host memory, renders, and
    # downloads the map.  Consecutive steps rotate over NB streams (each with
    # its own frame and device buffers), so one step's upload overlaps earlier
    # steps' downloads on the full-duplex host link.
    e2e = None
    e2e_ms = None
    try:
        nin, nout = q.qr_render_host_bytes(N_GAUSS, WIDTH, HEIGHT, K, C, q.QR_F32)
        NB = 3
        frames = [fr] + [frame_for(K)[0] for _ in range(NB - 1)]
        dins = [torch.empty(nin + 256, dtype=torch.uint8, device=dev) for _ in range(NB)]
        douts = [torch.empty(nout + 256, dtype=torch.uint8, device=dev) for _ in range(NB)]

        class _Aligned:
            def __init__(self, t):
                self.p = (t.data_ptr() + 255) // 256 * 256

            def data_ptr(self):
                return self.p
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()  # noqa: E731
        hm, hl, hq, ho, hf = (pin(g.mean), pin(g.log_scale), pin(g.quat), pin(g.opacity), pin(feat))
        houts = [torch.empty((P, C), dtype=torch.float32).pin_memory() for _ in range(NB)]
        side = [torch.cuda.Stream(device=dev) for _ in range(NB)]

        def e2e_run(nsteps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s in side:
                s.wait_event(e0)
            for i in range(nsteps):
                b = i % NB
                q.qr_render_host(frames[b], hm, hl, hq, ho, hf, None, q.QR_F32, C,
                                 _Aligned(dins[b]), _Aligned(douts[b]), houts[b], stream=side[b])
            for s in side:
                done = torch.cuda.Event()
                done.record(s)
                stream.wait_event(done)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        e2e_run(4)
        ne = max(4, args.steps // 4)
        e2e_ms = e2e_run(ne) / ne
        # the public call renders in screen-tile pixel order; the device-resident
        # steps above use row order, which sums a pixel's rows in another order
        np.testing.assert_allclose(houts[(ne - 1) % NB][:64].numpy(), out[:64].cpu().numpy(),
                                   rtol=1e-5, atol=1e-7)
    except Exception as exc:  # noqa: BLE001
        print(f"# e2e failed: {exc}", file=sys.stderr)

    # ---- max over ranks (a rank whose e2e leg failed reports -1)
    step_ms, eager_ms, blend_ms, dense_ms, e2e_max = max_over_ranks(
        [step_ms, eager_ms, blend_ms, dense_ms, e2e_ms if e2e_ms is not None else -1.0], ws, dev)
    e2e_fail = max_over_ranks([0.0 if e2e_ms is not None else 1.0], ws, dev)[0] > 0
    if not e2e_fail:
        e2e = {"value": round(whole_job_rate(ws, e2e_max), 3), "unit": "frames/s",
               "h2d_bytes_per_step": N_GAUSS * 11 * 4 + N_GAUSS * C * 4,
               "d2h_bytes_per_step": P * C * 4}

    hbm_peak, peak_src = _peaks()
    alg_bytes = U * C * 4 + P * K * 8 + P + P * C * 4
    achieved = alg_bytes / (blend_ms * 1e-3) / 1e9
    traffic = _traffic_from_profile()
    clocks = clk.summary()
    ctx = {"fr": fr, "gdev": gdev, "fdev": fdev, "ids": ids, "w": w, "cnt": cnt, "out": out,
           "U": U}
    return {
        "_ctx": ctx, "graph_repeats": graph_repeats,
        "value": round(whole_job_rate(ws, step_ms), 3),
        "ms_per_step": round(step_ms, 4),
        "eager_ms_per_step": round(eager_ms, 4),
        "graph_ms_per_step": round(graph_ms, 4) if graph_ms else None,
        "dense_fps": round(whole_job_rate(ws, dense_ms), 3),
        "dense": dense_info,
        "speedup_vs_dense": round(dense_ms / step_ms, 3),
        "per_k_fps": per_k,
        "stages_ms": {"project+sort": round(float(stage_ms[0]), 4),
                      "select": round(float(stage_ms[1]), 4),
                      "blend": round(float(stage_ms[2]), 4)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": e2e,
        "roofline": {"bound": "hbm", "kernel": "blend (Algorithm 1 gather)",
                     "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "peak_source": peak_src,
                     "traffic": traffic, "algorithmic_bytes": int(alg_bytes),
                     "distinct_rows": U, "distinct_rows_per_tile_sum": U_tile,
                     "selected_per_px": round(sel_per_px, 3)},
        "_g": g, "_feat": feat, "_cam": cam,
    }


def _time_ms(fn, steps, warmup=2):
    """Mean CUDA-event milliseconds of fn() over `steps` calls on the current
    stream, after `warmup` untimed calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_rules(ctx, steps=20):
    """The paper's other select rules on the headline frame: top-K (Sec. 4.2,
    complexity table), Stratified-K (App. E) and Algorithm 1 with App. C's
    Riemann weights, each a whole frame (project, sort, the rule's selection,
    blend), K = 8, beside Algorithm 1 and dense."""
    from paper_2512_20927_gb300 import qrender as q
    fr, gdev, fdev, ids, w, cnt, out = (ctx[k] for k in ("fr", "gdev", "fdev", "ids", "w", "cnt",
                                                          "out"))
    res = {}
    for name, rule in (("topk", q.QR_RULE_TOPK), ("stratified", q.QR_RULE_STRATIFIED),
                       ("riemann", q.QR_RULE_RIEMANN)):
        def frame():
            q.qr_project(fr, *gdev)
            q.qr_sort(fr)
            q.qr_select_rule(fr, rule, ids, w, cnt)
            q.qr_blend(fdev, None, ids, w, cnt, out)
        ms = _time_ms(frame, steps)
        sel = _time_ms(lambda: q.qr_select_rule(fr, rule, ids, w, cnt), steps)
        res[name] = {"fps": round(1000.0 / ms, 2), "ms": round(ms, 4),
                     "select_ms": round(sel, 4),
                     "selected_per_px": round(float(cnt.float().mean().item()), 3)}
    # restore the Algorithm 1 selection of the frame
    q.qr_select(fr, ids, w, cnt)
    return res


def run_fused_relevance(ctx, hbm_peak, steps=20):
    """Relevance of the headline frame's Q-Render map against 64 unit BF16
    queries: blend then the TMA/tcgen05 relevance kernel (the map written and
    read back) against the fused blend + relevance kernel (no map)."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    fdev, ids, w, cnt, out, fr = (ctx[k] for k in ("fdev", "ids", "w", "cnt", "out", "fr"))
    P = fr.pixels
    Qn = 64
    qbits = q.qr_quantize_bf16(torch.from_numpy(scenes.unit_queries(7, Qn, C)).to(fdev.device))
    qbits = qbits.view(torch.int16)
    two = _time_ms(lambda: (q.qr_blend(fdev, None, ids, w, cnt, out),
                            q.qr_relevance(out, qbits)), steps)
    fused = _time_ms(lambda: q.qr_blend_relevance(fdev, None, ids, w, cnt, qbits, width=fr.width),
                     steps)
    U = ctx["U"]
    fused_bytes = U * C * 4 + P * K * 8 + P + P * Qn * 4
    return {"queries": Qn, "two_step_ms": round(two, 4), "fused_ms": round(fused, 4),
            "speedup": round(two / fused, 3),
            "fused_algorithmic_bytes": int(fused_bytes),
            "fused_GB_per_s": round(fused_bytes / fused / 1e6, 1),
            "fused_frac_of_hbm": round(fused_bytes / fused / 1e6 / hbm_peak, 4),
            "map_bytes_not_written": int(P * C * 4),
            "note": "fused: the blend of each 16x8 pixel block goes to shared memory and "
                    "through tcgen05 kind::tf32; the 512-D map never reaches HBM"}


def run_object(local, hbm_peak, steps=20):
    """Object-centric 512-D workload: 500k Gaussians around a unit sphere seen
    from outside, 640x480, FP32 features, K = 8.  Every pixel gathers rows of
    its own patch of surface, so the blend reads many distinct rows (large U)."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    dev = torch.device("cuda", local)
    g, feat = scenes.object_scene(seed=0, n=N_GAUSS, channels=C)
    cam = scenes.object_camera(WIDTH, HEIGHT)
    gdev = tuple(t.to(dev) for t in q.gaussians_to_device(g, device="cpu"))
    fdev = torch.from_numpy(feat).to(dev)
    del feat
    res = q.render_frame(gdev, fdev, cam, K=K)
    fr, ids, w, cnt, out = res["frame"], res["ids"], res["weights"], res["counts"], res["out"]
    P = fr.pixels
    U = int(torch.unique(ids[ids >= 0]).numel())

    def frame():
        q.qr_project(fr, *gdev)
        q.qr_sort(fr)
        q.qr_select(fr, ids, w, cnt)
        q.qr_blend(fdev, None, ids, w, cnt, out)
    ms = _time_ms(frame, steps)
    blend_ms = _time_ms(lambda: q.qr_blend(fdev, None, ids, w, cnt, out), steps)
    alg = U * C * 4 + P * K * 8 + P + P * C * 4
    return {"workload": "object-centric FP32: 500k Gaussians (70 % within 1 cm of a unit sphere, "
                        "30 % inside), 640x480 from 2.6 m, 512-D, Q-Render K=8",
            "fps": round(1000.0 / ms, 2), "ms": round(ms, 4), "blend_ms": round(blend_ms, 4),
            "distinct_rows": U,
            "distinct_rows_per_tile_sum": tile_distinct_rows(ids, fr.width, 16, 16),
            "selected_per_px": round(float(cnt.float().mean().item()), 3),
            "n_isect": int(res["n_isect"]),
            "blend_roofline": {"achieved": round(alg / blend_ms / 1e6, 1), "peak": hbm_peak,
                               "unit": "GB/s", "frac": round(alg / blend_ms / 1e6 / hbm_peak, 4),
                               "algorithmic_bytes": int(alg)}}


def run_precision(local, hbm_peak, steps=10, sample_px=160):
    """Precision configuration: 1M room Gaussians, 1296x968, K = 8, the
    feature table in FP32, BF16 and FP8 E4M3 with per-row scales: frames/s,
    the blend's roofline, and the max / mean mixed relative error of sampled
    pixels against the FP64 oracle on the FP32 features."""
    import torch
    import oracle
    from oracle import compare
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    dev = torch.device("cuda", local)
    W_, H_, N_ = 1296, 968, 1_000_000
    g, feat = scenes.room_scene(seed=0, n=N_, channels=C)
    cam = scenes.room_camera(W_, H_)
    gdev = tuple(t.to(dev) for t in q.gaussians_to_device(g, device="cpu"))
    f32 = torch.from_numpy(feat).to(dev)
    tables = {"f32": (f32, None, 4), "bf16": (q.qr_quantize_bf16(f32), None, 2)}
    codes, scale = q.qr_quantize_fp8(f32)
    tables["fp8"] = (codes, scale, 1)
    rng = np.random.default_rng(5)
    pix = np.stack([rng.integers(0, W_, sample_px), rng.integers(0, H_, sample_px)], 1).astype(np.int32)
    pr = oracle.project(g, cam.as_array())
    ref = oracle.render(pr, feat, K, pix, want_dense=False, alpha_min=oracle.ALPHA_MIN_F32,
                        alpha_max=oracle.ALPHA_MAX_F32)
    idx = pix[:, 1].astype(np.int64) * W_ + pix[:, 0]
    tie = (ref.tie & compare.Q_TIE_BITS) != 0
    out = {"workload": "precision: 1M room Gaussians, 1296x968, 512-D, K=8",
           "sample_pixels": sample_px, "near_tie_pixels": int(tie.sum())}
    res = None
    for name, (table, sc, bf) in tables.items():
        res = q.render_frame(gdev, (table, sc) if sc is not None else table, cam, K=K)
        fr, ids, w, cnt, o = res["frame"], res["ids"], res["weights"], res["counts"], res["out"]
        P = fr.pixels

        def frame():
            q.qr_project(fr, *gdev)
            q.qr_sort(fr)
            q.qr_select(fr, ids, w, cnt)
            q.qr_blend(table, sc, ids, w, cnt, o)
        ms = _time_ms(frame, steps)
        bms = _time_ms(lambda: q.qr_blend(table, sc, ids, w, cnt, o), steps)
        U = int(torch.unique(ids[ids >= 0]).numel())
        alg = U * (C * bf + (4 if name == "fp8" else 0)) + P * K * 8 + P + P * C * 4
        got = o.cpu().numpy()[idx]
        same = (ids.cpu().numpy()[idx] == ref.ids).all(axis=1)
        ok = same & ~tie
        err = compare.feature_error(got, ref.out_q, ref.scale_q)[ok]
        out[name] = {"fps": round(1000.0 / ms, 2), "blend_ms": round(bms, 4),
                     "blend_frac_of_hbm": round(alg / bms / 1e6 / hbm_peak, 4),
                     "err_vs_fp64_max": float(err.max()) if err.size else None,
                     "err_vs_fp64_mean": float(err.mean()) if err.size else None,
                     "selection_mismatch_nontie": int((~same & ~tie).sum())}
        del res, o
        torch.cuda.empty_cache()
    return out


def run_train_eq2(local, steps=10, masks=32):
    """Differentiation workload with the paper's loss, Eq. 2: forward, then
    the contrastive loss against 32 synthetic patches (Voronoi cells with
    random unit embeddings) and the backward to features and opacities,
    replayed from a CUDA graph on fixed buffers."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    dev, cam, gd, table, _ = _train_workload(local)
    r0 = q.render_frame(gd, table, cam, K=K, max_isect=2_000_000)
    fr, ids, w, cnt, out = r0["frame"], r0["ids"], r0["weights"], r0["counts"], r0["out"]
    mid = torch.from_numpy(scenes.patch_masks(cam.width, cam.height, masks, seed=2)).to(dev)
    tg = torch.from_numpy(scenes.patch_targets(masks, C, seed=5)).to(dev)
    keep = {}

    def step():
        q.qr_project(fr, *gd)
        q.qr_sort(fr)
        q.qr_select(fr, ids, w, cnt)
        q.qr_blend(table, None, ids, w, cnt, out)
        keep["loss"] = q.qr_contrastive_backward(fr, table, None, ids, w, cnt, out, tg, mid,
                                                 want_conic=False)[0]
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    ms = _time_ms(graph.replay, steps, warmup=3)
    loss_ms = _time_ms(lambda: q.qr_contrastive_loss(out, tg, mid), steps)
    return {"graph_ms_per_step": round(ms, 4), "steps_per_s": round(1000.0 / ms, 2),
            "masks": masks, "loss": round(float(keep["loss"].item()), 6),
            "eq2_loss_and_grad_ms": round(loss_ms, 4),
            "note": "forward + Eq. 2 loss (its dL/dF written once) + backward, 300k room, "
                    "BF16 512-D, 640x480, K=8"}


def run_config_table(local, headline, precision, budget_s=4.0):
    """The configuration table: GPU and FP64-oracle frames/s of Q-Render (K = 8)
    and dense Eq. 1 for the tiny, indoor and precision configurations, and the
    blend's fraction of the measured HBM bandwidth.  Oracle: tiny frames are
    rendered whole; indoor and precision frames are extrapolated from a
    random pixel sample (each about budget_s seconds of host time)."""
    import torch
    import oracle
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    dev = torch.device("cuda", local)
    hbm, _ = _peaks()
    cores = os.cpu_count() or 1

    def oracle_fps(g, feat, cam, dense, whole):
        pr = oracle.project(g, cam.as_array())
        P = cam.width * cam.height
        rng = np.random.default_rng(1)
        kw = dict(want_q=not dense, want_dense=dense, threads=cores,
                  alpha_min=oracle.ALPHA_MIN_F32, alpha_max=oracle.ALPHA_MAX_F32)
        if whole:
            pix = oracle.all_pixels(cam.width, cam.height)
        else:
            pix = np.stack([rng.integers(0, cam.width, 2 * cores),
                            rng.integers(0, cam.height, 2 * cores)], 1).astype(np.int32)
            t0 = time.perf_counter()
            oracle.render(pr, feat, K, pix, **kw)
            per = (time.perf_counter() - t0) / len(pix)
            n = int(max(cores, min(P, budget_s / max(per, 1e-9))))
            pix = np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], 1).astype(np.int32)
        t0 = time.perf_counter()
        oracle.render(pr, feat, K, pix, **kw)
        return 1.0 / ((time.perf_counter() - t0) * P / len(pix))

    rows = {}
    # tiny: 2,000 Gaussians, 128x128, 16-D
    g, f = scenes.tiny_scene()
    cam = scenes.tiny_camera()
    gd = q.gaussians_to_device(g, device=dev)
    fd = torch.from_numpy(f).to(dev)
    r = q.render_frame(gd, fd, cam, K=K, dense=True)
    fr, ids, w, cnt, o = r["frame"], r["ids"], r["weights"], r["counts"], r["out"]

    def qf():
        q.qr_project(fr, *gd)
        q.qr_sort(fr)
        q.qr_select(fr, ids, w, cnt)
        q.qr_blend(fd, None, ids, w, cnt, o)

    def df():
        q.qr_project(fr, *gd)
        q.qr_sort(fr)
        q.qr_dense(fr, fd, None, r["dense"], r["T_final"])
    rows["tiny"] = {"gpu_q_fps": round(1000.0 / _time_ms(qf, 50), 1),
                    "gpu_dense_fps": round(1000.0 / _time_ms(df, 50), 1),
                    "oracle_q_fps": round(oracle_fps(g, f, cam, False, True), 3),
                    "oracle_dense_fps": round(oracle_fps(g, f, cam, True, True), 3),
                    "oracle_frames": "whole 128x128 frames"}
    # indoor: the headline frame
    g, f = scenes.room_scene(seed=0, n=N_GAUSS, channels=C)
    cam = scenes.room_camera(WIDTH, HEIGHT)
    rows["indoor"] = {"gpu_q_fps": headline["per_k_fps"], "gpu_dense_fps": headline["dense_fps"],
                      "oracle_q_fps": round(oracle_fps(g, f, cam, False, False), 5),
                      "oracle_dense_fps": round(oracle_fps(g, f, cam, True, False), 5),
                      "blend_frac_of_hbm": headline["roofline"]["frac"],
                      "oracle_frames": "extrapolated from a random pixel sample"}
    del g, f
    # precision: 1M room, 1296x968
    g, f = scenes.room_scene(seed=0, n=1_000_000, channels=C)
    cam = scenes.room_camera(1296, 968)
    prow = {"oracle_q_fps": round(oracle_fps(g, f, cam, False, False), 6),
            "oracle_dense_fps": round(oracle_fps(g, f, cam, True, False), 6),
            "oracle_frames": "extrapolated from a random pixel sample"}
    if isinstance(precision, dict):
        for dt in ("f32", "bf16", "fp8"):
            if isinstance(precision.get(dt), dict):
                prow[f"gpu_q_fps_{dt}"] = precision[dt].get("fps")
                prow[f"blend_frac_of_hbm_{dt}"] = precision[dt].get("blend_frac_of_hbm")
    gd = q.gaussians_to_device(g, device=dev)
    fd = torch.from_numpy(f).to(dev)
    del f
    r = q.render_frame(gd, fd, cam, K=K, dense=True)
    fr = r["frame"]
    prow["gpu_dense_fps_f32"] = round(1000.0 / _time_ms(
        lambda: (q.qr_project(fr, *gd), q.qr_sort(fr), q.qr_dense(fr, fd, None, r["dense"], r["T_final"])),
        5), 2)
    rows["precision"] = prow
    rows["oracle_cores"] = cores
    return rows


def run_batched(local, steps=3):
    """Many-view workload: 4 rooms (200k, 500k, 1M, 2M Gaussians), 32 views from
    320x240 to 1296x968, 512-D BF16 features, K = 8, autotuned tile shape and
    pixel group, one graph per batch (per-view projection and binning, one
    persistent select+blend launch, relevance against 64 BF16 queries)."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    from paper_2512_20927_gb300.batch import Scene, autotune, time_batch
    dev = torch.device("cuda", local)
    sc = []
    for seed, n in enumerate((200_000, 500_000, 1_000_000, 2_000_000)):
        g, f = scenes.room_scene(seed=seed, n=n, channels=C)
        gd = tuple(t.to(dev) for t in q.gaussians_to_device(g, device="cpu"))
        sc.append(Scene(gd, q.qr_quantize_bf16(torch.from_numpy(f).to(dev))))
        del f
    views = scenes.batched_views(seed=0, n_views=32, scenes=4)
    qbits = q.qr_quantize_bf16(torch.from_numpy(scenes.unit_queries(7, 64, C)).to(dev))
    qbits = qbits.view(torch.int16)
    best, timings = autotune(sc, views, K=K, queries=qbits, steps=steps)
    ms = time_batch(best, steps=max(steps, 3))
    pixels = int(best.offsets[-1])
    # relevance alone, for its own roofline (BF16 operands read from an FP32 map)
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record()
    for _ in range(3):
        best.relevance()
    r1.record()
    torch.cuda.synchronize()
    rel_ms = r0.elapsed_time(r1) / 3
    rel_bytes = pixels * C * 4 + pixels * 64 * 4
    rel_flops = 2.0 * pixels * C * 64
    # the persistent select + blend launch alone: bytes written (the FP32 map,
    # ids, weights, counts); the feature rows it reads are not counted
    sb_ms = _time_ms(best.select_blend, 5)
    sb_bytes = pixels * C * 4 + pixels * K * 8 + pixels
    hbm = _peaks()[0]
    return {"views": len(views), "pixels": pixels, "ms_per_batch": round(ms, 3),
            "views_per_s": round(len(views) * 1000.0 / ms, 2),
            "mpixels_per_s": round(pixels / ms / 1000.0, 1),
            "autotune_ms": timings,
            "chosen": {"tile": list(best.tile), "group": best.group, "chunks": best.chunks,
                       "blend_warps": best.blend_warps or 8},
            "select_blend": {"ms": round(sb_ms, 4), "GB_per_s": round(sb_bytes / sb_ms / 1e6, 1),
                             "frac_of_hbm": round(sb_bytes / sb_ms / 1e6 / hbm, 4),
                             "bytes": sb_bytes, "bytes_counted": "map + ids + weights + counts written"},
            "relevance": {"ms": round(rel_ms, 4), "GB_per_s": round(rel_bytes / rel_ms / 1e6, 1),
                          "TFLOP_per_s": round(rel_flops / rel_ms / 1e9, 1)}}


def _train_workload(local):
    """Differentiation workload: 300k-Gaussian room, 512-D BF16 features,
    640x480, K = 8, and the target map: the dense render of a second Gaussian
    set."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    dev = torch.device("cuda", local)
    g, f = scenes.room_scene(seed=0, n=300_000, channels=C)
    g2, f2 = scenes.room_scene(seed=1, n=300_000, channels=C)
    cam = scenes.room_camera(WIDTH, HEIGHT)
    gd = tuple(t.to(dev) for t in q.gaussians_to_device(g, device="cpu"))
    table = q.qr_quantize_bf16(torch.from_numpy(f).to(dev))
    g2d = tuple(t.to(dev) for t in q.gaussians_to_device(g2, device="cpu"))
    tgt = q.render_frame(g2d, torch.from_numpy(f2).to(dev), cam, K=K, dense=True)["dense"]
    return dev, cam, gd, table, tgt


def profile_train(local, steps=3):
    """Forward + loss + backward of the differentiation workload on fixed
    buffers, eager (for ncu launch lists)."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    dev, cam, gd, table, tgt = _train_workload(local)
    r0 = q.render_frame(gd, table, cam, K=K, max_isect=2_000_000)
    fr, ids, w, cnt, out = r0["frame"], r0["ids"], r0["weights"], r0["counts"], r0["out"]
    for _ in range(steps):
        q.qr_project(fr, *gd)
        q.qr_sort(fr)
        q.qr_select(fr, ids, w, cnt)
        q.qr_blend(table, None, ids, w, cnt, out)
        loss = q.qr_cosine_backward(fr, table, None, ids, w, cnt, out, tgt, want_conic=False)[0]
    torch.cuda.synchronize()
    return {"profile": "train", "steps": steps, "loss": round(float(loss.item()), 6)}


def run_train_step(local, steps=10):
    """Differentiation workload (see _train_workload): forward + mean (1 - cos)
    loss + backward to features and opacities."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    dev, cam, gd, table, tgt = _train_workload(local)

    def step():
        res = q.render_frame(gd, table, cam, K=K, max_isect=2_000_000)
        loss = q.qr_cosine_backward(res["frame"], table, None, res["ids"], res["weights"],
                                    res["counts"], res["out"], tgt, want_conic=False)[0]
        return loss
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        loss = step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000.0 / steps

    # the same step on a fixed frame and fixed buffers, captured once as a CUDA
    # graph and replayed: what the kernels cost without host work
    r0 = q.render_frame(gd, table, cam, K=K, max_isect=2_000_000)
    fr, ids, w, cnt, out = r0["frame"], r0["ids"], r0["weights"], r0["counts"], r0["out"]
    keep = {}

    def gstep():
        q.qr_project(fr, *gd)
        q.qr_sort(fr)
        q.qr_select(fr, ids, w, cnt)
        q.qr_blend(table, None, ids, w, cnt, out)
        keep["loss"], _, keep["gf"], keep["ga"], _ = q.qr_cosine_backward(
            fr, table, None, ids, w, cnt, out, tgt, want_conic=False)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            gstep()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gstep()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    gms = e0.elapsed_time(e1) / steps
    return {"ms_per_step": round(ms, 3), "steps_per_s": round(1000.0 / ms, 2),
            "loss": round(float(loss.item()), 6),
            "graph_ms_per_step": round(gms, 4), "graph_loss": round(float(keep["loss"].item()), 6),
            "note": "ms_per_step host-timed (workspace allocation and a capacity check per "
                    "step); graph_ms_per_step: forward + loss + backward replayed from a "
                    "CUDA graph on fixed buffers"}


def profile_relevance(local, reps=13):
    """Relevance GEMM alone on a random FP32 map of 524,288 x 512 (1.07 GB,
    larger than L2) against 64 unit BF16 queries: the small case the ncu
    capture of the relevance kernel runs on."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    P_, C_, Q_ = 524288, C, 64
    dev = torch.device("cuda", local)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    fmap = torch.randn(P_, C_, device=dev, generator=g)
    qbits = q.qr_quantize_bf16(torch.from_numpy(scenes.unit_queries(7, Q_, C_)).to(dev)).view(torch.int16)
    for _ in range(3):
        q.qr_relevance(fmap, qbits)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps - 3):
        scores, st = q.qr_relevance(fmap, qbits)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (reps - 3)
    return {"profile": "relevance", "pixels": P_, "channels": C_, "queries": Q_,
            "us": round(ms * 1000, 1), "GB_per_s": round((P_ * C_ * 4 + P_ * Q_ * 4) / ms / 1e6, 1),
            "status": int(st.item())}


def profile_mode(local, mode, steps):
    """Workload set up once, then `steps` eager launches of one part of it, for
    ncu captures: indoor / object (a whole Q-Render frame: project, sort,
    select, blend), blend, fused (blend + relevance in one kernel), eq2 (the
    Eq. 2 loss and its gradient, 32 patches), rules (top-K, Stratified-K,
    then Riemann-weight selection), dense (Eq. 1), blend_bf16 / blend_fp8 (the blend from a BF16
    table / FP8 E4M3 codes with per-Gaussian scales, tile-ordered pixel
    groups) -- on the 500k indoor room (object: the object
    scene), 640x480, 512-D FP32, K = 8; batch: the many-view launch on a small
    batch (see below)."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    dev = torch.device("cuda", local)
    if mode == "batch":
        # a small many-view batch (2 rooms of 200k and 500k Gaussians, 4 views of
        # 640x480, BF16 512-D, K = 8, 16x16 tiles, built-in pixel groups and
        # channel chunks): the fused
        # select + blend launch alone
        from paper_2512_20927_gb300.batch import Batch, Scene
        sc = []
        for seed, n in enumerate((200_000, 500_000)):
            g, f = scenes.room_scene(seed=seed, n=n, channels=C)
            gd = tuple(t.to(dev) for t in q.gaussians_to_device(g, device="cpu"))
            sc.append(Scene(gd, q.qr_quantize_bf16(torch.from_numpy(f).to(dev))))
            del f
        views = [(i % 2, scenes.room_camera(WIDTH, HEIGHT, yaw=0.8 * i)) for i in range(4)]
        b = Batch(sc, views, K=K, tile=(16, 16))
        b.project_sort()
        torch.cuda.synchronize()
        for _ in range(steps):
            b.select_blend()
        torch.cuda.synchronize()
        return {"profile": mode, "steps": steps, "pixels": int(b.offsets[-1])}
    if mode == "object":
        g, feat = scenes.object_scene(seed=0, n=N_GAUSS, channels=C)
        cam = scenes.object_camera(WIDTH, HEIGHT)
    else:
        g, feat = scenes.room_scene(seed=0, n=N_GAUSS, channels=C)
        cam = scenes.room_camera(WIDTH, HEIGHT)
    gd = tuple(t.to(dev) for t in q.gaussians_to_device(g, device="cpu"))
    fd = torch.from_numpy(feat).to(dev)
    del feat
    r = q.render_frame(gd, fd, cam, K=K)
    fr, ids, w, cnt, o = r["frame"], r["ids"], r["weights"], r["counts"], r["out"]
    qb = q.qr_quantize_bf16(torch.from_numpy(scenes.unit_queries(7, 64, C)).to(dev)).view(torch.int16)
    mid = torch.from_numpy(scenes.patch_masks(WIDTH, HEIGHT, 32, seed=2)).to(dev)
    tg = torch.from_numpy(scenes.patch_targets(32, C, seed=5)).to(dev)
    dout = torch.empty_like(o)
    tf = torch.empty(fr.pixels, device=dev)
    tab, tsc = fd, None
    if mode == "blend_bf16":
        tab = q.qr_quantize_bf16(fd)
    elif mode == "blend_fp8":
        tab, tsc = q.qr_quantize_fp8(fd)
    torch.cuda.synchronize()
    for _ in range(steps):
        if mode in ("indoor", "object"):
            q.qr_project(fr, *gd)
            q.qr_sort(fr)
            q.qr_select(fr, ids, w, cnt)
            q.qr_blend(fd, None, ids, w, cnt, o)
        elif mode == "blend":
            q.qr_blend(fd, None, ids, w, cnt, o)
        elif mode in ("blend_bf16", "blend_fp8"):
            q.qr_blend(tab, tsc, ids, w, cnt, o)
        elif mode == "fused":
            q.qr_blend_relevance(fd, None, ids, w, cnt, qb, width=fr.width)
        elif mode == "eq2":
            q.qr_contrastive_loss(o, tg, mid)
        elif mode == "rules":
            q.qr_select_rule(fr, q.QR_RULE_TOPK, ids, w, cnt)
            q.qr_select_rule(fr, q.QR_RULE_STRATIFIED, ids, w, cnt)
            q.qr_select_rule(fr, q.QR_RULE_RIEMANN, ids, w, cnt)
        elif mode == "dense":
            q.qr_dense(fr, fd, None, dout, tf)
    torch.cuda.synchronize()
    return {"profile": mode, "steps": steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="only set up the frame and run the eager steps (for ncu captures)")
    ap.add_argument("--profile-train", action="store_true",
                    help="only run eager training steps of the differentiation workload (for ncu)")
    ap.add_argument("--profile-relevance", action="store_true",
                    help="only run the relevance GEMM on a 1.07 GB map (for ncu captures)")
    ap.add_argument("--profile-mode", default=None,
                    choices=["indoor", "object", "blend", "blend_bf16", "blend_fp8", "fused", "eq2",
                             "rules", "dense", "batch"],
                    help="set up one workload and run --steps eager launches of one part (for ncu)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the many-view and training-step measurements")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = _dist()
    n = max(args.gpus, ws)

    if args.impl == "reference":
        # The reference arm is the FP64 CPU oracle (this paper ships no code).
        if rank != 0:
            return
        from paper_2512_20927_gb300 import scenes
        g, feat = scenes.room_scene(seed=0, n=N_GAUSS, channels=C)
        feat = feat.astype(np.float64)
        cam = scenes.room_camera(WIDTH, HEIGHT)
        per_step = max(0.25, min(args.cpu_budget, 120.0 / max(args.steps + args.warmup, 1)))
        vals, samples, timed = [], [], []
        proj = None
        for s in range(args.warmup + args.steps):
            fps, cores, npx, secs = oracle_frames_per_s(g, feat, cam, per_step, seed=s, proj=proj)
            proj = oracle_frames_per_s.last_proj
            if s >= args.warmup:
                vals.append(fps)
                samples.append(npx)
                timed.append(secs)
        v = float(np.median(vals))
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s",
            "n_gpus": n, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(n),
            "ms_per_step_extrapolated": True,
            "timed_s_per_step": round(float(np.median(timed)), 3),
            "note": "each step renders a random pixel sample of the frame with the FP64 oracle "
                    "and scales its time to the whole frame; ms_per_step is that extrapolated "
                    "frame time, not the time the step took (timed_s_per_step)",
            "cpu_baseline": {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"{int(np.median(samples))} random pixels per step of the "
                                       "640x480 frame, brute force over all 500k Gaussians"},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return

    if args.profile_mode:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(profile_mode(local, args.profile_mode, args.steps)))
        return
    if args.profile_relevance or args.profile_train:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(profile_relevance(local) if args.profile_relevance else profile_train(local)))
        return
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    r = run_gpu(args, ws, rank, local)
    if args.profile:
        if rank == 0:
            print(json.dumps(r))
        return
    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        fps, cores, npx, secs = oracle_frames_per_s(r["_g"], r["_feat"], r["_cam"], args.cpu_budget)
        cpu = {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
               "sample": f"{npx} random pixels of the 640x480 frame, brute force over all "
                         f"500k Gaussians, plus the full projection ({secs:.1f} s)"}
        ctx = r["_ctx"]
        pix, ref = oracle_frames_per_s.last_sample
        parity = sample_parity(ctx["ids"].cpu().numpy(), ctx["cnt"].cpu().numpy(),
                               ctx["out"].cpu().numpy(), WIDTH, pix, ref)
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": "frames/s", "n_gpus": n,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": config_dict(n),
        }
        for k in ("eager_ms_per_step", "graph_ms_per_step", "graph_repeats", "dense_fps", "dense",
                  "speedup_vs_dense", "per_k_fps", "stages_ms", "gpu_launches", "clocks", "e2e",
                  "roofline"):
            line[k] = r[k]
        line["cpu_baseline"] = cpu
        line["parity_sample"] = parity
        if not args.no_extras and ws == 1:
            hbm_peak, _ = _peaks()
            ctx = r["_ctx"]
            extras = (("rules", lambda: run_rules(ctx)),
                      ("relevance_fused", lambda: run_fused_relevance(ctx, hbm_peak)),
                      ("object", lambda: run_object(local, hbm_peak)),
                      ("precision", lambda: run_precision(local, hbm_peak)),
                      ("batched", lambda: run_batched(local)),
                      ("train_step", lambda: run_train_step(local)),
                      ("train_step_eq2", lambda: run_train_eq2(local)))
            extras = extras + (("config_table",
                                lambda: run_config_table(local, line, line.get("precision"))),)
            for key, fn in extras:
                try:
                    line[key] = fn()
                except Exception as exc:  # noqa: BLE001 - keep the headline line
                    line[key] = {"error": f"{type(exc).__name__}: {exc}"[:200]}
                import torch
                torch.cuda.empty_cache()
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
