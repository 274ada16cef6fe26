"""Many views of several scenes rendered by one persistent launch (C ABI
qr_batch_prepare / qr_render_batch), optionally followed by the relevance GEMM
over all rendered maps, captured as one CUDA graph; plus a small autotuner that
picks the screen-tile shape, the blend's pixel-group size and its per-warp
channel chunk by timing them.

Marshalling and orchestration only: every step runs in libqrender's kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import qrender as q


def _torch():
    import torch
    return torch


@dataclass
class Scene:
    """Device-resident Gaussians and their feature table."""
    gdev: tuple                   # (mean, log_scale, quat, opacity) float32 device tensors
    table: object                 # [N, C] float32 / bfloat16 tensor, or (codes uint8, scale float32)

    @property
    def n(self) -> int:
        return int(self.gdev[0].shape[0])

    @property
    def feat(self):
        return self.table[0] if isinstance(self.table, tuple) else self.table

    @property
    def scale(self):
        return self.table[1] if isinstance(self.table, tuple) else None


@dataclass
class Batch:
    scenes: list
    views: list                   # [(scene index, Camera)]
    K: int = 8
    tile: tuple = (16, 16)
    group: int = 0
    chunks: int = 0               # channel chunks per feature row in the blend (0 = built-in)
    blend_warps: int = 0          # blend warps per CTA beside 4 selection warps (0 = 8)
    ctas_per_sm: int = 0
    queries: object = None        # [Q, C] BF16 bit patterns (int16 tensor) or None
    streams: int = 4              # side streams the per-view projection and binning use
    frames: list = field(default_factory=list)
    graph: object = None

    def __post_init__(self):
        torch = _torch()
        dev = self.scenes[0].gdev[0].device
        self.C = int(self.scenes[0].feat.shape[1])
        self.dtype = q._dtype_code(self.scenes[0].feat)
        params = q.default_params(self.K, tile_w=self.tile[0], tile_h=self.tile[1])
        self.params = params
        sizes = [v[1].width * v[1].height for v in self.views]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        Ptot = int(self.offsets[-1])
        self.out = torch.empty((Ptot, self.C), dtype=torch.float32, device=dev)
        self.ids = torch.empty((Ptot, self.K), dtype=torch.int32, device=dev)
        self.weights = torch.empty((Ptot, self.K), dtype=torch.float32, device=dev)
        self.counts = torch.empty(Ptot, dtype=torch.uint8, device=dev)
        # size each view's intersection lists with one sizing pass
        for si, cam in self.views:
            sc = self.scenes[si]
            cap = max(1 << 16, 8 * sc.n)
            while True:
                fr = q.frame_create(sc.n, cam, params, cap, device=dev)
                q.qr_project(fr, *sc.gdev)
                q.qr_sort(fr)
                code, nis = q.qr_frame_status(fr)
                if code == q.QR_ERR_CAPACITY:
                    cap = int(nis * 1.25) + 4096
                    continue
                q._check(code, "qr_sort")
                break
            if cap > int(nis * 1.5) + 65536:      # shrink an oversized first guess
                fr = q.frame_create(sc.n, cam, params, int(nis * 1.2) + 4096, device=dev)
            self.frames.append(fr)
        self.views_c = (q.qr_view * len(self.views))()
        for i, ((si, cam), fr) in enumerate(zip(self.views, self.frames)):
            sc = self.scenes[si]
            a, b = int(self.offsets[i]), int(self.offsets[i + 1])
            v = self.views_c[i]
            v.frame = ctypes.addressof(fr.frame)
            v.feat = sc.feat.data_ptr()
            v.feat_scale = sc.scale.data_ptr() if sc.scale is not None else None
            v.ids = self.ids[a:b].data_ptr()
            v.weights = self.weights[a:b].data_ptr()
            v.counts = self.counts[a:b].data_ptr()
            v.out = self.out[a:b].data_ptr()
        self.side = [torch.cuda.Stream(device=dev) for _ in range(max(self.streams, 1))]
        nbytes = int(q.load().qr_batch_workspace_bytes(len(self.views)))
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        self.ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        total = ctypes.c_uint32(0)
        q._check(q.load().qr_batch_prepare(self.views_c, len(self.views),
                                           ctypes.c_void_p(self.ws_ptr), nbytes,
                                           ctypes.byref(total), q._stream(None)),
                 "qr_batch_prepare")
        self.total_tiles = int(total.value)
        if self.queries is not None:
            self.scores = torch.empty((Ptot, self.queries.shape[0]), dtype=torch.float32,
                                      device=dev)
            self.rel_status = torch.zeros(1, dtype=torch.int32, device=dev)

    # ---------------------------------------------------------------- work
    def project_sort(self, stream=None):
        """Projection and binning of every view.  The views are independent, so
        they are spread round-robin over the side streams, forked from and
        joined back into `stream` with events (also inside graph capture)."""
        torch = _torch()
        base = stream if stream is not None else torch.cuda.current_stream()
        if len(self.side) <= 1:
            for (si, _), fr in zip(self.views, self.frames):
                q.qr_project(fr, *self.scenes[si].gdev, stream=base)
                q.qr_sort(fr, stream=base)
            return
        fork = torch.cuda.Event()
        fork.record(base)
        for s in self.side:
            s.wait_event(fork)
        for k, ((si, _), fr) in enumerate(zip(self.views, self.frames)):
            s = self.side[k % len(self.side)]
            q.qr_project(fr, *self.scenes[si].gdev, stream=s)
            q.qr_sort(fr, stream=s)
        for s in self.side:
            join = torch.cuda.Event()
            join.record(s)
            base.wait_event(join)

    def select_blend(self, stream=None):
        q._check(q.load().qr_render_batch(ctypes.c_void_p(self.ws_ptr), len(self.views),
                                          self.total_tiles, self.dtype, self.C, self.K,
                                          self.group, self.chunks, self.blend_warps,
                                          self.ctas_per_sm, q._stream(stream)),
                 "qr_render_batch")

    def relevance(self, stream=None):
        if self.queries is None:
            return
        Q = self.queries.shape[0]
        q._check(q.load().qr_relevance(q._ptr(self.out), q._ptr(self.queries), Q, self.C,
                                       self.out.shape[0], q._ptr(self.scores),
                                       q._ptr(self.rel_status), q._stream(stream)),
                 "qr_relevance")

    def step(self, stream=None):
        self.project_sort(stream)
        self.select_blend(stream)
        self.relevance(stream)

    def status(self):
        """Device status of every view (QR_OK or QR_ERR_CAPACITY) and of the GEMM."""
        codes = [q.qr_frame_status(fr)[0] for fr in self.frames]
        rel = int(self.rel_status.item()) if self.queries is not None else 0
        return codes, rel

    # ---------------------------------------------------------------- graph
    def capture(self):
        torch = _torch()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def view_slice(self, i):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        cam = self.views[i][1]
        return {"ids": self.ids[a:b], "weights": self.weights[a:b], "counts": self.counts[a:b],
                "out": self.out[a:b], "width": cam.width, "height": cam.height}


def time_batch(batch: Batch, steps: int = 5, warmup: int = 2) -> float:
    """Milliseconds per graph replay of the whole batch step."""
    torch = _torch()
    if batch.graph is None:
        batch.capture()
    for _ in range(warmup):
        batch.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        batch.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


# (tile shape, pixel group, channel chunks per row, blend warps per CTA):
# 0 = the built-in choice
DEFAULT_CANDIDATES = (((16, 16), 0, 0, 0), ((16, 16), 0, 0, 4), ((16, 16), 0, 1, 0),
                      ((16, 16), 0, 2, 0), ((16, 16), 0, 4, 0), ((16, 16), 0, 2, 4),
                      ((8, 32), 0, 0, 0), ((16, 16), 2, 0, 0), ((8, 32), 2, 0, 0))


def _quads_per_lane(C: int) -> int:
    return C // 128


def autotune(scenes, views, K=8, queries=None, candidates=DEFAULT_CANDIDATES, steps=3):
    """Try each (tile shape, pixel group, channel chunks, blend warps) on the batch, return
    (best Batch, timings); combinations the row width or K rule out are skipped."""
    timings = {}
    best, best_ms = None, float("inf")
    C = int(scenes[0].feat.shape[1])
    qt = _quads_per_lane(C)
    for tile, group, chunks, bw in candidates:
        if group and group * K > 32:
            continue
        if chunks and (qt % chunks or qt // chunks > 4 or (group or (4 if K <= 8 else 2)) != 4):
            continue
        b = Batch(scenes, views, K=K, tile=tile, group=group, chunks=chunks, blend_warps=bw,
                  queries=queries)
        ms = time_batch(b, steps=steps)
        timings[f"{tile[0]}x{tile[1]}/g{group or 'auto'}/c{chunks or 'auto'}/w{bw or 8}"] = round(ms, 4)
        if ms < best_ms:
            if best is not None:
                best.graph = None
            best, best_ms = b, ms
        else:
            b.graph = None
    return best, timings
