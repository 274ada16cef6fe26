"""Thin ctypes binding of libqrender (include/qrender.h).

Argument marshalling only: every step of the render runs in the library's
CUDA kernels.  PyTorch provides device memory (the workspace and the output
tensors) and the current CUDA stream.  The functions keep the C names.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2512_20927_gb300.build_lib``); loading fails loudly
otherwise -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqrender.so")

QR_OK, QR_ERR_INVALID_ARG, QR_ERR_ALIGNMENT, QR_ERR_CAPACITY, QR_ERR_CUDA, \
    QR_ERR_DEVICE_TIMEOUT, QR_ERR_NOT_SUPPORTED = range(7)
QR_F32, QR_BF16, QR_FP8E4M3 = 0, 1, 2
QR_RULE_QUANTILE, QR_RULE_TOPK, QR_RULE_STRATIFIED, QR_RULE_RIEMANN = 0, 1, 2, 3
FRAME_SLOTS = 24


class QRError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


class qr_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("near_plane", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class qr_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("T_min", ctypes.c_float),
                ("dilation", ctypes.c_float), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32)]


class qr_frame(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("max_isect", ctypes.c_int64), ("camera", qr_camera),
                ("params", qr_params), ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32),
                ("sort_blocks", ctypes.c_int32), ("isect_buf", ctypes.c_int32),
                ("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t),
                ("off", ctypes.c_size_t * FRAME_SLOTS)]


class qr_view(ctypes.Structure):
    _fields_ = [("frame", ctypes.c_void_p), ("feat", ctypes.c_void_p),
                ("feat_scale", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("counts", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


class qr_frame_view(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in (
        "mean2d_hi_lo", "axes", "opacity", "depth_key", "tile_count", "kept_gid", "kept_offset",
        "isect_gid", "tile_range", "counters")]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_S = ctypes.c_int

# name -> (restype, argtypes); every function declared in include/qrender.h
SIGNATURES = {
    "qr_abi_version": (_I32, []),
    "qr_status_string": (ctypes.c_char_p, [_S]),
    "qr_default_params": (None, [ctypes.POINTER(qr_params)]),
    "qr_workspace_bytes": (ctypes.c_size_t, [_I64, _I32, _I32, ctypes.POINTER(qr_params), _I64]),
    "qr_frame_init": (_S, [ctypes.POINTER(qr_frame), _I64, ctypes.POINTER(qr_camera),
                           ctypes.POINTER(qr_params), _I64, _P, ctypes.c_size_t]),
    "qr_frame_view_get": (_S, [ctypes.POINTER(qr_frame), ctypes.POINTER(qr_frame_view)]),
    "qr_frame_status": (_S, [ctypes.POINTER(qr_frame), _P, ctypes.POINTER(_I64)]),
    "qr_project": (_S, [ctypes.POINTER(qr_frame), _P, _P, _P, _P, _P]),
    "qr_sort": (_S, [ctypes.POINTER(qr_frame), _P]),
    "qr_select": (_S, [ctypes.POINTER(qr_frame), _P, _P, _P, _P]),
    "qr_select_rule": (_S, [ctypes.POINTER(qr_frame), _S, _P, _P, _P, _P, _P]),
    "qr_blend": (_S, [_P, _P, _S, _I32, _I64, _P, _P, _P, _I64, _I32, _I32, _P, _P]),
    "qr_dense": (_S, [ctypes.POINTER(qr_frame), _P, _P, _S, _I32, _P, _P, _P]),
    "qr_dense_work": (_S, [ctypes.POINTER(qr_frame), _P, _P, _S, _I32, _P, _P, _P, _P]),
    "qr_render": (_S, [ctypes.POINTER(qr_frame), _P, _P, _P, _P, _P, _P, _S, _I32, _P, _P, _P,
                       _P, _P]),
    "qr_render_host_bytes": (_S, [_I64, _I32, _I32, _I32, _I32, _S,
                                  ctypes.POINTER(ctypes.c_size_t),
                                  ctypes.POINTER(ctypes.c_size_t)]),
    "qr_render_host": (_S, [ctypes.POINTER(qr_frame), _P, _P, _P, _P, _P, _P, _S, _I32, _P, _P,
                            _P, _P]),
    "qr_launch_count": (ctypes.c_uint64, []),
    "qr_set_wait_limit": (None, [ctypes.c_uint32]),
    "qr_set_blend_chunks": (_S, [_I32]),
    "qr_backward_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(qr_frame), _I32]),
    "qr_backward": (_S, [ctypes.POINTER(qr_frame), _P, _P, _S, _I32, _P, _P, _P, _P, _P, _P, _P,
                         _P, ctypes.c_size_t, _P]),
    "qr_cosine_loss": (_S, [_P, _P, _P, _I64, _I32, _P, _P, _P, _P]),
    "qr_cosine_backward_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(qr_frame), _I32]),
    "qr_cosine_backward": (_S, [ctypes.POINTER(qr_frame), _P, _P, _S, _I32, _P, _P, _P, _P, _P,
                                _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "qr_relevance": (_S, [_P, _P, _I32, _I32, _I64, _P, _P, _P]),
    "qr_blend_relevance": (_S, [_P, _P, _S, _I32, _I64, _P, _P, _P, _I64, _I32, _I32, _P, _I32,
                                _P, _P, _P]),
    "qr_contrastive_workspace_bytes": (ctypes.c_size_t, [_I64, _I32, _I32]),
    "qr_contrastive_loss": (_S, [_P, _P, _I32, _I32, _P, _I64, _P, _P, _P, ctypes.c_size_t, _P]),
    "qr_contrastive_backward_workspace_bytes": (ctypes.c_size_t,
                                                [ctypes.POINTER(qr_frame), _I32, _I32]),
    "qr_contrastive_backward": (_S, [ctypes.POINTER(qr_frame), _P, _P, _S, _I32, _P, _P, _P, _P,
                                     _P, _I32, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "qr_batch_workspace_bytes": (ctypes.c_size_t, [_I32]),
    "qr_batch_prepare": (_S, [ctypes.POINTER(qr_view), _I32, _P, ctypes.c_size_t,
                              ctypes.POINTER(ctypes.c_uint32), _P]),
    "qr_render_batch": (_S, [_P, _I32, ctypes.c_uint32, _S, _I32, _I32, _I32, _I32, _I32, _I32,
                             _P]),
    "qr_quantize_bf16": (_S, [_P, _I64, _P, _P]),
    "qr_quantize_fp8": (_S, [_P, _I64, _I32, _P, _P, _P]),
    "qr_render_noalloc": (_S, [_P, _P, _P, _P, _I64, ctypes.POINTER(qr_camera),
                               ctypes.POINTER(qr_params), _P, _P, _S, _I32, _P, _P, _P, _P,
                               ctypes.POINTER(qr_frame), _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libqrender.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_string(code: int) -> str:
    try:
        return load().qr_status_string(code).decode()
    except Exception:  # noqa: BLE001 - used while formatting another error
        return "status"


def _check(code: int, where: str):
    if code != QR_OK:
        raise QRError(code, where)


# ---------------------------------------------------------------- torch glue
def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return QR_F32
    if t.dtype == torch.bfloat16:
        return QR_BF16
    if t.dtype in (torch.uint8, getattr(torch, "float8_e4m3fn", torch.uint8)):
        return QR_FP8E4M3
    raise TypeError(f"unsupported feature dtype {t.dtype}")


def default_params(K: int = 8, **kw) -> qr_params:
    p = qr_params()
    load().qr_default_params(ctypes.byref(p))
    p.K = K
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_camera(cam) -> qr_camera:
    """qr_camera from a scenes.Camera (or anything with R, t, fx, fy, cx, cy, width, height, near)."""
    c = qr_camera()
    R = np.asarray(cam.R, np.float32).reshape(-1)
    t = np.asarray(cam.t, np.float32).reshape(-1)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane = float(cam.near)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


@dataclass
class Frame:
    """A qr_frame plus the torch tensor that backs its workspace."""
    frame: qr_frame
    workspace: object
    camera: qr_camera
    params: qr_params

    @property
    def width(self) -> int:
        return int(self.camera.width)

    @property
    def height(self) -> int:
        return int(self.camera.height)

    @property
    def pixels(self) -> int:
        return self.width * self.height

    @property
    def K(self) -> int:
        return int(self.params.K)


def workspace_bytes(n: int, width: int, height: int, params: qr_params, max_isect: int) -> int:
    return int(load().qr_workspace_bytes(n, width, height, ctypes.byref(params), max_isect))


def frame_create(n: int, cam, params: qr_params, max_isect: int, device="cuda") -> Frame:
    """Allocate a workspace with torch and lay out a frame in it (qr_frame_init)."""
    torch = _torch()
    camc = cam if isinstance(cam, qr_camera) else make_camera(cam)
    nbytes = workspace_bytes(n, camc.width, camc.height, params, max_isect)
    if nbytes == 0:
        raise QRError(QR_ERR_INVALID_ARG, "qr_workspace_bytes")
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    f = qr_frame()
    _check(load().qr_frame_init(ctypes.byref(f), n, ctypes.byref(camc), ctypes.byref(params),
                                max_isect, ctypes.c_void_p(aligned), nbytes), "qr_frame_init")
    return Frame(f, ws, camc, params)


def qr_frame_status(fr: Frame, stream=None):
    """Synchronise and read the device status; returns (status code, n_isect)."""
    n = _I64(0)
    code = load().qr_frame_status(ctypes.byref(fr.frame), _stream(stream), ctypes.byref(n))
    return code, int(n.value)


def qr_frame_view_get(fr: Frame) -> qr_frame_view:
    v = qr_frame_view()
    _check(load().qr_frame_view_get(ctypes.byref(fr.frame), ctypes.byref(v)), "qr_frame_view_get")
    return v


def qr_project(fr: Frame, mean, log_scale, quat, opacity, stream=None):
    _check(load().qr_project(ctypes.byref(fr.frame), _ptr(mean), _ptr(log_scale), _ptr(quat),
                             _ptr(opacity), _stream(stream)), "qr_project")


def qr_sort(fr: Frame, stream=None):
    _check(load().qr_sort(ctypes.byref(fr.frame), _stream(stream)), "qr_sort")


def qr_select(fr: Frame, ids, weights, counts, stream=None):
    _check(load().qr_select(ctypes.byref(fr.frame), _ptr(ids), _ptr(weights), _ptr(counts),
                            _stream(stream)), "qr_select")


def qr_select_rule(fr: Frame, rule, ids, weights, counts, tau=None, stream=None):
    """Top-K / Stratified-K / Riemann-weight / Algorithm 1 selection into
    qr_select's outputs."""
    _check(load().qr_select_rule(ctypes.byref(fr.frame), int(rule), _ptr(ids), _ptr(weights),
                                 _ptr(counts), _ptr(tau), _stream(stream)), "qr_select_rule")


def qr_blend(feat, feat_scale, ids, weights, counts, out, width=0, stream=None):
    P, K = ids.shape
    C = feat.shape[1]
    _check(load().qr_blend(_ptr(feat), _ptr(feat_scale), _dtype_code(feat), C, feat.shape[0],
                           _ptr(ids), _ptr(weights), _ptr(counts), P, K, width, _ptr(out),
                           _stream(stream)), "qr_blend")


def qr_dense(fr: Frame, feat, feat_scale, out, T_final=None, stream=None):
    _check(load().qr_dense(ctypes.byref(fr.frame), _ptr(feat), _ptr(feat_scale),
                           _dtype_code(feat), feat.shape[1], _ptr(out), _ptr(T_final),
                           _stream(stream)), "qr_dense")


def qr_dense_work(fr: Frame, feat, feat_scale, out, T_final=None, stream=None):
    """qr_dense counting its work: returns a device int64 tensor [blended
    (pixel, Gaussian) pairs, executed multiply-adds]."""
    torch = _torch()
    counts = torch.zeros(2, dtype=torch.int64, device=out.device)
    _check(load().qr_dense_work(ctypes.byref(fr.frame), _ptr(feat), _ptr(feat_scale),
                                _dtype_code(feat), feat.shape[1], _ptr(out), _ptr(T_final),
                                _ptr(counts), _stream(stream)), "qr_dense_work")
    return counts


def qr_render(fr: Frame, mean, log_scale, quat, opacity, feat, feat_scale, ids, weights, counts,
              out, stream=None):
    _check(load().qr_render(ctypes.byref(fr.frame), _ptr(mean), _ptr(log_scale), _ptr(quat),
                            _ptr(opacity), _ptr(feat), _ptr(feat_scale), _dtype_code(feat),
                            feat.shape[1], _ptr(ids), _ptr(weights), _ptr(counts), _ptr(out),
                            _stream(stream)), "qr_render")


def qr_render_host_bytes(n, width, height, K, C, dtype_code):
    a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(load().qr_render_host_bytes(n, width, height, K, C, dtype_code, ctypes.byref(a),
                                       ctypes.byref(b)), "qr_render_host_bytes")
    return int(a.value), int(b.value)


def qr_render_host(fr: Frame, mean_h, log_scale_h, quat_h, opacity_h, feat_h, feat_scale_h,
                   dtype_code, C, dev_inputs, dev_outputs, out_h, stream=None):
    """Host-buffer render: arguments are pinned torch CPU tensors (or numpy arrays)."""
    def hp(x):
        if x is None:
            return None
        if hasattr(x, "data_ptr"):
            return ctypes.c_void_p(x.data_ptr())
        return ctypes.c_void_p(x.ctypes.data)
    _check(load().qr_render_host(ctypes.byref(fr.frame), hp(mean_h), hp(log_scale_h),
                                 hp(quat_h), hp(opacity_h), hp(feat_h), hp(feat_scale_h),
                                 dtype_code, C, _ptr(dev_inputs), _ptr(dev_outputs), hp(out_h),
                                 _stream(stream)), "qr_render_host")


def qr_render_noalloc(mean, log_scale, quat, opacity, cam, params, feat, feat_scale, ids,
                      weights, counts, out, stream=None) -> Frame:
    """qr_render without any device allocation (scratch in the library's static array).

    Returns a Frame describing the static workspace (valid until the next
    call) for qr_frame_status."""
    camc = cam if isinstance(cam, qr_camera) else make_camera(cam)
    f = qr_frame()
    _check(load().qr_render_noalloc(_ptr(mean), _ptr(log_scale), _ptr(quat), _ptr(opacity),
                                    mean.shape[0], ctypes.byref(camc), ctypes.byref(params),
                                    _ptr(feat), _ptr(feat_scale), _dtype_code(feat),
                                    feat.shape[1], _ptr(ids), _ptr(weights), _ptr(counts),
                                    _ptr(out), ctypes.byref(f), _stream(stream)),
           "qr_render_noalloc")
    return Frame(f, None, camc, params)


def qr_backward(fr: Frame, feat, feat_scale, ids, weights, counts, grad_out, want_conic=True,
                stream=None):
    """Gradients of the Q-Render forward of `fr` w.r.t. features, opacity and conic.

    Returns (grad_feat [n, C] float32, grad_opacity [n], grad_conic [n, 3] or None)."""
    torch = _torch()
    n = int(fr.frame.n)
    C = feat.shape[1]
    dev = grad_out.device
    nbytes = int(load().qr_backward_workspace_bytes(ctypes.byref(fr.frame), C))
    if nbytes == 0:
        raise QRError(QR_ERR_INVALID_ARG, "qr_backward_workspace_bytes")
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    wsp = ctypes.c_void_p((ws.data_ptr() + 255) // 256 * 256)
    gf = torch.empty((n, C), dtype=torch.float32, device=dev)
    ga = torch.empty(n, dtype=torch.float32, device=dev)
    gc = torch.empty((n, 3), dtype=torch.float32, device=dev) if want_conic else None
    _check(load().qr_backward(ctypes.byref(fr.frame), _ptr(feat), _ptr(feat_scale),
                              _dtype_code(feat), C, _ptr(ids), _ptr(weights), _ptr(counts),
                              _ptr(grad_out.contiguous()), _ptr(gf), _ptr(ga), _ptr(gc), wsp,
                              nbytes, _stream(stream)), "qr_backward")
    return gf, ga, gc


def qr_cosine_backward(fr: Frame, feat, feat_scale, ids, weights, counts, feature_map, target,
                       mask=None, want_conic=True, stream=None):
    """Cosine loss of `feature_map` against `target` over `mask` (default: the
    counts) and the backward of the forward of `fr` under that loss, with the
    loss's per-pixel pass fused into the backward's.

    Returns (loss scalar tensor, dL/dF [P, C], grad_feat [n, C], grad_opacity [n],
    grad_conic [n, 3] or None)."""
    torch = _torch()
    n = int(fr.frame.n)
    C = feat.shape[1]
    dev = feature_map.device
    P = feature_map.shape[0]
    nbytes = int(load().qr_cosine_backward_workspace_bytes(ctypes.byref(fr.frame), C))
    if nbytes == 0:
        raise QRError(QR_ERR_INVALID_ARG, "qr_cosine_backward_workspace_bytes")
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    wsp = ctypes.c_void_p((ws.data_ptr() + 255) // 256 * 256)
    out2 = torch.empty(2, dtype=torch.float32, device=dev)
    gmap = torch.empty((P, C), dtype=torch.float32, device=dev)
    gf = torch.empty((n, C), dtype=torch.float32, device=dev)
    ga = torch.empty(n, dtype=torch.float32, device=dev)
    gc = torch.empty((n, 3), dtype=torch.float32, device=dev) if want_conic else None
    mask = counts if mask is None else mask
    _check(load().qr_cosine_backward(ctypes.byref(fr.frame), _ptr(feat), _ptr(feat_scale),
                                     _dtype_code(feat), C, _ptr(ids), _ptr(weights), _ptr(counts),
                                     _ptr(feature_map.contiguous()), _ptr(target.contiguous()),
                                     _ptr(mask), _ptr(out2), _ptr(gmap), _ptr(gf), _ptr(ga),
                                     _ptr(gc), wsp, nbytes, _stream(stream)), "qr_cosine_backward")
    return out2[0], gmap, gf, ga, gc


def qr_cosine_loss(feature_map, target, counts, stream=None):
    """(loss scalar tensor, dL/dF) of the mean (1 - cos) loss over covered pixels."""
    torch = _torch()
    P, C = feature_map.shape
    dev = feature_map.device
    out2 = torch.empty(2, dtype=torch.float32, device=dev)
    grad = torch.empty((P, C), dtype=torch.float32, device=dev)
    scratch = torch.empty(P, dtype=torch.float32, device=dev)
    _check(load().qr_cosine_loss(_ptr(feature_map.contiguous()), _ptr(target.contiguous()),
                                 _ptr(counts), P, C, _ptr(out2), _ptr(grad), _ptr(scratch),
                                 _stream(stream)), "qr_cosine_loss")
    return out2[0], grad


def _aligned_ws(nbytes, dev):
    torch = _torch()
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    return ws, ctypes.c_void_p((ws.data_ptr() + 255) // 256 * 256)


def qr_contrastive_loss(feature_map, targets, mask_id, stream=None):
    """Eq. 2 loss of a [P, C] map against [M, C] mask embeddings, mask_id [P]
    int32 (-1: not in the loss).  Returns (loss scalar tensor, dL/dF [P, C])."""
    torch = _torch()
    P, C = feature_map.shape
    M = targets.shape[0]
    dev = feature_map.device
    nbytes = int(load().qr_contrastive_workspace_bytes(P, M, C))
    if nbytes == 0:
        raise QRError(QR_ERR_NOT_SUPPORTED, "qr_contrastive_workspace_bytes")
    ws, wsp = _aligned_ws(nbytes, dev)
    out2 = torch.empty(2, dtype=torch.float32, device=dev)
    grad = torch.empty((P, C), dtype=torch.float32, device=dev)
    _check(load().qr_contrastive_loss(_ptr(feature_map.contiguous()), _ptr(targets.contiguous()),
                                      M, C, _ptr(mask_id), P, _ptr(out2), _ptr(grad), wsp, nbytes,
                                      _stream(stream)), "qr_contrastive_loss")
    return out2[0], grad


def qr_contrastive_backward(fr: Frame, feat, feat_scale, ids, weights, counts, feature_map,
                            targets, mask_id, want_conic=True, stream=None):
    """Eq. 2 loss of the rendered map and the backward of the forward of `fr`
    under it.  Returns (loss scalar tensor, dL/dF [P, C], grad_feat [n, C],
    grad_opacity [n], grad_conic [n, 3] or None)."""
    torch = _torch()
    n = int(fr.frame.n)
    C = feat.shape[1]
    M = targets.shape[0]
    dev = feature_map.device
    P = feature_map.shape[0]
    nbytes = int(load().qr_contrastive_backward_workspace_bytes(ctypes.byref(fr.frame), M, C))
    if nbytes == 0:
        raise QRError(QR_ERR_NOT_SUPPORTED, "qr_contrastive_backward_workspace_bytes")
    ws, wsp = _aligned_ws(nbytes, dev)
    out2 = torch.empty(2, dtype=torch.float32, device=dev)
    gmap = torch.empty((P, C), dtype=torch.float32, device=dev)
    gf = torch.empty((n, C), dtype=torch.float32, device=dev)
    ga = torch.empty(n, dtype=torch.float32, device=dev)
    gc = torch.empty((n, 3), dtype=torch.float32, device=dev) if want_conic else None
    _check(load().qr_contrastive_backward(ctypes.byref(fr.frame), _ptr(feat), _ptr(feat_scale),
                                          _dtype_code(feat), C, _ptr(ids), _ptr(weights),
                                          _ptr(counts), _ptr(feature_map.contiguous()),
                                          _ptr(targets.contiguous()), M, _ptr(mask_id),
                                          _ptr(out2), _ptr(gmap), _ptr(gf), _ptr(ga), _ptr(gc),
                                          wsp, nbytes, _stream(stream)), "qr_contrastive_backward")
    return out2[0], gmap, gf, ga, gc


def qr_relevance(feature_map, queries_bf16, stream=None):
    """Relevance scores [P, Q] float32 of a [P, C] float32 map against [Q, C] BF16 queries.

    Returns (scores, status) where status is a 1-element device int32 tensor
    (nonzero if a device-side wait timed out)."""
    torch = _torch()
    P, C = feature_map.shape
    Q = queries_bf16.shape[0]
    out = torch.empty((P, Q), dtype=torch.float32, device=feature_map.device)
    status = torch.zeros(1, dtype=torch.int32, device=feature_map.device)
    _check(load().qr_relevance(_ptr(feature_map), _ptr(queries_bf16), Q, C, P, _ptr(out),
                               _ptr(status), _stream(stream)), "qr_relevance")
    return out, status


def qr_blend_relevance(feat, feat_scale, ids, weights, counts, queries_bf16, width=0,
                       stream=None):
    """Relevance scores [P, Q] of the blend of (ids, weights, counts) against
    [Q, C] BF16 queries without writing the map.  Returns (scores, status)."""
    torch = _torch()
    P, K = ids.shape
    C = feat.shape[1]
    Q = queries_bf16.shape[0]
    out = torch.empty((P, Q), dtype=torch.float32, device=ids.device)
    status = torch.zeros(1, dtype=torch.int32, device=ids.device)
    _check(load().qr_blend_relevance(_ptr(feat), _ptr(feat_scale), _dtype_code(feat), C,
                                     feat.shape[0], _ptr(ids), _ptr(weights), _ptr(counts), P, K,
                                     width, _ptr(queries_bf16), Q, _ptr(out), _ptr(status),
                                     _stream(stream)), "qr_blend_relevance")
    return out, status


def qr_quantize_bf16(x, stream=None):
    """BF16 copy of a float32 device tensor (returned as torch.bfloat16)."""
    torch = _torch()
    out = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    _check(load().qr_quantize_bf16(_ptr(x), x.numel(), _ptr(out), _stream(stream)),
           "qr_quantize_bf16")
    return out


def qr_quantize_fp8(x, stream=None):
    """(codes uint8 [rows, C], scale float32 [rows]) of a float32 [rows, C] device tensor."""
    torch = _torch()
    rows, C = x.shape
    codes = torch.empty((rows, C), dtype=torch.uint8, device=x.device)
    scale = torch.empty(rows, dtype=torch.float32, device=x.device)
    _check(load().qr_quantize_fp8(_ptr(x), rows, C, _ptr(codes), _ptr(scale), _stream(stream)),
           "qr_quantize_fp8")
    return codes, scale


def qr_launch_count() -> int:
    return int(load().qr_launch_count())


def qr_set_wait_limit(polls: int):
    """Test hook: bound the relevance kernels' waits to `polls` polls (0 = default)."""
    load().qr_set_wait_limit(int(polls))


def qr_set_blend_chunks(chunks: int):
    """Tuning: channel chunks per feature row in the wide-row blend (0 = built-in)."""
    _check(load().qr_set_blend_chunks(int(chunks)), "qr_set_blend_chunks")


# ---------------------------------------------------------------- convenience
def gaussians_to_device(g, device="cuda"):
    """Upload a scenes.Gaussians to the GPU as contiguous float32 tensors."""
    torch = _torch()
    return tuple(torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
                 for a in (g.mean, g.log_scale, g.quat, g.opacity))


def render_frame(gdev, feat, cam, K=8, max_isect=None, params=None, stream=None, dense=False,
                 rule=QR_RULE_QUANTILE):
    """Project, sort, select (Algorithm 1, or another qr_rule) and blend one
    frame; grows the intersection capacity and retries when the device reports
    an overflow.  Returns a dict of device tensors (ids, weights, counts,
    out[, dense, T_final][, tau]) and the frame."""
    torch = _torch()
    mean = gdev[0]
    n = mean.shape[0]
    params = params or default_params(K)
    cap = max_isect or max(1 << 16, 8 * n)
    camc = make_camera(cam)
    while True:
        fr = frame_create(n, camc, params, cap, device=mean.device)
        P = fr.pixels
        ids = torch.empty((P, params.K), dtype=torch.int32, device=mean.device)
        w = torch.empty((P, params.K), dtype=torch.float32, device=mean.device)
        cnt = torch.empty(P, dtype=torch.uint8, device=mean.device)
        qr_project(fr, *gdev, stream=stream)
        qr_sort(fr, stream=stream)
        code, nis = qr_frame_status(fr, stream)
        if code == QR_ERR_CAPACITY:
            cap = int(nis * 1.25) + 1024
            continue
        _check(code, "qr_sort")
        break
    res = {"ids": ids, "weights": w, "counts": cnt, "n_isect": nis, "frame": fr}
    if rule == QR_RULE_QUANTILE:
        qr_select(fr, ids, w, cnt, stream=stream)
    else:
        tau = (torch.empty((P, params.K), dtype=torch.float32, device=mean.device)
               if rule == QR_RULE_STRATIFIED else None)
        qr_select_rule(fr, rule, ids, w, cnt, tau, stream=stream)
        if tau is not None:
            res["tau"] = tau
    if feat is not None:
        f, fs = feat if isinstance(feat, tuple) else (feat, None)
        C = f.shape[1]
        out = torch.empty((P, C), dtype=torch.float32, device=mean.device)
        qr_blend(f, fs, ids, w, cnt, out, stream=stream)
        res["out"] = out
        if dense:
            dout = torch.empty((P, C), dtype=torch.float32, device=mean.device)
            tf = torch.empty(P, dtype=torch.float32, device=mean.device)
            qr_dense(fr, f, fs, dout, tf, stream=stream)
            res["dense"] = dout
            res["T_final"] = tf
    return res
