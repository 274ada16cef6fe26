"""FP64 CPU oracle for the Q-Render hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and this package never imports the product.

The arithmetic lives in ``qr_oracle.c`` (plain C, double precision, brute force
per pixel, no tiles).  This module only builds that file with gcc, marshals
numpy arrays through ctypes and adds a few definitions that are clearer as
numpy (cosine loss, relevance matmul, feature decoding).

Parity pins for every function live in ``tests/test_oracle_*.py``.  Functions
without an independent pin say "parity unpinned" in their docstring (none at
present).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
# The same parameters rounded to FP32, as the CUDA library receives them; the
# parity tests evaluate the oracle with these exact values.
ALPHA_MIN_F32 = float(np.float32(1.0 / 255.0))
ALPHA_MAX_F32 = float(np.float32(0.99))
DEFAULT_DILATION = 0.3
# FP32 relative-error constant for alpha' used by the near-tie classifier
# (see the comment above classify_ties in qr_oracle.c).
DEFAULT_TIE_EPS = 2.0 ** -22


def build(force: bool = False) -> str:
    """Compile qr_oracle.c into _build/liboracle.so with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


def _declare(L):
    L.or_project.argtypes = [_I64, _P, _P, _P, _P, _D, _P, _P, _P, _P, _P]
    L.or_project.restype = _I
    L.or_render.argtypes = ([_I64, _P, _P, _P, _P, _P, _P, _I, _I, _D, _D, _D, _D, _I64, _P, _I]
                            + [_P] * 11 + [_I, _P, _P, _P])
    L.or_render.restype = _I
    L.or_backward.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _I, _I, _D, _D, _I64, _P, _P,
                              _P, _P, _P, _P, _P, _P]
    L.or_classify_candidates.argtypes = [_I64, _P, _P, _P, _P, _I, _D, _D, _D, _D, _P, _P]
    L.or_classify_candidates.restype = _I
    L.or_topk_list.argtypes = [_I64, _P, _I, _D, _P, _P, _P]
    L.or_topk_list.restype = _I
    L.or_stratified_list.argtypes = [_I64, _P, _I, _D, _P, _P, _P, _P, _P, _P]
    L.or_stratified_list.restype = _I
    L.or_riemann_list.argtypes = [_I64, _P, _I, _P, _P, _P]
    L.or_riemann_list.restype = _I
    L.or_render_rule.argtypes = ([_I64, _P, _P, _P, _P, _P, _P, _I, _I, _I, _D, _D, _D, _D, _I64,
                                  _P, _I] + [_P] * 9)
    L.or_render_rule.restype = _I
    L.or_classify_rule_candidates.argtypes = [_I64, _P, _P, _P, _P, _I, _I, _D, _D, _D, _D, _P,
                                              _P]
    L.or_classify_rule_candidates.restype = _I
    L.or_backward.restype = _I
    L.or_qrender_list.argtypes = [_I64, _P, _I, _P, _P, _P, _P]
    L.or_qrender_list.restype = _I
    L.or_qselect_closed_form.argtypes = [_I64, _P, _I, _P]
    L.or_qselect_closed_form.restype = _I
    L.or_dense_list.argtypes = [_I64, _P, _D, _P, _P]
    L.or_dense_list.restype = _I64
    L.or_quat_to_rotation.argtypes = [_P, _P]
    L.or_covariance3d.argtypes = [_P, _P, _P]
    L.or_bf16_encode.argtypes = [_P, _I64, _P]
    L.or_bf16_decode.argtypes = [_P, _I64, _P]
    L.or_fp8_encode.argtypes = [_P, _I64, _P]
    L.or_fp8_decode.argtypes = [_P, _I64, _P]
    L.or_fp8_quantize_rows.argtypes = [_P, _I64, _I, _P, _P]


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Sec. 3: covariance, projection
# --------------------------------------------------------------------------
def quat_to_rotation(q) -> np.ndarray:
    q = _c(q, np.float32)
    R = np.zeros(9)
    lib().or_quat_to_rotation(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def covariance3d(log_scale, quat) -> np.ndarray:
    ls, q = _c(log_scale, np.float32), _c(quat, np.float32)
    S = np.zeros(9)
    lib().or_covariance3d(_ptr(ls), _ptr(q), _ptr(S))
    return S.reshape(3, 3)


@dataclass
class Projected:
    mean2d: np.ndarray   # [N,2]
    conic: np.ndarray    # [N,3] (A00, A01, A11)
    cov2d: np.ndarray    # [N,3] (S00, S01, S11)
    depth: np.ndarray    # [N]
    alpha: np.ndarray    # [N] opacity (float64 copy of the input)
    valid: np.ndarray    # [N] int32


def project(gauss, cam_array, dilation: float = DEFAULT_DILATION) -> Projected:
    """EWA projection of every Gaussian (Sec. 3), FP64."""
    n = gauss.n
    mean, ls, q = (_c(gauss.mean, np.float32), _c(gauss.log_scale, np.float32),
                   _c(gauss.quat, np.float32))
    cam = _c(cam_array, np.float32)
    out = Projected(np.zeros((n, 2)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n),
                    np.asarray(gauss.opacity, np.float64).copy(), np.zeros(n, np.int32))
    rc = lib().or_project(n, _ptr(mean), _ptr(ls), _ptr(q), _ptr(cam), dilation,
                          _ptr(out.mean2d), _ptr(out.conic), _ptr(out.cov2d),
                          _ptr(out.depth), _ptr(out.valid))
    assert rc == 0, rc
    return out


# --------------------------------------------------------------------------
# Algorithm 1 and Eq. 1 on a single list
# --------------------------------------------------------------------------
def qrender_list(a, K: int):
    """Algorithm 1 on one front-to-back list of alpha' values.

    Returns (selected mask, unnormalised weights, T^Q, number of visited entries).
    """
    a = _c(a, np.float64)
    n = a.shape[0]
    sel = np.zeros(n, np.int32)
    w = np.zeros(n)
    tq = np.zeros(1)
    npro = np.zeros(1, np.int64)
    lib().or_qrender_list(n, _ptr(a), K, _ptr(sel), _ptr(w), _ptr(tq), _ptr(npro))
    return sel.astype(bool), w, float(tq[0]), int(npro[0])


def qselect_closed_form(a, K: int) -> np.ndarray:
    a = _c(a, np.float64)
    sel = np.zeros(a.shape[0], np.int32)
    lib().or_qselect_closed_form(a.shape[0], _ptr(a), K, _ptr(sel))
    return sel.astype(bool)


def dense_list(a, T_min: float = 0.0):
    """Eq. 1 weights on one list; returns (weights, T_final, number blended)."""
    a = _c(a, np.float64)
    w = np.zeros(a.shape[0])
    tf = np.zeros(1)
    used = lib().or_dense_list(a.shape[0], _ptr(a), T_min, _ptr(w), _ptr(tf))
    return w, float(tf[0]), int(used)


RULE_TOPK = 1
RULE_STRATIFIED = 2
RULE_RIEMANN = 3


def topk_list(a, K: int, T_min: float = 0.0):
    """Top-K on one list (Sec. 4.2's comparison renderer): the K largest Eq. 1
    weights of the dense walk.  Returns (kept mask, their Eq. 1 weights,
    entries blended by the walk)."""
    a = _c(a, np.float64)
    n = a.shape[0]
    sel = np.zeros(n, np.int32)
    w = np.zeros(n)
    nused = np.zeros(1, np.int64)
    m = lib().or_topk_list(n, _ptr(a), K, T_min, _ptr(sel), _ptr(w), _ptr(nused))
    assert m >= 0
    return sel.astype(bool), w, int(nused[0])


def stratified_list(a, K: int, T_min: float = 0.0):
    """Stratified-K on one list (App. E).  Returns (kept mask, unnormalised
    weights, T^Q, entries visited by pass 2, boundaries tau [K], (mu, sigma, n))."""
    a = _c(a, np.float64)
    n = a.shape[0]
    sel = np.zeros(n, np.int32)
    w = np.zeros(n)
    tq = np.zeros(1)
    npro = np.zeros(1, np.int64)
    tau = np.zeros(K)
    st = np.zeros(3)
    m = lib().or_stratified_list(n, _ptr(a), K, T_min, _ptr(sel), _ptr(w), _ptr(tq), _ptr(npro),
                                 _ptr(tau), _ptr(st))
    assert m >= 0
    return sel.astype(bool), w, float(tq[0]), int(npro[0]), tau, (st[0], st[1], int(st[2]))


def riemann_list(a, K: int):
    """Algorithm 1's selection with App. C's right-Riemann weights on one list:
    each quantile Gaussian weighs the number of segment boundaries its test
    transmittance crosses.  Returns (kept mask, crossing counts, entries
    visited)."""
    a = _c(a, np.float64)
    n = a.shape[0]
    sel = np.zeros(n, np.int32)
    w = np.zeros(n)
    npro = np.zeros(1, np.int64)
    m = lib().or_riemann_list(n, _ptr(a), K, _ptr(sel), _ptr(w), _ptr(npro))
    assert m >= 0
    return sel.astype(bool), w, int(npro[0])


def classify_rule_candidates(depth, ids, g, qabs, rule: int, K: int, T_min: float = 0.0,
                             alpha_min: float = ALPHA_MIN, alpha_max: float = ALPHA_MAX,
                             tie_eps: float = DEFAULT_TIE_EPS):
    """Near-tie flags of one pixel under top-K / Stratified-K, from its
    candidates (see classify_candidates).  Returns (flags, kept ids in depth
    order, boundaries tau [K] (stratified))."""
    d = _c(depth, np.float64)
    i = _c(ids, np.int64)
    gg = _c(g, np.float64)
    qa = _c(qabs, np.float64)
    kept = np.zeros(K, np.int64)
    tau = np.zeros(K)
    flags = lib().or_classify_rule_candidates(d.shape[0], _ptr(d), _ptr(i), _ptr(gg), _ptr(qa),
                                              rule, K, alpha_min, alpha_max, T_min, tie_eps,
                                              _ptr(kept), _ptr(tau))
    assert flags >= 0, flags
    return int(flags), kept[kept >= 0], tau


@dataclass
class RuleRendered:
    out: np.ndarray | None
    ids: np.ndarray
    wq: np.ndarray
    cnt: np.ndarray
    n_members: np.ndarray
    n_proc: np.ndarray
    tie: np.ndarray
    scale: np.ndarray | None
    tau: np.ndarray | None


def render_rule(proj: Projected, feat, rule: int, K: int, pixels, T_min: float = 1e-4,
                alpha_min: float = ALPHA_MIN, alpha_max: float = ALPHA_MAX,
                tie_eps: float = DEFAULT_TIE_EPS, threads: int | None = None) -> RuleRendered:
    """Brute-force render of the listed pixels with the top-K (RULE_TOPK),
    Stratified-K (RULE_STRATIFIED) or App. C Riemann-weight (RULE_RIEMANN)
    select rule in place of Algorithm 1's weights, FP64."""
    n = proj.mean2d.shape[0]
    pix = _c(pixels, np.int32)
    m = pix.shape[0]
    f = None if feat is None else _c(feat, np.float64)
    C = 0 if f is None else f.shape[1]
    threads = threads or max(1, os.cpu_count() or 1)
    out = np.zeros((m, C)) if f is not None else None
    sc = np.zeros(m) if f is not None else None
    ids = np.zeros((m, K), np.int32)
    wq = np.zeros((m, K))
    cnt = np.zeros(m, np.int32)
    nmem = np.zeros(m, np.int32)
    npro = np.zeros(m, np.int32)
    tie = np.zeros(m, np.int32)
    tau = np.zeros((m, K)) if rule == RULE_STRATIFIED else None
    rc = lib().or_render_rule(n, _ptr(proj.mean2d), _ptr(proj.conic), _ptr(proj.depth),
                              _ptr(proj.alpha), _ptr(proj.valid), _ptr(f), C, rule, K, alpha_min,
                              alpha_max, T_min, tie_eps, m, _ptr(pix), threads, _ptr(out),
                              _ptr(ids), _ptr(wq), _ptr(cnt), _ptr(nmem), _ptr(npro), _ptr(tie),
                              _ptr(sc), _ptr(tau))
    assert rc == 0, rc
    return RuleRendered(out, ids, wq, cnt, nmem, npro, tie, sc, tau)


# --------------------------------------------------------------------------
# Per-pixel renderer
# --------------------------------------------------------------------------
@dataclass
class Rendered:
    out_q: np.ndarray | None
    ids: np.ndarray
    wq: np.ndarray
    cnt: np.ndarray
    tq: np.ndarray
    out_dense: np.ndarray | None
    t_final: np.ndarray
    n_members: np.ndarray
    n_proc: np.ndarray
    tie: np.ndarray
    members: np.ndarray | None = None
    scale_q: np.ndarray | None = None
    scale_dense: np.ndarray | None = None
    n_dense: np.ndarray | None = None


def all_pixels(width: int, height: int) -> np.ndarray:
    ys, xs = np.mgrid[0:height, 0:width]
    return np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int32)


def render(proj: Projected, feat, K: int, pixels, T_min: float = 1e-4,
           alpha_min: float = ALPHA_MIN, alpha_max: float = ALPHA_MAX,
           tie_eps: float = DEFAULT_TIE_EPS, threads: int | None = None,
           want_q: bool = True, want_dense: bool = True, max_members: int = 0) -> Rendered:
    """Brute-force render of the listed pixels ([M,2] int (x, y)) in FP64.

    ``feat`` is the [N,C] feature table in any float dtype (converted to
    float64 exactly) or None to compute only selections.
    """
    n = proj.mean2d.shape[0]
    pix = _c(pixels, np.int32)
    m = pix.shape[0]
    f = None if feat is None else _c(feat, np.float64)
    C = 0 if f is None else f.shape[1]
    threads = threads or max(1, os.cpu_count() or 1)
    out_q = np.zeros((m, C)) if (want_q and f is not None) else None
    out_d = np.zeros((m, C)) if (want_dense and f is not None) else None
    ids = np.zeros((m, K), np.int32)
    wq = np.zeros((m, K))
    cnt = np.zeros(m, np.int32)
    tq = np.zeros(m)
    tf = np.zeros(m)
    nmem = np.zeros(m, np.int32)
    npro = np.zeros(m, np.int32)
    tie = np.zeros(m, np.int32)
    mem = np.zeros((m, max_members), np.int32) if max_members > 0 else None
    sq = np.zeros(m) if out_q is not None else None
    sd = np.zeros(m) if out_d is not None else None
    nd = np.zeros(m, np.int32)
    rc = lib().or_render(n, _ptr(proj.mean2d), _ptr(proj.conic), _ptr(proj.depth),
                         _ptr(proj.alpha), _ptr(proj.valid), _ptr(f), C, K, alpha_min,
                         alpha_max, T_min, tie_eps, m, _ptr(pix), threads,
                         _ptr(out_q), _ptr(ids), _ptr(wq), _ptr(cnt), _ptr(tq), _ptr(out_d),
                         _ptr(tf), _ptr(nmem), _ptr(npro), _ptr(tie), _ptr(mem), max_members,
                         _ptr(sq), _ptr(sd), _ptr(nd))
    assert rc == 0, rc
    return Rendered(out_q, ids, wq, cnt, tq, out_d, tf, nmem, npro, tie, mem, sq, sd, nd)


def backward(proj: Projected, feat, K: int, pixels, grad_out,
             alpha_min: float = ALPHA_MIN, alpha_max: float = ALPHA_MAX,
             with_scales: bool = False):
    """Gradients of Algorithm 1 w.r.t. features, opacity and conic (selection held fixed).

    Returns (grad_feat [n,C], grad_alpha [n], grad_conic [n,3]); with
    ``with_scales`` also (scale_feat [n], scale_alpha [n], scale_conic [n,3]):
    per Gaussian, the sum over pixels of the magnitudes of the terms its
    gradient adds up (|w| max|g| for a feature row), the yardstick of the
    rounding error of that sum."""
    n = proj.mean2d.shape[0]
    f = _c(feat, np.float64)
    C = f.shape[1]
    pix = _c(pixels, np.int32)
    g = _c(grad_out, np.float64)
    gf = np.zeros((n, C))
    ga = np.zeros(n)
    gc = np.zeros((n, 3))
    sf = np.zeros(n) if with_scales else None
    sa = np.zeros(n) if with_scales else None
    sc = np.zeros((n, 3)) if with_scales else None
    rc = lib().or_backward(n, _ptr(proj.mean2d), _ptr(proj.conic), _ptr(proj.depth),
                           _ptr(proj.alpha), _ptr(proj.valid), _ptr(f), C, K, alpha_min,
                           alpha_max, pix.shape[0], _ptr(pix), _ptr(g), _ptr(gf), _ptr(ga),
                           _ptr(gc), _ptr(sf), _ptr(sa), _ptr(sc))
    assert rc == 0, rc
    if with_scales:
        return gf, ga, gc, sf, sa, sc
    return gf, ga, gc


def classify_candidates(depth, ids, g, qabs, K: int, T_min: float = 0.0,
                        alpha_min: float = ALPHA_MIN, alpha_max: float = ALPHA_MAX,
                        tie_eps: float = DEFAULT_TIE_EPS):
    """Near-tie flags of one pixel given its candidates (test hook of the classifier).

    depth, ids, g (= alpha * G, unclamped) and qabs (the conditioning
    magnitude of q) describe the Gaussians evaluated at the pixel, in any
    order.  Returns (flags, entries Algorithm 1 visited, entries the dense
    walk blended); flag bits as in ``compare``: 1 / 2 / 4 for Algorithm 1's
    boundary, alpha_min border and equal-depth checks, 8 / 16 / 64 / 128 for
    the dense walk's T_min, boundary, border and equal-depth checks."""
    d = _c(depth, np.float64)
    i = _c(ids, np.int64)
    gg = _c(g, np.float64)
    qa = _c(qabs, np.float64)
    npro = np.zeros(1, np.int64)
    nused = np.zeros(1, np.int64)
    flags = lib().or_classify_candidates(d.shape[0], _ptr(d), _ptr(i), _ptr(gg), _ptr(qa), K,
                                         alpha_min, alpha_max, T_min, tie_eps, _ptr(npro),
                                         _ptr(nused))
    assert flags >= 0, flags
    return int(flags), int(npro[0]), int(nused[0])


# --------------------------------------------------------------------------
# Feature storage formats
# --------------------------------------------------------------------------
def bf16_encode(x) -> np.ndarray:
    x = _c(x, np.float32)
    out = np.zeros(x.shape, np.uint16)
    lib().or_bf16_encode(_ptr(x), x.size, _ptr(out))
    return out


def bf16_decode(h) -> np.ndarray:
    h = _c(h, np.uint16)
    out = np.zeros(h.shape)
    lib().or_bf16_decode(_ptr(h), h.size, _ptr(out))
    return out


def fp8_encode(x) -> np.ndarray:
    x = _c(x, np.float32)
    out = np.zeros(x.shape, np.uint8)
    lib().or_fp8_encode(_ptr(x), x.size, _ptr(out))
    return out


def fp8_decode(v) -> np.ndarray:
    v = _c(v, np.uint8)
    out = np.zeros(v.shape)
    lib().or_fp8_decode(_ptr(v), v.size, _ptr(out))
    return out


def fp8_quantize_rows(f):
    """Per-Gaussian FP8 E4M3 table: (codes [N,C] uint8, scale [N] float32)."""
    f = _c(f, np.float32)
    n, C = f.shape
    codes = np.zeros((n, C), np.uint8)
    scale = np.zeros(n, np.float32)
    lib().or_fp8_quantize_rows(_ptr(f), n, C, _ptr(codes), _ptr(scale))
    return codes, scale


def fp8_dequantize_rows(codes, scale) -> np.ndarray:
    return fp8_decode(codes) * np.asarray(scale, np.float64)[:, None]


# --------------------------------------------------------------------------
# Loss and relevance (numpy, FP64)
# --------------------------------------------------------------------------
def cosine_loss(F, target, mask, eps: float = 1e-8):
    """L = mean over masked pixels of 1 - cos(F_p, t_p), cos = F.t / (max(|F|,eps) max(|t|,eps)).

    Returns (L, dL/dF).  Pixels outside the mask get zero gradient.
    """
    F = np.asarray(F, np.float64)
    t = np.asarray(target, np.float64)
    mask = np.asarray(mask, bool)
    n = max(int(mask.sum()), 1)
    nf = np.maximum(np.linalg.norm(F, axis=1), eps)
    nt = np.maximum(np.linalg.norm(t, axis=1), eps)
    dot = (F * t).sum(axis=1)
    cos = dot / (nf * nt)
    L = float(((1.0 - cos) * mask).sum() / n)
    # d cos / dF = t/(nf nt) - dot F / (nf^3 nt) when |F| > eps
    big = np.linalg.norm(F, axis=1) > eps
    dcos = t / (nf * nt)[:, None] - np.where(big, dot / (nf ** 3 * nt), 0.0)[:, None] * F
    g = -dcos * (mask / n)[:, None]
    return L, g


def contrastive_loss(F, targets, mask_id, eps: float = 1e-8):
    """Eq. 2 (Sec. 4.3) on a rendered map, FP64.

    Pixel p belongs to mask (patch) i = mask_id[p] with target embedding
    t_i = targets[i]; pixels with mask_id < 0 are not in the loss.  With
    s_j = cos(F_p, t_j) = F.t_j / (max(|F|,eps) max(|t_j|,eps)), the pixel's
    term is  -log( exp(s_i) / sum_{j != i} exp(s_j) )  (the denominator sums
    over the other masks, as Eq. 2 prints it), and L is the mean over the
    pixels in the loss (their count floored at 1).  Returns (L, dL/dF [P,C]):
    dL_p/dF = (1/n) sum_j c_j ds_j/dF with c_i = -1, c_j = softmax_{j != i}(s)_j,
    ds_j/dF = t_j / (nf nt_j) - s_j F / nf^2 (the second term vanishes where
    |F| <= eps, nf = max(|F|, eps) being constant there)."""
    F = np.asarray(F, np.float64)
    T = np.asarray(targets, np.float64)
    mid = np.asarray(mask_id, np.int64)
    on = mid >= 0
    n = max(int(on.sum()), 1)
    nf_raw = np.linalg.norm(F, axis=1)
    nf = np.maximum(nf_raw, eps)
    nt = np.maximum(np.linalg.norm(T, axis=1), eps)
    S = (F @ T.T) / (nf[:, None] * nt[None, :])          # [P, M] cosine similarities
    M = T.shape[0]
    L = 0.0
    g = np.zeros_like(F)
    for p in np.nonzero(on)[0]:
        i = mid[p]
        others = np.arange(M) != i
        e = np.exp(S[p, others])
        L += -S[p, i] + np.log(e.sum())
        c = np.zeros(M)
        c[others] = e / e.sum()
        c[i] = -1.0
        grad = (c / nt) @ T / nf[p]
        if nf_raw[p] > eps:
            grad -= (c @ S[p]) * F[p] / nf[p] ** 2
        g[p] = grad / n
    return L / n, g


def relevance(feature_map, queries) -> np.ndarray:
    """Open-vocabulary relevance (Sec. 5): map [P,C] times queries^T [C,Q] in FP64."""
    return np.asarray(feature_map, np.float64) @ np.asarray(queries, np.float64).T
