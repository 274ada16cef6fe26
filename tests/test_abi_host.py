"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/qrender.h declares, and validates its arguments before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2512_20927_gb300 import qrender as q
from paper_2512_20927_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_20927_gb300 import build_lib
    build_lib.build()
    return q.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(qr_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(q.SIGNATURES) == names


def test_abi_version_and_strings(lib):
    assert lib.qr_abi_version() == 1
    for code in range(7):
        assert q.status_string(code)


def test_default_params(lib):
    p = q.default_params(8)
    assert p.K == 8 and p.tile_w * p.tile_h == 256
    assert abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.alpha_max - 0.99) < 1e-7


def _frame(n=1000, K=8, cap=4096, ws=1 << 20, nbytes=1 << 40, cam=None, **kw):
    p = q.default_params(K, **kw)
    c = q.make_camera(cam or scenes.tiny_camera())
    f = q.qr_frame()
    return q.load().qr_frame_init(ctypes.byref(f), n, ctypes.byref(c), ctypes.byref(p), cap,
                                  ctypes.c_void_p(ws), nbytes), f


def test_frame_init_validates_arguments(lib):
    assert _frame()[0] == q.QR_OK
    assert _frame(K=0)[0] == q.QR_ERR_INVALID_ARG
    assert _frame(K=33)[0] == q.QR_ERR_INVALID_ARG
    assert _frame(n=-1)[0] == q.QR_ERR_INVALID_ARG
    assert _frame(tile_w=12, tile_h=21)[0] == q.QR_ERR_INVALID_ARG
    assert _frame(ws=(1 << 20) + 16)[0] == q.QR_ERR_ALIGNMENT
    assert _frame(nbytes=1000)[0] == q.QR_ERR_INVALID_ARG
    bad = scenes.tiny_camera()
    bad.fx = float("nan")
    assert _frame(cam=bad)[0] == q.QR_ERR_INVALID_ARG
    rc, f = _frame(tile_w=8, tile_h=32)
    assert rc == q.QR_OK and f.tiles_x == 16 and f.tiles_y == 4


def test_workspace_bytes_scale(lib):
    p = q.default_params(8)
    a = q.workspace_bytes(1000, 64, 64, p, 1000)
    b = q.workspace_bytes(2000, 64, 64, p, 1000)
    c = q.workspace_bytes(1000, 64, 64, p, 100000)
    assert 0 < a < b and a < c
    assert q.workspace_bytes(-5, 64, 64, p, 10) == 0


def test_blend_rejects_bad_arguments_before_launch(lib):
    L = q.load()
    P = ctypes.c_void_p
    good = P(1 << 20)
    launches = L.qr_launch_count()
    # null features
    assert L.qr_blend(None, None, q.QR_F32, 16, 10, good, good, good, 4, 8, 0, good, None) == q.QR_ERR_INVALID_ARG
    # misaligned feature pointer
    assert L.qr_blend(P((1 << 20) + 4), None, q.QR_F32, 16, 10, good, good, good, 4, 8, 0, good, None) == q.QR_ERR_ALIGNMENT
    # row not a multiple of 16 bytes
    assert L.qr_blend(good, None, q.QR_F32, 6, 10, good, good, good, 4, 8, 0, good, None) == q.QR_ERR_ALIGNMENT
    # FP8 without scales
    assert L.qr_blend(good, None, q.QR_FP8E4M3, 32, 10, good, good, good, 4, 8, 0, good, None) == q.QR_ERR_INVALID_ARG
    # K out of range
    assert L.qr_blend(good, None, q.QR_F32, 16, 10, good, good, good, 4, 40, 0, good, None) == q.QR_ERR_INVALID_ARG
    # unsupported width
    assert L.qr_blend(good, None, q.QR_F32, 20, 10, good, good, good, 4, 8, 0, good, None) == q.QR_ERR_NOT_SUPPORTED
    # nothing launched by any of these
    assert L.qr_launch_count() == launches


def test_render_host_sizes(lib):
    nin, nout = q.qr_render_host_bytes(100, 32, 16, 8, 16, q.QR_F32)
    assert nin >= 100 * 11 * 4 + 100 * 16 * 4 and nout >= 32 * 16 * (8 * 8 + 1 + 16 * 4)


def test_cosine_backward_rejects_bad_arguments_before_launch(lib):
    """qr_cosine_backward checks its pointers, alignment and workspace size on
    the host, and its workspace is the backward's plus one float per pixel."""
    L = q.load()
    P = ctypes.c_void_p
    rc, f = _frame(n=1000, K=8, cap=4096)
    assert rc == q.QR_OK
    fp = ctypes.byref(f)
    C = 64
    wb = L.qr_backward_workspace_bytes(fp, C)
    wc = L.qr_cosine_backward_workspace_bytes(fp, C)
    pixels = f.camera.width * f.camera.height
    assert wb > 0 and wc >= wb + 4 * pixels and wc - wb < 4 * pixels + 256
    assert L.qr_cosine_backward_workspace_bytes(fp, 6) == 0     # C not a multiple of 4
    good = P(1 << 20)
    launches = L.qr_launch_count()

    def call(**kw):
        a = dict(feat=good, scale=None, dt=q.QR_F32, C=C, ids=good, w=good, cnt=good, F=good,
                 t=good, mask=good, loss=good, gmap=good, gf=good, ga=None, gc=None, ws=good,
                 wsb=wc)
        a.update(kw)
        return L.qr_cosine_backward(fp, a["feat"], a["scale"], a["dt"], a["C"], a["ids"], a["w"],
                                    a["cnt"], a["F"], a["t"], a["mask"], a["loss"], a["gmap"],
                                    a["gf"], a["ga"], a["gc"], a["ws"], a["wsb"], None)
    assert call(F=None) == q.QR_ERR_INVALID_ARG
    assert call(mask=None) == q.QR_ERR_INVALID_ARG
    assert call(loss=None) == q.QR_ERR_INVALID_ARG
    assert call(gmap=None) == q.QR_ERR_INVALID_ARG
    assert call(t=P((1 << 20) + 4)) == q.QR_ERR_ALIGNMENT
    assert call(gmap=P((1 << 20) + 8)) == q.QR_ERR_ALIGNMENT
    assert call(ws=P((1 << 20) + 16)) == q.QR_ERR_ALIGNMENT
    assert call(wsb=wc - 1) == q.QR_ERR_INVALID_ARG
    assert call(dt=q.QR_FP8E4M3) == q.QR_ERR_INVALID_ARG             # FP8 without scales
    assert L.qr_launch_count() == launches


def test_header_enumerators_match_the_binding():
    """Every `QR_NAME = value` enumerator of the header has the same value in
    the Python binding (status codes, dtypes, select rules)."""
    src = open(os.path.join(ROOT, "include", "qrender.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    enums = {m.group(1): int(m.group(2), 0)
             for m in re.finditer(r"\b(QR_[A-Z0-9_]+)\s*=\s*(-?(?:0x[0-9a-fA-F]+|\d+))", src)}
    assert {"QR_RULE_QUANTILE", "QR_RULE_TOPK", "QR_RULE_STRATIFIED", "QR_RULE_RIEMANN",
            "QR_OK", "QR_F32", "QR_BF16", "QR_FP8E4M3"} <= set(enums)
    for name, value in enums.items():
        assert hasattr(q, name), name
        assert getattr(q, name) == value, (name, getattr(q, name), value)


def test_select_rule_rejects_unknown_rules_before_launch(lib):
    rc, f = _frame()
    assert rc == q.QR_OK
    good = ctypes.c_void_p(1 << 20)
    for rule in (-1, 4, 99):
        assert lib.qr_select_rule(ctypes.byref(f), rule, good, good, good, None, None) == \
            q.QR_ERR_INVALID_ARG
    assert lib.qr_select_rule(None, q.QR_RULE_RIEMANN, good, good, good, None, None) == \
        q.QR_ERR_INVALID_ARG
