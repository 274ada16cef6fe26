"""The blend fused with the relevance product (qr_blend_relevance) against its
definition in FP64: R = (sum_j w_pj f_{id_pj}) Q^T, through the C ABI.

The map is blended in FP32, rounded to BF16 and multiplied on the tensor
cores with FP32 accumulation, so |R - R_64| <= 2^-8 sum_c |F|_c |q|_c, with
|F|_c = sum_j |w_j| |f_j,c| (which also covers the FP32 blend rounding): the
test uses 2^-8 of that magnitude product plus 1e-6.
"""
import numpy as np
import pytest

import oracle
from oracle import compare
from paper_2512_20927_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check(got, ids, w, cnt, fdec, qbits):
    qd = oracle.bf16_decode(qbits)
    F = compare.blend(ids, w, cnt, fdec)
    Fmag = compare.blend(ids, np.abs(w), cnt, np.abs(fdec))
    exact = oracle.relevance(F, qd)
    mag = Fmag @ np.abs(qd).T
    err = np.abs(np.asarray(got, np.float64) - exact)
    worst = float((err / (mag + 1e-30)).max())
    assert (err <= 2.0 ** -8 * mag + 1e-6).all(), worst
    return worst


def _table(kind, f, q, torch):
    fdev = torch.from_numpy(f).cuda()
    if kind == "f32":
        return fdev, None, f.astype(np.float64)
    if kind == "bf16":
        return q.qr_quantize_bf16(fdev), None, oracle.bf16_decode(oracle.bf16_encode(f))
    codes, scale = q.qr_quantize_fp8(fdev)
    c, s = oracle.fp8_quantize_rows(f)
    return codes, scale, oracle.fp8_dequantize_rows(c, s)


@pytest.mark.parametrize("kind,C,Q,K", [("f32", 512, 64, 8), ("f32", 128, 16, 4), ("f32", 256, 32, 8),
                                        ("bf16", 512, 64, 8), ("fp8", 512, 64, 8),
                                        ("f32", 384, 128, 1), ("bf16", 1024, 64, 3)])
def test_fused_matches_definition_consecutive_pixels(kind, C, Q, K):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    rng = np.random.default_rng(C + Q + K)
    n, P = 3000, 5000 + 77                              # ragged last block of 128
    f = rng.normal(size=(n, C)).astype(np.float32)
    ids, w, cnt = scenes.random_selection(seed=C + K, pixels=P, k=K, n=n)
    table, scale, fdec = _table(kind, f, q, torch)
    qbits = q.qr_quantize_bf16(torch.from_numpy(scenes.unit_queries(7, Q, C)).cuda())
    dev = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    got, st = q.qr_blend_relevance(table, scale, dev(ids), dev(w), dev(cnt), qbits.view(torch.int16))
    torch.cuda.synchronize()
    assert st.item() == 0
    worst = _check(got.cpu().numpy(), ids, w, cnt, fdec, qbits.view(torch.int16).cpu().numpy().view(np.uint16))
    print(f"fused {kind} C={C} Q={Q} K={K}: worst error {worst:.2e} of the magnitude bound")


def test_fused_on_a_rendered_frame_matches_the_two_step_path():
    """Room scene 150x110 (ragged 16x8 blocks), 512-D FP32: the fused scores
    equal qr_blend followed by qr_relevance within the TF32 bound, and the
    definition on every pixel."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = scenes.room_scene(seed=0, n=20000, channels=512)
    cam = scenes.room_camera(150, 110)
    fdev = torch.from_numpy(f).cuda()
    res = q.render_frame(q.gaussians_to_device(g), fdev, cam, K=8)
    qbits = q.qr_quantize_bf16(torch.from_numpy(scenes.unit_queries(7, 64, 512)).cuda()).view(torch.int16)
    fused, st = q.qr_blend_relevance(fdev, None, res["ids"], res["weights"], res["counts"], qbits,
                                     width=cam.width)
    two, st2 = q.qr_relevance(res["out"], qbits)
    torch.cuda.synchronize()
    assert st.item() == 0 and st2.item() == 0
    ids, w, cnt = (res[k].cpu().numpy() for k in ("ids", "weights", "counts"))
    qn = qbits.cpu().numpy().view(np.uint16)
    _check(fused.cpu().numpy(), ids, w, cnt, f.astype(np.float64), qn)
    _check(two.cpu().numpy(), ids, w, cnt, f.astype(np.float64), qn)
    assert (fused[torch.from_numpy(cnt == 0).cuda()] == 0).all()


def test_fused_rejects_what_it_does_not_serve():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    f = torch.zeros((100, 96), device="cuda")
    ids = torch.zeros((10, 8), dtype=torch.int32, device="cuda")
    w = torch.zeros((10, 8), device="cuda")
    cnt = torch.zeros(10, dtype=torch.uint8, device="cuda")
    qb = torch.zeros((64, 96), dtype=torch.int16, device="cuda")
    with pytest.raises(q.QRError) as e:
        q.qr_blend_relevance(f, None, ids, w, cnt, qb)          # C = 96: not a multiple of 128
    assert e.value.code == q.QR_ERR_NOT_SUPPORTED
    ids16 = torch.zeros((10, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(q.QRError) as e:
        q.qr_blend_relevance(torch.zeros((100, 128), device="cuda"), None, ids16,
                             torch.zeros((10, 16), device="cuda"), cnt,
                             torch.zeros((64, 128), dtype=torch.int16, device="cuda"))
    assert e.value.code == q.QR_ERR_NOT_SUPPORTED             # K = 16 > 8
