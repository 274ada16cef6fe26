"""Relevance GEMM (tcgen05, BF16 x BF16 -> FP32 in TMEM) against FP64.

The map is rounded to BF16 by the kernel (round to nearest even, like the
oracle's encoder) and the queries are BF16, so the exact reference is the FP64
product of the BF16-rounded operands; the only GPU error is the FP32
accumulation order (<= C * 2^-24 * sum |a b|, gated at 1e-4 of sum |a b|).
Against the unrounded FP32 map the error is bounded by the BF16 rounding,
2^-8 * sum |a b|.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("P,C,Q", [(1000, 512, 64), (128, 64, 16), (4099, 512, 128), (777, 256, 32)])
def test_relevance_matches_fp64(P, C, Q):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300 import scenes
    rng = np.random.default_rng(P + C + Q)
    fmap = rng.normal(size=(P, C)).astype(np.float32)
    fmap[::7] /= np.linalg.norm(fmap[::7], axis=1, keepdims=True)
    queries = scenes.unit_queries(seed=Q, q=Q, channels=C)
    qbits = oracle.bf16_encode(queries)
    qdev = torch.from_numpy(qbits.view(np.int16)).cuda()
    scores, status = q.qr_relevance(torch.from_numpy(fmap).cuda(), qdev)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = scores.cpu().numpy().astype(np.float64)
    a = oracle.bf16_decode(oracle.bf16_encode(fmap))
    b = oracle.bf16_decode(qbits)
    ref = oracle.relevance(a, b)
    mag = np.abs(a) @ np.abs(b).T
    assert (np.abs(got - ref) <= 1e-4 * mag + 1e-30).all(), np.abs(got - ref).max()
    ref32 = oracle.relevance(fmap, b)
    assert (np.abs(got - ref32) <= 2.0 ** -8 * mag + 1e-6).all()


def test_relevance_rejects_unsupported_shapes():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    m = torch.zeros((10, 96), device="cuda")
    qq = torch.zeros((64, 96), dtype=torch.int16, device="cuda")
    with pytest.raises(q.QRError) as e:
        q.qr_relevance(m, qq)
    assert e.value.code == q.QR_ERR_NOT_SUPPORTED
