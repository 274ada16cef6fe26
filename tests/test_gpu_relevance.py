"""Relevance GEMM (tcgen05, FP32 accumulation in TMEM) against FP64.

The queries are BF16, exact in both operand formats the kernels use.  The map
enters the tensor cores either as TF32 (the TMA kernel: at least 10 mantissa
bits, relative error below 2^-10 per element) or rounded to BF16 (round to
nearest even, like the oracle's encoder; the register-staged kernel used
where the TMA kernel's shared memory does not fit).  Every result is within
the BF16 bound 2^-8 * sum |a b| of the exact product of the FP32 map; a
result outside the TF32 bound 2^-10 * sum |a b| must equal the FP64 product
of the BF16-rounded map up to FP32 accumulation (1e-4 * sum |a b|).
"""
import numpy as np
import pytest

import oracle

import gpu_harness as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# The TMA kernel holds the queries in FP32 shared memory: C * Q * 4 bytes plus
# four 16 KB map stages must fit, so 128 queries of 512 channels take the
# register-staged BF16 kernel.
@pytest.mark.parametrize("P,C,Q,kernel", [(1000, 512, 64, "tma"), (128, 64, 16, "tma"),
                                          (4099, 512, 128, "bf16"), (777, 256, 32, "tma"),
                                          (130, 1024, 32, "tma")])
def test_relevance_matches_fp64(P, C, Q, kernel):
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
    H.check_relevance(scores.cpu().numpy(), fmap, qbits, kernel)


def test_relevance_rejects_unsupported_shapes():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    m = torch.zeros((10, 96), device="cuda")
    qq = torch.zeros((64, 96), dtype=torch.int16, device="cuda")
    with pytest.raises(q.QRError) as e:
        q.qr_relevance(m, qq)
    assert e.value.code == q.QR_ERR_NOT_SUPPORTED
