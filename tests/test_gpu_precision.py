"""BF16 and FP8-E4M3 feature tables (FP32 accumulation) against the FP64 oracle.

* The GPU encoders are bit-exact with the oracle's independent encoders.
* Rendering from a BF16 / FP8 table matches the oracle rendering the same
  table (decoded by the oracle) within the FP32 tolerance.
* On the precision workload (1M Gaussians, 1296x968, K = 8) the error of the
  rendered map against the FP64 oracle on the original FP32 features is
  reported per dtype and gated: FP32 <= 1e-5, BF16 <= 5e-3 (element rounding
  2^-9 relative), FP8 <= 7e-2 (element rounding 2^-4 relative).
"""
import numpy as np
import pytest

import oracle
from oracle import compare
from paper_2512_20927_gb300 import scenes

import gpu_harness as H

pytestmark = pytest.mark.gpu

FEAT_TOL = 1e-5
GATES = {"f32": 1e-5, "bf16": 5e-3, "fp8": 7e-2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_20927_gb300 import qrender
    qrender.load()


def _finite_sample(rng, n):
    bits = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x)]
    extra = np.array([0.0, -0.0, 1.0, -1.0, 448.0, 464.0, 2.0 ** -9, 2.0 ** -10, 1e-30,
                      3.3895314e38, -3.3895314e38], np.float32)
    return np.concatenate([x, extra, rng.normal(0, 3, n).astype(np.float32)])


def test_bf16_encoder_bit_exact():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    x = _finite_sample(np.random.default_rng(1), 1 << 20)
    got = q.qr_quantize_bf16(torch.from_numpy(x).cuda()).view(torch.int16).cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint16), oracle.bf16_encode(x))


def test_fp8_encoder_bit_exact():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    rng = np.random.default_rng(2)
    rows = [scenes.unit_features(rng, 500, 512), rng.normal(0, 1, (300, 512)).astype(np.float32),
            (rng.normal(0, 1, (200, 512)) * 10.0 ** rng.uniform(-8, 8, (200, 1))).astype(np.float32),
            np.zeros((3, 512), np.float32)]
    f = np.concatenate(rows)
    f[-1, 7] = -2.5
    codes, scale = q.qr_quantize_fp8(torch.from_numpy(f).cuda())
    rc, rs = oracle.fp8_quantize_rows(f)
    np.testing.assert_array_equal(scale.cpu().numpy(), rs)
    np.testing.assert_array_equal(codes.cpu().numpy(), rc)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_low_precision_tables_match_oracle_on_decoded_features(dtype):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = H.small_room(n=20000, channels=64)
    cam = scenes.room_camera(150, 110)
    fd = torch.from_numpy(f).cuda()
    if dtype == "bf16":
        table = q.qr_quantize_bf16(fd)
        decoded = oracle.bf16_decode(oracle.bf16_encode(f))
    else:
        table = q.qr_quantize_fp8(fd)
        codes, sc = oracle.fp8_quantize_rows(f)
        decoded = oracle.fp8_dequantize_rows(codes, sc)
    gpu = H.run_gpu(g, None, cam, K=8, feat_dev=table)
    pr, pix, ref = H.run_oracle(g, decoded, cam, 8)
    rep = H.check_frame(gpu, ref, pix, cam.width, decoded, FEAT_TOL, 2e-5, label=dtype)
    print(dtype, rep)


def test_precision_config_error_vs_fp64_oracle():
    """1M-Gaussian room at 1296x968, K = 8: error of each storage dtype against
    the FP64 oracle on the FP32 features, on sampled pixels."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = scenes.room_scene(seed=0, n=1_000_000, channels=512)
    cam = scenes.room_camera(1296, 968)
    fd = torch.from_numpy(f).cuda()
    tables = {"f32": fd, "bf16": q.qr_quantize_bf16(fd), "fp8": q.qr_quantize_fp8(fd)}
    pix = H.sample_pixels(1296, 968, 160, seed=4)
    pr, pix, ref = H.run_oracle(g, f, cam, 8, pixels=pix)
    idx = H.pixel_index(pix, cam.width)
    report = {}
    ids_f32 = None
    for name, table in tables.items():
        gpu = H.run_gpu(g, None, cam, K=8, feat_dev=table, dense=True)
        sel = compare.selection_report(gpu["ids"][idx], gpu["weights"][idx], gpu["counts"][idx], ref)
        same = sel["same"]
        assert sel["mismatch_nontie"] == 0
        if ids_f32 is None:
            ids_f32 = gpu["ids"]
        else:   # the selection does not depend on the feature dtype
            np.testing.assert_array_equal(gpu["ids"], ids_f32)
        err = compare.feature_error(gpu["out"][idx], ref.out_q, ref.scale_q)[same]
        dtie = (ref.tie & compare.DENSE_TIE_BITS) == 0
        derr = compare.feature_error(gpu["dense"][idx], ref.out_dense, ref.scale_dense)[dtie]
        report[name] = {"q_max": float(err.max()), "q_mean": float(err.mean()),
                        "dense_max": float(derr.max()), "dense_mean": float(derr.mean())}
        assert err.max() <= GATES[name], (name, report[name])
        assert derr.max() <= max(GATES[name], 2e-5), (name, report[name])
    print("precision-config error vs FP64 oracle:", report)
