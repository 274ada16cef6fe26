"""Device-side error paths, exercised without faulting or hanging the GPU.

* A bounded wait that runs out: qr_set_wait_limit makes the relevance
  kernels' waits give up after one poll (the data a wait expects cannot have
  arrived by then); the kernel must report QR_ERR_DEVICE_TIMEOUT in its status
  word, drain its own copies and MMAs, and leave the context usable -- the
  next call with the default bound is correct.
* Non-finite inputs: Gaussians with NaN / Inf means, NaN / Inf opacities,
  NaN / Inf log-scales or a zero quaternion are culled before any tile index
  is derived from them (read in project.cu: the opacity and depth tests, the
  determinant test and the isfinite guard on the projected mean); the frame
  must equal the oracle's, which drops the same Gaussians.
"""
import numpy as np
import pytest

import oracle
from oracle import compare
from paper_2512_20927_gb300 import scenes

import gpu_harness as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("fused", [False, True])
def test_wait_that_runs_out_reports_timeout_and_recovers(fused):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    rng = np.random.default_rng(3)
    P, C, Q = 64 * 1024, 512, 64
    qbits = q.qr_quantize_bf16(torch.from_numpy(scenes.unit_queries(7, Q, C)).cuda()).view(torch.int16)
    if fused:
        n, K = 4000, 8
        f = torch.from_numpy(rng.normal(size=(n, C)).astype(np.float32)).cuda()
        ids, w, cnt = (torch.from_numpy(a).cuda() for a in scenes.random_selection(seed=1, pixels=P, k=K, n=n))
        run = lambda: q.qr_blend_relevance(f, None, ids, w, cnt, qbits)  # noqa: E731
    else:
        fmap = torch.from_numpy(rng.normal(size=(P, C)).astype(np.float32)).cuda()
        run = lambda: q.qr_relevance(fmap, qbits)  # noqa: E731
    good, st = run()
    torch.cuda.synchronize()
    assert st.item() == 0
    try:
        q.qr_set_wait_limit(1)
        _, st = run()
        torch.cuda.synchronize()
        assert st.item() == q.QR_ERR_DEVICE_TIMEOUT
    finally:
        q.qr_set_wait_limit(0)
    again, st = run()
    torch.cuda.synchronize()
    assert st.item() == 0
    assert torch.equal(again, good)


def test_non_finite_gaussians_are_culled():
    g, f = scenes.tiny_scene(seed=6)
    rng = np.random.default_rng(6)
    bad = rng.choice(g.n, 60, replace=False)
    kinds = np.arange(60) % 6
    for i, k in zip(bad, kinds):
        if k == 0:
            g.mean[i, 0] = np.nan
        elif k == 1:
            g.mean[i, 2] = np.inf
        elif k == 2:
            g.opacity[i] = np.nan
        elif k == 3:
            g.opacity[i] = np.inf
        elif k == 4:
            g.log_scale[i, 1] = np.nan if i % 2 else np.inf
        else:
            g.quat[i] = 0.0
    cam = scenes.tiny_camera()
    gpu = H.run_gpu(g, f, cam, K=8)
    pr, pix, ref = H.run_oracle(g, f, cam, 8)
    rep = H.check_frame(gpu, ref, pix, cam.width, f, 1e-5, 2e-5, label="non-finite")
    assert not np.isin(gpu["ids"], bad).any()
    assert np.isfinite(gpu["out"]).all() and np.isfinite(gpu["dense"]).all()
    print("non-finite inputs", rep)
