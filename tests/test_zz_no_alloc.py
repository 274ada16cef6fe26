"""qr_render_noalloc against qr_render, through the C ABI.

qr_render_noalloc serves callers that may not allocate device memory (a
plug-in whose host owns all device memory, a real-time loop, set-up ahead of
graph capture): its scratch is a static device array inside the library.
This test runs it twice in a row on different scenes and checks each result
against the same forward with a caller-allocated workspace on the same inputs,
so a second call cannot pass on leftovers of the first.  Both run the same
kernels in the same pixel order, so the results must agree bit for bit.  The
second call must also leave the device's free memory unchanged (the first one
may load the library's device code, which holds the static array).  It lives
in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2512_20927_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _reference(q, gdev, fdev, cam, K):
    res = q.render_frame(gdev, fdev, cam, K=K, dense=False)
    return {k: res[k].cpu().numpy() for k in ("ids", "weights", "counts", "out")}


def test_noalloc_matches_workspace_render_twice():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    cases = [(scenes.tiny_scene(seed=0, n=2000, channels=16), scenes.tiny_camera(128, 128), 8),
             (scenes.tiny_scene(seed=5, n=700, channels=16), scenes.tiny_camera(100, 72), 4)]
    for call, ((g, f), cam, K) in enumerate(cases):
        gdev = q.gaussians_to_device(g)
        fdev = torch.from_numpy(f).cuda()
        ref = _reference(q, gdev, fdev, cam, K)
        P = cam.width * cam.height
        ids = torch.full((P, K), 123, dtype=torch.int32, device="cuda")
        w = torch.full((P, K), 7.0, device="cuda")
        cnt = torch.full((P,), 99, dtype=torch.uint8, device="cuda")
        out = torch.full((P, f.shape[1]), 5.0, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        fr = q.qr_render_noalloc(*gdev, cam, q.default_params(K), fdev, None, ids, w, cnt, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call > 0:
            assert free1 == free0, (free0, free1)
        code, nis = q.qr_frame_status(fr)
        assert code == q.QR_OK and nis > 0
        np.testing.assert_array_equal(ids.cpu().numpy(), ref["ids"])
        np.testing.assert_array_equal(cnt.cpu().numpy(), ref["counts"])
        np.testing.assert_array_equal(w.cpu().numpy(), ref["weights"])
        np.testing.assert_array_equal(out.cpu().numpy(), ref["out"])


def test_noalloc_rejects_frames_beyond_its_limits():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = scenes.tiny_scene(n=100, channels=16)
    gdev = q.gaussians_to_device(g)
    fdev = torch.from_numpy(f).cuda()
    cam = scenes.tiny_camera(512, 512)      # 262,144 pixels > 65,536
    P = cam.width * cam.height
    with pytest.raises(q.QRError) as e:
        q.qr_render_noalloc(*gdev, cam, q.default_params(8), fdev, None,
                            torch.empty((P, 8), dtype=torch.int32, device="cuda"),
                            torch.empty((P, 8), device="cuda"),
                            torch.empty(P, dtype=torch.uint8, device="cuda"),
                            torch.empty((P, 16), device="cuda"))
    assert e.value.code == q.QR_ERR_INVALID_ARG
