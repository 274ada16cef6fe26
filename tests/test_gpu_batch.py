"""Many views in one persistent launch (qr_render_batch) against the
single-view path, plus the many-view workload against the FP64 oracle."""
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


def _small_batch(tile, channels=128, dtype="f32"):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300.batch import Batch, Scene
    sc = []
    for seed, n in ((0, 20000), (1, 12000)):
        g, f = scenes.room_scene(seed=seed, n=n, channels=channels)
        fd = torch.from_numpy(f).cuda()
        table = fd if dtype == "f32" else q.qr_quantize_bf16(fd)
        sc.append((g, f, Scene(q.gaussians_to_device(g), table)))
    views = [(0, scenes.room_camera(150, 110)), (1, scenes.room_camera(96, 64, yaw=1.0)),
             (0, scenes.room_camera(200, 150, eye=(0.5, 0.5, 1.2), yaw=-0.7, pitch=0.1)),
             (1, scenes.room_camera(33, 17, yaw=2.5))]
    b = Batch([s[2] for s in sc], views, K=8, tile=tile)
    return sc, views, b


@pytest.mark.parametrize("tile", [(16, 16), (8, 32)])
def test_batch_matches_single_views(tile):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    sc, views, b = _small_batch(tile)
    b.step()
    torch.cuda.synchronize()
    codes, _ = b.status()
    assert all(c == q.QR_OK for c in codes)
    for i, (si, cam) in enumerate(views):
        ref = q.render_frame(sc[si][2].gdev, sc[si][2].table, cam, K=8,
                             params=q.default_params(8, tile_w=tile[0], tile_h=tile[1]))
        got = b.view_slice(i)
        torch.testing.assert_close(got["ids"], ref["ids"], rtol=0, atol=0)
        torch.testing.assert_close(got["counts"], ref["counts"], rtol=0, atol=0)
        torch.testing.assert_close(got["weights"], ref["weights"], rtol=0, atol=0)
        if tile == (16, 16):      # same 2x2 pixel groups as the tile-ordered qr_blend
            tab = sc[si][2].table
            f, fs = tab if isinstance(tab, tuple) else (tab, None)
            tiled = torch.empty_like(ref["out"])
            q.qr_blend(f, fs, ref["ids"], ref["weights"], ref["counts"], tiled, width=cam.width)
            torch.testing.assert_close(got["out"], tiled, rtol=0, atol=0)
            torch.testing.assert_close(got["out"], ref["out"], rtol=1e-6, atol=1e-6)
        else:                     # 2x2 groups of 8x32 tiles: another summation order
            torch.testing.assert_close(got["out"], ref["out"], rtol=1e-6, atol=1e-6)


def test_batch_graph_replay_and_relevance():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300.batch import Batch
    sc, views, b0 = _small_batch((16, 16), channels=256, dtype="bf16")
    queries = scenes.unit_queries(seed=7, q=64, channels=256)
    qbits = torch.from_numpy(oracle.bf16_encode(queries).view(np.int16)).cuda()
    b = Batch(b0.scenes, views, K=8, queries=qbits)
    b.step()
    torch.cuda.synchronize()
    eager = b.out.clone(), b.scores.clone()
    b.out.zero_()
    b.scores.zero_()
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    torch.testing.assert_close(b.out, eager[0], rtol=0, atol=0)
    torch.testing.assert_close(b.scores, eager[1], rtol=0, atol=0)
    assert int(b.rel_status.item()) == 0
    H.check_relevance(b.scores.cpu().numpy(), b.out.cpu().numpy(), oracle.bf16_encode(queries))


def test_many_view_workload_against_oracle():
    """4 rooms (200k, 500k, 1M, 2M Gaussians), 32 views from 320x240 to
    1296x968, 512-D BF16 features, K = 8, autotuned; two views checked against
    the FP64 oracle on sampled pixels."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300.batch import Scene, autotune
    sizes = (200_000, 500_000, 1_000_000, 2_000_000)
    raw, sc = [], []
    for seed, n in enumerate(sizes):
        g, f = scenes.room_scene(seed=seed, n=n, channels=512)
        raw.append((g, f))
        sc.append(Scene(q.gaussians_to_device(g), q.qr_quantize_bf16(torch.from_numpy(f).cuda())))
    views = scenes.batched_views(seed=0, n_views=32, scenes=4)
    queries = scenes.unit_queries(seed=7, q=64, channels=512)
    qbits = torch.from_numpy(oracle.bf16_encode(queries).view(np.int16)).cuda()
    best, timings = autotune(sc, views, K=8, queries=qbits, steps=2)
    best.replay()
    torch.cuda.synchronize()
    codes, rel = best.status()
    assert all(c == q.QR_OK for c in codes) and rel == 0
    print("many-view autotune (ms per batch):", timings, "chosen", best.tile, best.group, best.chunks)
    for i in (3, 31):          # a view of the 200k room and one of the 2M room
        si, cam = views[i]
        g, f = raw[si]
        decoded = oracle.bf16_decode(oracle.bf16_encode(f))
        pix = H.sample_pixels(cam.width, cam.height, 60, seed=i)
        pr, pix, ref = H.run_oracle(g, decoded, cam, 8, pixels=pix)
        v = best.view_slice(i)
        gpu = {k: v[k].cpu().numpy() for k in ("ids", "weights", "counts", "out")}
        H.check_frame(gpu, ref, pix, cam.width, decoded, 1e-5, label=f"view {i}")
        idx = H.pixel_index(pix, cam.width)
        a = int(best.offsets[i])
        got = best.scores[a:a + cam.width * cam.height].cpu().numpy()[idx]
        ref_rel = oracle.relevance(ref.out_q, oracle.bf16_decode(qbits.cpu().numpy().view(np.uint16)))
        mag = np.abs(ref.out_q) @ np.abs(oracle.bf16_decode(qbits.cpu().numpy().view(np.uint16))).T
        assert (np.abs(got - ref_rel) <= 2.0 ** -7 * mag + 1e-5).all()


@pytest.mark.parametrize("dtype,channels", [("f32", 512), ("bf16", 512), ("bf16", 256)])
def test_batch_chunks_and_blend_warps_bit_identical(dtype, channels):
    """The autotuner's channel-chunk and blend-warp axes change who computes
    which channels, not the sums: every setting gives the same bits (ids,
    weights, counts and map) as the default, and the default's map equals the
    tile-ordered qr_blend of its own selection."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300.batch import Batch
    sc, views, b0 = _small_batch((16, 16), channels=channels, dtype=dtype)
    b0.step()
    torch.cuda.synchronize()
    ref = [b0.view_slice(i) for i in range(len(views))]
    qt = channels // 128   # quads (4 channels) per lane over a row
    settings = [(c, w) for c in (1, 2, 4) for w in (0, 4) if qt % c == 0 and qt // c <= 4] + [(0, 4)]
    for chunks, bw in settings:
        b = Batch(b0.scenes, views, K=8, chunks=chunks, blend_warps=bw)
        b.step()
        torch.cuda.synchronize()
        codes, _ = b.status()
        assert all(c == q.QR_OK for c in codes)
        for i in range(len(views)):
            got = b.view_slice(i)
            for k in ("ids", "weights", "counts", "out"):
                assert torch.equal(got[k], ref[i][k]), (chunks, bw, i, k)
    for i, (si, cam) in enumerate(views):
        tab = sc[si][2].table
        tiled = torch.empty_like(ref[i]["out"])
        q.qr_blend(tab, None, ref[i]["ids"], ref[i]["weights"], ref[i]["counts"], tiled,
                   width=cam.width)
        assert torch.equal(tiled, ref[i]["out"]), i
