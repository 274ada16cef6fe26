"""Backward of Algorithm 1 on the GPU against the FP64 oracle's gradient
(itself pinned by finite differences in tests/test_oracle_pins.py).

Upstream gradients are zero on the pixels the oracle flags as near ties, so
both sides sum over the same selections.  Every Gaussian is checked on its own
against the oracle's yardstick for it: the sum over pixels of the magnitudes
of the parts its gradient adds up (|w| max|g| for a feature row; for the
opacity and conic terms the dL/dalpha' formula with every dot product and sum
taken by magnitude).  An FP32 evaluation errs by a few hundred units in the
last place of that yardstick at most (dot products of up to 512 channels,
sums over a Gaussian's pixels), so the tolerance is 2e-5 of it; Gaussians no
unflagged pixel selected must get exactly zero.
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


def _compare(name, got, ref, rel):
    """GPU against GPU (two routes of the same computation): relative to the
    largest entry."""
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= rel * max(scale, 1e-30), (name, err, scale)
    return err / max(scale, 1e-30)


def _compare_each(name, got, ref, yard, rel):
    """Per Gaussian (per row for features, per element otherwise) against the
    oracle's yardstick; returns the largest error in yardstick units."""
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref)
    if err.ndim == 2 and yard.ndim == 1:
        err = err.max(axis=1)
    zero = yard == 0
    assert (err[zero] == 0).all(), (name, "gradient where nothing was selected")
    ratio = err[~zero] / yard[~zero]
    worst = float(ratio.max()) if ratio.size else 0.0
    assert worst <= rel, (name, worst, int(np.argmax(ratio)))
    return worst


def _check_all(got, ref, rel=2e-5, names=("feat", "alpha", "conic")):
    gf, ga, gc = got
    rf, ra, rc, sf, sa, sc = ref
    out = {}
    for name, x, r, y in (("feat", gf, rf, sf), ("alpha", ga, ra, sa), ("conic", gc, rc, sc)):
        if name in names:
            out[name] = _compare_each(name, x, r, y, rel)
    return out


def _run(g, f, cam, K, table=None, decoded=None, seed=0):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    decoded = f if decoded is None else decoded
    fdev = torch.from_numpy(f).cuda() if table is None else table
    res = q.render_frame(q.gaussians_to_device(g), fdev, cam, K=K)
    pr, pix, ref = H.run_oracle(g, decoded, cam, K)
    tie = (ref.tie & compare.Q_TIE_BITS) != 0
    rng = np.random.default_rng(seed)
    gout = rng.normal(size=(cam.width * cam.height, f.shape[1]))
    gout[tie] = 0.0
    gdev = torch.from_numpy(gout.astype(np.float32)).cuda()
    feat_t, scale_t = (fdev, None) if not isinstance(fdev, tuple) else fdev
    gf, ga, gc = q.qr_backward(res["frame"], feat_t, scale_t, res["ids"], res["weights"],
                               res["counts"], gdev)
    torch.cuda.synchronize()
    ref = oracle.backward(pr, decoded, K, pix, gout.astype(np.float32).astype(np.float64),
                          alpha_min=oracle.ALPHA_MIN_F32, alpha_max=oracle.ALPHA_MAX_F32,
                          with_scales=True)
    return (gf.cpu().numpy(), ga.cpu().numpy(), gc.cpu().numpy()), ref


def test_backward_tiny_matches_oracle():
    g, f = scenes.tiny_scene()
    got, ref = _run(g, f, scenes.tiny_camera(), 8)
    e = _check_all(got, ref)
    untouched = (ref[0] == 0).all(axis=1)
    assert (got[0][untouched] == 0).all()
    print("tiny backward errors in yardstick units", e)


@pytest.mark.parametrize("C", [1040, 2056])
def test_backward_wide_rows(C):
    """Rows wider than one CTA's warps cover at once (C / 128 blocks > 8, the
    last one partial) and widths the blend does not serve: the backward alone,
    on the forward's selection."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, _ = scenes.tiny_scene(n=1500)
    cam = scenes.tiny_camera(64, 48)
    K = 8
    rng = np.random.default_rng(11)
    f = rng.normal(size=(g.n, C)).astype(np.float32)
    res = q.render_frame(q.gaussians_to_device(g), None, cam, K=K)
    pr, pix, ref = H.run_oracle(g, f, cam, K)
    tie = (ref.tie & compare.Q_TIE_BITS) != 0
    gout = rng.normal(size=(cam.width * cam.height, C))
    gout[tie] = 0.0
    gf, ga, gc = q.qr_backward(res["frame"], torch.from_numpy(f).cuda(), None, res["ids"],
                               res["weights"], res["counts"],
                               torch.from_numpy(gout.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    ref = oracle.backward(pr, f, K, pix, gout.astype(np.float32).astype(np.float64),
                          alpha_min=oracle.ALPHA_MIN_F32, alpha_max=oracle.ALPHA_MAX_F32,
                          with_scales=True)
    e = _check_all((gf.cpu().numpy(), ga.cpu().numpy(), gc.cpu().numpy()), ref)
    print(f"wide rows C={C} errors in yardstick units", e)


@pytest.mark.parametrize("K", [4, 16])
def test_backward_room_matches_oracle(K):
    g, f = H.small_room(n=20000, channels=64)
    got, ref = _run(g, f, scenes.room_camera(150, 110), K, seed=K)
    e = _check_all(got, ref)
    print(f"room K={K} backward errors in yardstick units", e)


def test_backward_bf16_table():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = H.small_room(n=20000, channels=64)
    table = q.qr_quantize_bf16(torch.from_numpy(f).cuda())
    decoded = oracle.bf16_decode(oracle.bf16_encode(f))
    got, ref = _run(g, f, scenes.room_camera(150, 110), 8, table=table, decoded=decoded)
    e = _check_all(got, ref, names=("feat", "alpha"))
    print("bf16 table backward errors in yardstick units", e)


def test_autograd_function_matches_c_abi_and_is_linear_in_features():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    from paper_2512_20927_gb300.autograd import quantile_render
    g, f = scenes.tiny_scene(seed=3)
    cam = scenes.tiny_camera(96, 96)
    mean, ls, quat, op = q.gaussians_to_device(g)
    op = op.clone().requires_grad_(True)
    feat = torch.from_numpy(f).cuda().requires_grad_(True)
    out, counts = quantile_render(mean, ls, quat, op, feat, cam, K=8)
    gout = torch.randn_like(out)
    (out * gout).sum().backward()
    fr = q.render_frame((mean, ls, quat, op.detach()), feat.detach(), cam, K=8)
    gf, ga, _ = q.qr_backward(fr["frame"], feat.detach(), None, fr["ids"], fr["weights"],
                              fr["counts"], gout.reshape(-1, f.shape[1]).contiguous())
    torch.testing.assert_close(feat.grad, gf, rtol=0, atol=0)
    torch.testing.assert_close(op.grad, ga, rtol=0, atol=0)
    # the map is linear in the features: a finite difference is exact up to rounding
    idx = torch.nonzero(gf.abs().sum(dim=1) > 0)[:5, 0]
    for i in idx.tolist():
        fp = feat.detach().clone()
        fm = feat.detach().clone()
        fp[i, 3] += 0.5
        fm[i, 3] -= 0.5
        Lp = (quantile_render(mean, ls, quat, op.detach(), fp, cam, K=8)[0] * gout).sum()
        Lm = (quantile_render(mean, ls, quat, op.detach(), fm, cam, K=8)[0] * gout).sum()
        fd = (Lp - Lm).item() / 1.0
        assert abs(fd - gf[i, 3].item()) <= 1e-3 * max(1.0, abs(fd)), (i, fd, gf[i, 3].item())


@pytest.mark.parametrize("P,C,cover", [(3000, 64, 0.8),         # one CTA sums everything
                                       (16385, 16, 0.8),        # two ranges, ragged tail
                                       (8192 * 40 + 77, 8, 0.3),  # many ranges, last-CTA combine
                                       (5000, 8, 0.0)])         # nothing covered: L = 0, zero rows
def test_cosine_loss_matches_oracle(P, C, cover):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    rng = np.random.default_rng(5)
    F = rng.normal(size=(P, C)).astype(np.float32)
    t = rng.normal(size=(P, C)).astype(np.float32)
    F[7] = 0.0
    cnt = (rng.uniform(size=P) < cover).astype(np.uint8)
    loss, grad = q.qr_cosine_loss(torch.from_numpy(F).cuda(), torch.from_numpy(t).cuda(),
                                  torch.from_numpy(cnt).cuda())
    L, gref = oracle.cosine_loss(F, t, cnt > 0)
    assert abs(loss.item() - L) <= 1e-6 * max(1.0, abs(L))
    np.testing.assert_allclose(grad.cpu().numpy(), gref, rtol=0, atol=1e-5 * max(np.abs(gref).max(), 1e-30))


def test_differentiation_config_sampled_pixels():
    """300k-Gaussian room, 640x480, 512-D, K = 8, loss = mean (1 - cos) against
    the dense map of a second Gaussian set; the loss is restricted to sampled
    pixels so the oracle (own forward, own target, own upstream gradient) can
    compute the same gradients."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = scenes.room_scene(seed=0, n=300_000, channels=512)
    g2, f2 = scenes.room_scene(seed=1, n=300_000, channels=512)
    cam = scenes.room_camera(640, 480)
    K = 8
    res = q.render_frame(q.gaussians_to_device(g), torch.from_numpy(f).cuda(), cam, K=K)
    tgt = q.render_frame(q.gaussians_to_device(g2), torch.from_numpy(f2).cuda(), cam, K=K,
                         dense=True)["dense"]
    pix = H.sample_pixels(640, 480, 200, seed=9)
    pr, pix, ref = H.run_oracle(g, f, cam, K, pixels=pix)
    pr2, _, ref2 = H.run_oracle(g2, f2, cam, K, pixels=pix)
    tie = ((ref.tie & compare.Q_TIE_BITS) != 0) | ((ref2.tie & compare.DENSE_TIE_BITS) != 0)
    use = (~tie) & (ref.cnt > 0)
    idx = H.pixel_index(pix, cam.width)
    mask = torch.zeros(cam.width * cam.height, dtype=torch.uint8, device="cuda")
    mask[torch.from_numpy(idx[use]).cuda()] = 1
    loss, gmap = q.qr_cosine_loss(res["out"], tgt, mask)
    fdev = torch.from_numpy(f).cuda()
    gf, ga, gc = q.qr_backward(res["frame"], fdev, None, res["ids"], res["weights"],
                               res["counts"], gmap)
    # the same loss and gradients from the fused call (512 FP32 channels: fused route)
    loss2, gmap2, gf2, ga2, gc2 = q.qr_cosine_backward(res["frame"], fdev, None, res["ids"],
                                                       res["weights"], res["counts"], res["out"],
                                                       tgt, mask=mask)
    torch.cuda.synchronize()
    Lref, gref = oracle.cosine_loss(ref.out_q, ref2.out_dense, use)
    assert abs(loss.item() - Lref) <= 1e-4 * max(1.0, abs(Lref)), (loss.item(), Lref)
    assert abs(loss2.item() - Lref) <= 1e-4 * max(1.0, abs(Lref)), (loss2.item(), Lref)
    ref = oracle.backward(pr, f, K, pix, gref, alpha_min=oracle.ALPHA_MIN_F32,
                          alpha_max=oracle.ALPHA_MAX_F32, with_scales=True)
    # the upstream gradients differ by the forward's and the target's own
    # rounding (~1e-6 of each pixel's gradient), hence 1e-4 of the yardstick
    e1 = _check_all((gf.cpu().numpy(), ga.cpu().numpy(), gc.cpu().numpy()), ref, rel=1e-4)
    e2 = _check_all((gf2.cpu().numpy(), ga2.cpu().numpy(), gc2.cpu().numpy()), ref, rel=1e-4)
    print("differentiation config errors in yardstick units", e1, "fused", e2)


@pytest.mark.parametrize("kind,C,K", [("f32", 64, 8),     # 16 float4 per row: the unfused route
                                      ("f32", 128, 8), ("bf16", 512, 8), ("fp8", 512, 8),
                                      ("bf16", 512, 16)])  # 64-bit tile keys, staged without TMA
def test_cosine_backward_matches_separate_calls(kind, C, K):
    """qr_cosine_backward = qr_cosine_loss then qr_backward, up to summation order."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = H.small_room(n=20000, channels=C)
    cam = scenes.room_camera(150, 110)
    fdev = torch.from_numpy(f).cuda()
    table = {"f32": fdev, "bf16": None, "fp8": None}[kind]
    if kind == "bf16":
        table = q.qr_quantize_bf16(fdev)
    elif kind == "fp8":
        table = q.qr_quantize_fp8(fdev)
    feat_t, scale_t = table if isinstance(table, tuple) else (table, None)
    res = q.render_frame(q.gaussians_to_device(g), table, cam, K=K)
    rng = np.random.default_rng(3)
    tgt = torch.from_numpy(rng.normal(size=(cam.width * cam.height, C)).astype(np.float32)).cuda()
    loss, gmap = q.qr_cosine_loss(res["out"], tgt, res["counts"])
    gf, ga, gc = q.qr_backward(res["frame"], feat_t, scale_t, res["ids"], res["weights"],
                               res["counts"], gmap)
    loss2, gmap2, gf2, ga2, gc2 = q.qr_cosine_backward(res["frame"], feat_t, scale_t, res["ids"],
                                                       res["weights"], res["counts"], res["out"], tgt)
    torch.cuda.synchronize()
    assert abs(loss2.item() - loss.item()) <= 1e-6 * max(1.0, abs(loss.item()))
    _compare("grad map", gmap2.cpu().numpy(), gmap.cpu().numpy().astype(np.float64), 1e-5)
    _compare("feat", gf2.cpu().numpy(), gf.cpu().numpy().astype(np.float64), 1e-5)
    _compare("alpha", ga2.cpu().numpy(), ga.cpu().numpy().astype(np.float64), 1e-4)
    _compare("conic", gc2.cpu().numpy(), gc.cpu().numpy().astype(np.float64), 1e-4)
    assert (res["counts"] > 0).any()


def test_cosine_backward_is_deterministic_and_graph_capturable():
    """Two eager runs give bit-identical gradients (no floating-point atomics
    anywhere), and a CUDA-graph replay of the same call -- whose output
    clearing runs on a forked side stream -- gives the same bits again."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = H.small_room(n=20000, channels=128)
    cam = scenes.room_camera(150, 110)
    fdev = torch.from_numpy(f).cuda()
    res = q.render_frame(q.gaussians_to_device(g), fdev, cam, K=8)
    rng = np.random.default_rng(21)
    tgt = torch.from_numpy(rng.normal(size=(cam.width * cam.height, 128)).astype(np.float32)).cuda()
    args = (res["frame"], fdev, None, res["ids"], res["weights"], res["counts"], res["out"], tgt)
    a = [t.clone() for t in q.qr_cosine_backward(*args)]
    b = [t.clone() for t in q.qr_cosine_backward(*args)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        q.qr_cosine_backward(*args)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        outs = q.qr_cosine_backward(*args)
    for t in outs:
        t.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    for x, y in zip(a, outs):
        assert torch.equal(x, y)
