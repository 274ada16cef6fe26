"""The contrastive loss of Eq. 2 (Sec. 4.3) on the GPU against the FP64
oracle, through the C ABI: the loss and its gradient on random maps (every
supported width, 2..64 masks, pixels outside every mask), and through the
renderer the gradients of the features, opacities and conics of a room scene
with synthetic patches and patch embeddings.

Tolerances: the loss is a compensated sum of FP32 terms (1e-5 relative); a
pixel's gradient is a sum of M target rows with softmax weights and the
F term, each term a dot product of C channels (FP32 on the CUDA cores for
more than 32 masks; for up to 32, tensor-core TF32 products with both
operands split into hi + lo parts, about 2^-22 of |x||y| each), so it is checked against
its own yardstick (1/n)(sum_j |c_j| max|t^_j| / nf + |sum_j c_j s_j| max|F| / nf^2)
at 2e-5 of it.
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


def _yardstick(F, T, mid, eps=1e-8):
    """Per pixel: the gradient's size without cancellation (see the module doc)."""
    F = np.asarray(F, np.float64)
    T = np.asarray(T, np.float64)
    nf = np.maximum(np.linalg.norm(F, axis=1), eps)
    Tn = T / np.maximum(np.linalg.norm(T, axis=1), eps)[:, None]
    S = (F @ Tn.T) / nf[:, None]
    n = max(int((mid >= 0).sum()), 1)
    y = np.zeros(len(F))
    tmax = np.abs(Tn).max(axis=1)
    for p in np.nonzero(mid >= 0)[0]:
        e = np.exp(S[p])
        e[mid[p]] = 0.0
        c = e / e.sum()
        c[mid[p]] = -1.0
        y[p] = ((np.abs(c) * tmax).sum() / nf[p] + abs(c @ S[p]) * np.abs(F[p]).max() / nf[p] ** 2) / n
    return y


@pytest.mark.parametrize("P,C,M", [(3001, 128, 2), (5000, 256, 7), (4099, 384, 33),
                                   (20000, 512, 64), (777, 512, 16),
                                   # tensor-core path (M <= 32): 16 and 32 target rows, ragged P
                                   (6003, 512, 32), (1999, 128, 17)])
def test_contrastive_loss_matches_oracle(P, C, M):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    rng = np.random.default_rng(P + M)
    F = rng.normal(size=(P, C)).astype(np.float32)
    F[5] = 0.0                                         # |F| below eps
    T = rng.normal(size=(M, C)).astype(np.float32)
    mid = rng.integers(-1, M, P).astype(np.int32)
    loss, grad = q.qr_contrastive_loss(torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda(),
                                       torch.from_numpy(mid).cuda())
    torch.cuda.synchronize()
    L, gref = oracle.contrastive_loss(F, T, mid)
    assert abs(loss.item() - L) <= 1e-5 * max(1.0, abs(L)), (loss.item(), L)
    g = grad.cpu().numpy().astype(np.float64)
    y = _yardstick(F, T, mid)
    err = np.abs(g - gref).max(axis=1)
    on = mid >= 0
    assert (g[~on] == 0).all()
    worst = float((err[on] / y[on]).max())
    assert worst <= 2e-5, worst
    print(f"contrastive P={P} C={C} M={M}: loss {loss.item():.6f} vs {L:.6f}, "
          f"gradient err {worst:.2e} of its yardstick")


def test_contrastive_loss_no_pixels_in_the_loss():
    import torch
    from paper_2512_20927_gb300 import qrender as q
    F = torch.randn(1000, 128, device="cuda")
    T = torch.randn(4, 128, device="cuda")
    mid = torch.full((1000,), -1, dtype=torch.int32, device="cuda")
    loss, grad = q.qr_contrastive_loss(F, T, mid)
    assert loss.item() == 0.0 and (grad == 0).all()


def test_contrastive_backward_through_the_renderer():
    """Room scene, 128-D features, 24 synthetic patches: the gradients of
    features, opacities and conics against the oracle's (its own forward, its
    own Eq. 2 gradient), per Gaussian against the oracle's yardstick; near-tie
    pixels are left out of the loss on both sides."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = H.small_room(n=20000, channels=128)
    cam = scenes.room_camera(150, 110)
    K = 8
    fdev = torch.from_numpy(f).cuda()
    res = q.render_frame(q.gaussians_to_device(g), fdev, cam, K=K)
    pr, pix, ref = H.run_oracle(g, f, cam, K)
    tie = (ref.tie & compare.Q_TIE_BITS) != 0
    M = 24
    mid = scenes.patch_masks(cam.width, cam.height, M, seed=2)
    mid[tie] = -1
    T = scenes.patch_targets(M, 128, seed=5)
    loss, gmap, gf, ga, gc = q.qr_contrastive_backward(
        res["frame"], fdev, None, res["ids"], res["weights"], res["counts"], res["out"],
        torch.from_numpy(T).cuda(), torch.from_numpy(mid).cuda())
    # the same through the two calls
    loss2, gmap2 = q.qr_contrastive_loss(res["out"], torch.from_numpy(T).cuda(),
                                         torch.from_numpy(mid).cuda())
    gf2, ga2, gc2 = q.qr_backward(res["frame"], fdev, None, res["ids"], res["weights"],
                                  res["counts"], gmap2)
    torch.cuda.synchronize()
    assert torch.equal(gmap, gmap2) and torch.equal(gf, gf2) and torch.equal(ga, ga2)
    Lref, gref = oracle.contrastive_loss(ref.out_q, T, mid)
    assert abs(loss.item() - Lref) <= 1e-4 * max(1.0, abs(Lref)), (loss.item(), Lref)
    rf, ra, rc, sf, sa, sc = oracle.backward(pr, f, K, pix, gref, alpha_min=oracle.ALPHA_MIN_F32,
                                             alpha_max=oracle.ALPHA_MAX_F32, with_scales=True)
    worst = {}
    for name, got, want, yard in (("feat", gf, rf, sf), ("alpha", ga, ra, sa), ("conic", gc, rc, sc)):
        err = np.abs(got.cpu().numpy().astype(np.float64) - want)
        if err.ndim == 2 and yard.ndim == 1:
            err = err.max(axis=1)
        assert (err[yard == 0] == 0).all(), name
        worst[name] = float((err[yard > 0] / yard[yard > 0]).max())
        # the two sides' upstream gradients come from their own forwards
        assert worst[name] <= 1e-4, (name, worst[name])
    print("contrastive through the renderer: loss", loss.item(), Lref, "errors", worst)
