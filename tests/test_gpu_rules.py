"""GPU parity of the top-K, Stratified-K and Riemann-weight select rules
(qr_select_rule) against the FP64 oracle (or_render_rule), through the C ABI.

Same bar as Algorithm 1: kept ids and counts exact on every pixel the oracle
does not flag (RULE_TIE_BITS: the rule's own decision, the alpha_min border,
equal depths, the T_min stop), features rendered by qr_blend from the rule's
ids and weights within 1e-5 of the mixed relative metric.
"""
import numpy as np
import pytest

import oracle
from oracle import compare
from paper_2512_20927_gb300 import scenes

import gpu_harness as H

pytestmark = pytest.mark.gpu

FEAT_TOL = 1e-5
TAU_TOL = 2e-5      # boundaries: FP32 statistics and normal CDF / inverse (few ulps, |z| <= 2.2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(g, f, cam, rule, K, pixels=None, params_kw=None, max_tie_frac=0.02, label=""):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    params = q.default_params(K, **(params_kw or {}))
    fdev = None if f is None else torch.from_numpy(np.ascontiguousarray(f, np.float32)).cuda()
    res = q.render_frame(q.gaussians_to_device(g), fdev, cam, K=K, params=params, rule=rule)
    torch.cuda.synchronize()
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(cam.width, cam.height) if pixels is None else pixels
    ref = oracle.render_rule(pr, f, rule, K, pix, T_min=float(np.float32(1e-4)),
                             alpha_min=oracle.ALPHA_MIN_F32, alpha_max=oracle.ALPHA_MAX_F32)
    idx = H.pixel_index(pix, cam.width)
    ids = res["ids"].cpu().numpy()[idx]
    cnt = res["counts"].cpu().numpy()[idx].astype(np.int64)
    w = res["weights"].cpu().numpy()[idx]
    tie = (ref.tie & compare.RULE_TIE_BITS) != 0
    same = (ids == ref.ids).all(axis=1) & (cnt == ref.cnt)
    rep = {"pixels": len(idx), "tie_pixels": int(tie.sum()),
           "mismatch_nontie": int((~same & ~tie).sum()), "mismatch_tie": int((~same & tie).sum()),
           "kept_mean": float(cnt.mean())}
    assert rep["mismatch_nontie"] == 0, (label, rep)
    assert rep["tie_pixels"] <= max_tie_frac * rep["pixels"] + 2, (label, rep)
    rep["weight_abs_err_max"] = float(np.abs(w[same] - ref.wq[same]).max()) if same.any() else 0.0
    assert rep["weight_abs_err_max"] <= FEAT_TOL, (label, rep)
    if f is not None:
        out = res["out"].cpu().numpy()[idx]
        err = compare.feature_error(out, ref.out, ref.scale)
        rep["feat_err_max"] = float(err[same].max()) if same.any() else 0.0
        assert rep["feat_err_max"] <= FEAT_TOL, (label, rep)
        assert (out[same & (ref.cnt == 0)] == 0).all()
    if rule == oracle.RULE_STRATIFIED:
        tau = res["tau"].cpu().numpy()[idx]
        ok = ~tie
        rep["tau_err_max"] = float(np.abs(tau[ok] - ref.tau[ok]).max()) if ok.any() else 0.0
        assert rep["tau_err_max"] <= TAU_TOL, (label, rep)
    return rep


RULES = [oracle.RULE_TOPK, oracle.RULE_STRATIFIED, oracle.RULE_RIEMANN]
NAMES = {oracle.RULE_TOPK: "topk", oracle.RULE_STRATIFIED: "stratified",
         oracle.RULE_RIEMANN: "riemann"}


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("K", [1, 4, 8, 32])
def test_tiny_config(rule, K):
    g, f = scenes.tiny_scene()
    rep = _run(g, f, scenes.tiny_camera(), rule, K, label=f"tiny {NAMES[rule]} K={K}")
    print(f"tiny {NAMES[rule]} K={K}", rep)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("tile", [(16, 16), (8, 32)])
def test_room_small_ragged(rule, tile):
    g, f = H.small_room(n=20000, channels=64)
    cam = scenes.room_camera(150, 110)
    rep = _run(g, f, cam, rule, 8, params_kw={"tile_w": tile[0], "tile_h": tile[1]},
               label=f"room {NAMES[rule]} {tile}")
    print(f"room-small {NAMES[rule]} tile {tile}", rep)


@pytest.mark.parametrize("rule", RULES)
def test_indoor_full_size_sampled(rule):
    """The 500k-Gaussian 640x480 512-D workload, on sampled pixels."""
    g, f = scenes.room_scene(seed=0, n=500_000, channels=512)
    cam = scenes.room_camera(640, 480)
    pix = H.sample_pixels(640, 480, 200, seed=4)
    rep = _run(g, f, cam, rule, 8, pixels=pix, label=f"indoor {NAMES[rule]}")
    print(f"indoor sampled {NAMES[rule]}", rep)


@pytest.mark.parametrize("rule", RULES)
def test_deep_lists(rule):
    """Tiles with thousands of Gaussians (several staged batches per pixel,
    ~800 members walked to T_min).  The slab spans 3 m of depth so that FP32
    depth keys rarely collide; the oracle flags 0 (top-K) and 6 (Stratified-K)
    of these 104 pixels."""
    rng = np.random.default_rng(11)
    n = 3000
    mean = np.stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n),
                     rng.uniform(-1.5, 1.5, n)], 1).astype(np.float32)
    g = scenes.Gaussians(mean, np.full((n, 3), -2.0, np.float32),
                         np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                         np.full(n, 0.05, np.float32))
    f = rng.normal(size=(n, 16)).astype(np.float32)
    pix = H.sample_pixels(48, 48, 100, seed=6)
    rep = _run(g, f, scenes.tiny_camera(48, 48), rule, 8, pixels=pix, max_tie_frac=0.06,
               label=f"deep {NAMES[rule]}")
    print(f"deep lists {NAMES[rule]}", rep)


@pytest.mark.parametrize("rule", RULES)
def test_empty_scene(rule):
    g, f = scenes.tiny_scene(n=300)
    g.mean[:, 2] = 10.0      # behind the camera
    import torch
    from paper_2512_20927_gb300 import qrender as q
    cam = scenes.tiny_camera(40, 24)
    res = q.render_frame(q.gaussians_to_device(g), torch.from_numpy(f).cuda(), cam, K=8,
                         rule=rule)
    torch.cuda.synchronize()
    assert (res["counts"] == 0).all() and (res["out"] == 0).all() and (res["ids"] == -1).all()


@pytest.mark.parametrize("K", [1, 4, 8, 16, 32])
def test_riemann_selection_is_algorithm_1(K):
    """App. C changes Algorithm 1's weights only: on every pixel of a frame
    the Riemann rule keeps qr_select's ids and counts bit for bit, its weights
    sum to 1, and each is a crossing count c_j over the total D <= K."""
    import torch
    from paper_2512_20927_gb300 import qrender as q
    g, f = H.small_room(n=20000, channels=16)
    cam = scenes.room_camera(150, 110)
    gdev = q.gaussians_to_device(g)
    a = q.render_frame(gdev, None, cam, K=K)
    b = q.render_frame(gdev, None, cam, K=K, rule=q.QR_RULE_RIEMANN)
    torch.cuda.synchronize()
    assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["counts"], b["counts"])
    w = b["weights"].cpu().numpy().astype(np.float64)
    cnt = b["counts"].cpu().numpy().astype(np.int64)
    kept = cnt > 0
    assert kept.any()
    assert np.abs(w[kept].sum(1) - 1.0).max() <= K * 2e-7
    assert (w[~kept] == 0).all()
    # some total D in counts..K makes every c_j = w_j D a positive integer
    wk, ck = w[kept], cnt[kept]
    found = np.zeros(len(wk), bool)
    for D in range(1, K + 1):
        c = wk * D
        cj = np.rint(c)
        ok = (np.abs(c - cj) <= 1e-5 * D).all(1) & ((cj >= 1) | (wk == 0)).all(1) & (ck <= D)
        found |= ok
    assert found.all()
