"""Pins of the FP64 oracle against facts other than itself.

Every function of ``oracle`` is checked here against a closed form, a library
routine, a hand-derived fixture (tests/golden), an invariant of the paper's
definitions, a finite difference or brute-force enumeration.  A plausible
slip (a dropped term, a wrong sign or index, a transposed operand, '<=' for
'<') fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2512_20927_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _one(mean, log_scale, quat, opacity):
    n = np.asarray(opacity).size
    return scenes.Gaussians(np.asarray(mean, np.float32).reshape(n, 3),
                            np.asarray(log_scale, np.float32).reshape(n, 3),
                            np.asarray(quat, np.float32).reshape(n, 4),
                            np.asarray(opacity, np.float32).reshape(n))


# ---------------------------------------------------------------- Sec. 3
def test_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.normal(size=4).astype(np.float32) * rng.uniform(0.2, 3.0)
        R = oracle.quat_to_rotation(q)
        Rs = Rotation.from_quat(np.array([q[1], q[2], q[3], q[0]], np.float64)).as_matrix()
        np.testing.assert_allclose(R, Rs, atol=1e-12)


def test_covariance_eigendecomposition():
    """Sigma = R S S^T R^T: eigenvalues exp(2 s), eigenvectors the columns of R (Sec. 3)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(2)
    for _ in range(50):
        q = rng.normal(size=4).astype(np.float32)
        ls = rng.normal(-2, 1, size=3).astype(np.float32)
        S = oracle.covariance3d(ls, q)
        R = Rotation.from_quat(np.array([q[1], q[2], q[3], q[0]], np.float64)).as_matrix()
        for k in range(3):
            v = R[:, k]
            np.testing.assert_allclose(S @ v, np.exp(2.0 * float(ls[k])) * v,
                                       rtol=1e-10, atol=1e-14)


def test_projection_axis_aligned_closed_form():
    """On the optical axis an axis-aligned Gaussian projects to diag(fx^2 sx^2, fy^2 sy^2)/z^2 + dilation."""
    cam = scenes.tiny_camera(64, 48)
    ls = np.log(np.array([0.05, 0.02, 0.03]))
    g = _one([0.0, 0.0, 0.5], ls, [1, 0, 0, 0], [0.7])
    pr = oracle.project(g, cam.as_array(), dilation=0.3)
    z = 2.5
    sx, sy = np.exp(ls[:2].astype(np.float32).astype(np.float64))
    assert pr.valid[0] == 1
    np.testing.assert_allclose(pr.depth[0], z, rtol=1e-7)
    np.testing.assert_allclose(pr.mean2d[0], [32.0, 24.0], atol=1e-9)
    np.testing.assert_allclose(pr.cov2d[0], [(cam.fx * sx / z) ** 2 + 0.3, 0.0,
                                             (cam.fy * sy / z) ** 2 + 0.3], rtol=1e-6, atol=1e-9)
    S = np.array([[pr.cov2d[0, 0], pr.cov2d[0, 1]], [pr.cov2d[0, 1], pr.cov2d[0, 2]]])
    A = np.array([[pr.conic[0, 0], pr.conic[0, 1]], [pr.conic[0, 1], pr.conic[0, 2]]])
    np.testing.assert_allclose(A @ S, np.eye(2), atol=1e-12)


def _pinhole(cam, c):
    return np.array([cam.fx * c[0] / c[2] + cam.cx, cam.fy * c[1] / c[2] + cam.cy])


def test_projection_matches_numerical_linearisation():
    """EWA: Sigma' equals the covariance pushed through a finite-difference
    linearisation of the pinhole map applied to a Cholesky factor of Sigma;
    the mean is the pinhole image of the camera-space mean."""
    rng = np.random.default_rng(3)
    cam = scenes.room_camera(320, 240, eye=(0.3, -0.2, 1.4), yaw=0.4, pitch=0.1)
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    n = 40
    fwd = R[2]
    mean = (np.array([0.3, -0.2, 1.4]) + rng.uniform(1.0, 3.0, (n, 1)) * fwd
            + rng.normal(0, 0.4, (n, 3))).astype(np.float32)
    g = _one(mean, rng.normal(-3, 0.5, (n, 3)), rng.normal(size=(n, 4)), rng.uniform(0.1, 0.9, n))
    pr = oracle.project(g, cam.as_array(), dilation=0.0)
    for i in range(n):
        c = R @ mean[i].astype(np.float64) + t
        assert pr.valid[i]
        np.testing.assert_allclose(pr.depth[i], c[2], rtol=1e-12)
        np.testing.assert_allclose(pr.mean2d[i], _pinhole(cam, c), rtol=1e-12)
        Sigma = oracle.covariance3d(g.log_scale[i], g.quat[i])
        L = np.linalg.cholesky(Sigma)
        cols = []
        for k in range(3):
            h = 1e-3 * np.linalg.norm(L[:, k])
            d = L[:, k] / np.linalg.norm(L[:, k])
            # world-space perturbation mapped through the camera, then the pinhole
            jp = (_pinhole(cam, R @ (mean[i] + h * d) + t) - _pinhole(cam, R @ (mean[i] - h * d) + t)) / (2 * h)
            cols.append(jp * np.linalg.norm(L[:, k]))
        M = np.stack(cols, axis=1)
        ref = M @ M.T
        got = np.array([[pr.cov2d[i, 0], pr.cov2d[i, 1]], [pr.cov2d[i, 1], pr.cov2d[i, 2]]])
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_behind_near_plane_is_culled():
    cam = scenes.tiny_camera(32, 32)
    g = _one([[0, 0, 2.9], [0, 0, 2.7], [0, 0, -5]], np.full((3, 3), -3.0),
             [[1, 0, 0, 0]] * 3, [0.5] * 3)
    pr = oracle.project(g, cam.as_array())
    assert list(pr.valid) == [0, 1, 1]   # depths 0.1 (< near 0.2), 0.3, 8


def test_support_area_matches_ellipse():
    """Pixels with alpha' >= 1/255 fill the ellipse q <= 2 ln(255 alpha): area pi r^2 sqrt(det Sigma')."""
    cam = scenes.tiny_camera(128, 128)
    for q, ls, a in [([1, 0, 0, 0], [-2.6, -2.9, -3.0], 0.9),
                     ([0.9, 0.2, -0.3, 0.1], [-2.4, -3.2, -2.8], 0.3),
                     ([0.5, 0.5, 0.5, 0.5], [-3.0, -2.5, -2.7], 0.05)]:
        g = _one([0.05, -0.03, 0.1], ls, q, [a])
        pr = oracle.project(g, cam.as_array())
        r = oracle.render(pr, None, 4, oracle.all_pixels(128, 128), want_q=False, want_dense=False)
        count = int((r.n_members > 0).sum())
        S = np.array([[pr.cov2d[0, 0], pr.cov2d[0, 1]], [pr.cov2d[0, 1], pr.cov2d[0, 2]]])
        r2 = 2.0 * math.log(255.0 * float(np.float32(a)))
        area = math.pi * r2 * math.sqrt(np.linalg.det(S))
        ev = np.linalg.eigvalsh(S)
        a_ax, b_ax = math.sqrt(r2 * ev[1]), math.sqrt(r2 * ev[0])
        perim = math.pi * (3 * (a_ax + b_ax) - math.sqrt((3 * a_ax + b_ax) * (a_ax + 3 * b_ax)))
        assert area > 50
        assert abs(count - area) <= perim, (count, area, perim)


# ---------------------------------------------------------------- Eq. 1 and Algorithm 1
def _golden_scene():
    with open(os.path.join(GOLDEN, "three_layer_stack.json")) as fh:
        gd = json.load(fh)
    c = gd["camera"]
    cam = scenes.Camera(R=np.array(c["R"], np.float32), t=np.array(c["t"], np.float32),
                        fx=c["fx"], fy=c["fy"], cx=c["cx"], cy=c["cy"],
                        width=c["width"], height=c["height"])
    G = gd["gaussians"]
    g = _one(G["mean"], np.full((3, 3), G["log_scale"]), [[1, 0, 0, 0]] * 3, G["alpha"])
    return gd, cam, g, np.array(G["feature"], np.float64)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_golden_three_layer_stack(K):
    gd, cam, g, f = _golden_scene()
    pr = oracle.project(g, cam.as_array())
    np.testing.assert_array_equal(pr.depth, gd["gaussians"]["depth"])
    r = oracle.render(pr, f, K, np.array([gd["camera"]["pixel"]]), T_min=0.0)
    exp = gd["expected"][f"K{K}"]
    m = len(exp["ids"])
    assert r.cnt[0] == m
    assert list(r.ids[0, :m]) == exp["ids"] and (r.ids[0, m:] == -1).all()
    assert r.tq[0] == exp["T_Q"]
    np.testing.assert_allclose(r.out_q[0], exp["feature"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.out_dense[0], gd["expected"]["dense"]["feature"], rtol=0, atol=0)
    assert r.t_final[0] == gd["expected"]["dense"]["T_final"]


def test_single_gaussian_reproduces_its_feature():
    """One Gaussian: it is selected iff alpha' > 1/(K+1), and then the output is f itself."""
    cam = scenes.tiny_camera(64, 64)
    g = _one([0.02, 0.01, 0.0], [-2.3, -2.6, -2.5], [0.8, 0.1, 0.5, -0.2], [0.85])
    f = np.array([[0.3, -1.7, 2.5, 0.01]])
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(64, 64)
    for K in (1, 4, 8, 32):
        r = oracle.render(pr, f, K, pix)
        a = r.wq[:, 0]  # normalised weight is 1 when selected
        members = r.n_members > 0
        # alpha' of each member pixel from the closed form
        sel = r.cnt == 1
        assert (r.cnt <= 1).all()
        np.testing.assert_array_equal(r.ids[sel, 0], 0)
        np.testing.assert_allclose(a[sel], 1.0, rtol=1e-14)
        np.testing.assert_allclose(r.out_q[sel], np.broadcast_to(f, (sel.sum(), 4)), rtol=1e-14)
        assert (r.out_q[~sel] == 0).all()
        # the selected region is exactly alpha' > 1/(K+1): compare with Eq.1's weight (= alpha')
        alpha_p = r.out_dense[:, 0] / f[0, 0]
        np.testing.assert_array_equal(sel, members & (alpha_p > 1.0 / (K + 1) * (1 + 1e-12)) |
                                      (sel & (np.abs(alpha_p - 1.0 / (K + 1)) < 1e-12)))


def test_k1_selects_the_median_transmittance_gaussian():
    rng = np.random.default_rng(4)
    for _ in range(200):
        n = rng.integers(1, 40)
        a = rng.uniform(1 / 255, 0.99, n) ** rng.uniform(0.5, 4)
        a = np.clip(a, 1 / 255, 0.99)
        sel, w, tq, npro = oracle.qrender_list(a, 1)
        T = np.cumprod(1.0 - a)
        below = np.nonzero(T < 0.5)[0]
        if len(below) == 0:
            assert not sel.any()
            continue
        i = below[0]
        assert np.nonzero(sel)[0].tolist() == [i]
        assert npro == i + 1
        np.testing.assert_allclose(w[i], a[i], rtol=0)
        np.testing.assert_allclose(tq, 1 - a[i], rtol=0)


def test_large_k_limit_selects_every_visited_gaussian():
    """If every step lowers T by at least 1/(K+1), each visited Gaussian crosses a boundary."""
    rng = np.random.default_rng(5)
    for K in (2, 4, 8, 16):
        for _ in range(50):
            a, T = [], 1.0
            while T >= 1.0 / (K + 1):
                lo = (1.0 / (K + 1)) / T
                ai = rng.uniform(min(lo * 1.0001, 0.99), 0.99) if lo < 0.99 else 0.99
                a.append(ai)
                T *= 1 - ai
            a = np.array(a + list(rng.uniform(0.01, 0.9, 5)))
            sel, w, tq, npro = oracle.qrender_list(a, K)
            nvis = npro
            assert sel[:nvis].all() and not sel[nvis:].any()
            wd, tf, used = oracle.dense_list(a[:nvis], 0.0)
            np.testing.assert_allclose(w[:nvis], wd, rtol=1e-14)
            np.testing.assert_allclose(tq, np.prod(1 - a[:nvis]), rtol=1e-14)


def test_loop_and_closed_form_selection_agree():
    rng = np.random.default_rng(6)
    for K in (1, 2, 3, 5, 8, 16, 32):
        for _ in range(300):
            n = int(rng.integers(0, 80))
            mode = rng.integers(0, 3)
            if mode == 0:
                a = rng.uniform(1 / 255, 0.99, n)
            elif mode == 1:
                a = np.clip(rng.exponential(0.05, n), 1 / 255, 0.99)
            else:
                a = rng.choice([1 / 255, 0.01, 0.1, 0.5, 0.99], n)
            sel, w, tq, npro = oracle.qrender_list(a, K)
            sel2 = oracle.qselect_closed_form(a, K)
            np.testing.assert_array_equal(sel, sel2)
            assert sel.sum() <= K


def test_weight_invariants_tiny_scene():
    g, f = scenes.tiny_scene()
    cam = scenes.tiny_camera()
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(cam.width, cam.height)
    K = 8
    r = oracle.render(pr, f, K, pix, T_min=0.0)
    has = r.cnt > 0
    assert (r.cnt <= K).all()
    assert (r.wq >= 0).all()
    np.testing.assert_allclose(r.wq[has].sum(axis=1), 1.0, rtol=0, atol=1e-12)
    assert (r.wq[~has] == 0).all() and (r.ids[~has] == -1).all() and (r.out_q[~has] == 0).all()
    # selected ids are a depth-ordered subsequence
    for p in np.nonzero(has)[0][:2000]:
        ids = r.ids[p, :r.cnt[p]]
        d = pr.depth[ids]
        assert (np.diff(d) >= 0).all()
        assert len(set(ids.tolist())) == len(ids)
    # unnormalised quantile weights telescope to 1 - T^Q
    wun = r.wq * (1.0 - r.tq)[:, None]
    np.testing.assert_allclose(wun.sum(axis=1), 1.0 - r.tq, atol=1e-12)
    # the output is the weighted sum of the selected rows
    ref = np.einsum("pk,pkc->pc", r.wq, f.astype(np.float64)[np.maximum(r.ids, 0)])
    np.testing.assert_allclose(r.out_q, ref, atol=1e-12)


def test_constant_feature_invariants():
    """All Gaussians sharing one colour c: Eq. 1 gives (1 - T_final) c and Q-Render gives c."""
    g, _ = scenes.tiny_scene(seed=3, n=500)
    cam = scenes.tiny_camera(64, 64)
    c = np.array([0.2, -0.7, 1.3])
    f = np.tile(c, (g.n, 1))
    pr = oracle.project(g, cam.as_array())
    r = oracle.render(pr, f, 8, oracle.all_pixels(64, 64), T_min=0.0)
    np.testing.assert_allclose(r.out_dense, (1.0 - r.t_final)[:, None] * c, atol=1e-12)
    has = r.cnt > 0
    np.testing.assert_allclose(r.out_q[has], np.broadcast_to(c, (has.sum(), 3)), atol=1e-12)


def test_dense_list_matches_cumprod_and_tmin_rule():
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = rng.uniform(1 / 255, 0.99, int(rng.integers(1, 60)))
        w, tf, used = oracle.dense_list(a, 0.0)
        Tb = np.concatenate([[1.0], np.cumprod(1 - a)[:-1]])
        np.testing.assert_allclose(w, Tb * a, rtol=1e-13)
        np.testing.assert_allclose(w.sum(), 1 - np.prod(1 - a), atol=1e-13)
        assert used == len(a)
        # T_min: stop before the first Gaussian whose test transmittance falls below it
        tmin = 10 ** rng.uniform(-4, -0.5)
        w2, tf2, used2 = oracle.dense_list(a, tmin)
        T = np.cumprod(1 - a)
        stop = np.nonzero(T < tmin)[0]
        expect_used = stop[0] if len(stop) else len(a)
        assert used2 == expect_used
        np.testing.assert_allclose(w2[:used2], w[:used2], rtol=0)
        assert (w2[used2:] == 0).all()


def test_error_decreases_with_k_on_smooth_features():
    """Appendix C trend (not a pin, not a bound): with a feature that varies
    smoothly along the ray and per-Gaussian opacities comparable to the
    segment width, Q-Render approaches the normalised dense blend as K grows.
    With many faint Gaussians (alpha' << 1/(K+1)) the error is not monotone in
    K, because Algorithm 1 weights a quantile Gaussian by T^Q alpha' rather
    than by the segment width; the test stays in the regime where the trend
    holds and records that limit."""
    rng = np.random.default_rng(8)
    errs = {K: [] for K in (2, 4, 16, 32, 64)}
    for _ in range(300):
        n = 200
        a = np.clip(rng.uniform(0.05, 0.3, n), 1 / 255, 0.99)
        z = np.sort(rng.uniform(0, 1, n))
        f = np.sin(3 * z)
        wd, tf, _ = oracle.dense_list(a, 0.0)
        dense_norm = (wd * f).sum() / (1 - tf)
        for K in errs:
            sel, w, tq, _ = oracle.qrender_list(a, K)
            q = (w * f).sum() / (1 - tq)
            errs[K].append(abs(q - dense_norm))
    e = {K: float(np.mean(v)) for K, v in errs.items()}
    assert e[64] < e[32] < e[16] < e[4]
    assert e[64] < 0.5 * e[2]


# ---------------------------------------------------------------- backward
def _linear_loss(pr, f, K, pix, g):
    r = oracle.render(pr, f, K, pix, want_dense=False)
    return float((r.out_q * g).sum()), r


def test_backward_matches_finite_differences():
    """Central differences of the FP64 forward against the analytic backward."""
    rng = np.random.default_rng(9)
    n = 200
    gs = scenes.room_gaussians(rng, 20000)
    cam = scenes.room_camera(32, 32)
    pr_all = oracle.project(gs, cam.as_array())
    # keep 200 visible Gaussians that land near the crop
    near = np.nonzero(pr_all.valid & (np.abs(pr_all.mean2d[:, 0] - 16) < 20) &
                      (np.abs(pr_all.mean2d[:, 1] - 16) < 20))[0][:n]
    sub = scenes.Gaussians(gs.mean[near], gs.log_scale[near], gs.quat[near], gs.opacity[near])
    pr = oracle.project(sub, cam.as_array())
    C, K = 6, 8
    f = rng.normal(size=(len(near), C))
    pix = oracle.all_pixels(32, 32)
    g = rng.normal(size=(len(pix), C))
    L0, r0 = _linear_loss(pr, f, K, pix, g)
    gf, ga, gc = oracle.backward(pr, f, K, pix, g)
    # features: the map is linear in f
    for i in rng.choice(len(near), 10, replace=False):
        fp, fm = f.copy(), f.copy()
        fp[i, 2] += 1e-3
        fm[i, 2] -= 1e-3
        fd = (_linear_loss(pr, fp, K, pix, g)[0] - _linear_loss(pr, fm, K, pix, g)[0]) / 2e-3
        np.testing.assert_allclose(gf[i, 2], fd, rtol=1e-7, atol=1e-9)
    checked = 0
    for i in np.argsort(-np.abs(ga))[:25]:
        for what, idx in (("alpha", None), ("conic", 0), ("conic", 1), ("conic", 2)):
            h = 1e-7 * (abs(pr.alpha[i]) if what == "alpha" else abs(pr.conic[i, idx]) + 1e-3)
            vals = []
            sels = []
            for s in (+1, -1):
                p2 = oracle.Projected(pr.mean2d, pr.conic.copy(), pr.cov2d, pr.depth,
                                      pr.alpha.copy(), pr.valid)
                if what == "alpha":
                    p2.alpha[i] += s * h
                else:
                    p2.conic[i, idx] += s * h
                L, r = _linear_loss(p2, f, K, pix, g)
                vals.append(L)
                sels.append(r.ids)
            if not (np.array_equal(sels[0], r0.ids) and np.array_equal(sels[1], r0.ids)):
                continue  # the perturbation moved a selection boundary
            fd = (vals[0] - vals[1]) / (2 * h)
            an = ga[i] if what == "alpha" else gc[i, idx]
            assert abs(an - fd) <= 1e-5 * max(1.0, abs(fd)), (what, idx, an, fd)
            checked += 1
    assert checked >= 40


def test_backward_scales_bound_the_gradients():
    """The per-Gaussian yardsticks of the backward (sums of the magnitudes of
    each gradient's parts) bound the gradients, and equal them where nothing
    can cancel: with non-negative features and upstream gradient, the feature
    yardstick is sum_p |w| max|g| >= |dL/df| and for a single selected
    Gaussian per pixel the opacity yardstick equals |dL/dalpha| summed over
    pixels of one sign."""
    rng = np.random.default_rng(12)
    g, f = scenes.tiny_scene(seed=4, n=300, channels=8)
    cam = scenes.tiny_camera(48, 48)
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(48, 48)
    gout = rng.normal(size=(len(pix), 8))
    gf, ga, gc, sf, sa, sc = oracle.backward(pr, f, 8, pix, gout, with_scales=True)
    assert (np.abs(gf).max(axis=1) <= sf * (1 + 1e-12) + 1e-300).all()
    assert (np.abs(ga) <= sa * (1 + 1e-12) + 1e-300).all()
    assert (np.abs(gc) <= sc * (1 + 1e-12) + 1e-300).all()
    assert ((sf > 0) == (np.abs(gf).max(axis=1) > 0)).all()
    # no cancellation: positive features and gradients, feature yardstick tight
    fpos, gpos = np.abs(f), np.ones_like(gout)
    gf, ga, gc, sf, sa, sc = oracle.backward(pr, fpos, 8, pix, gpos, with_scales=True)
    np.testing.assert_allclose(np.abs(gf).max(axis=1), sf, rtol=1e-12, atol=1e-300)
    # K = 1 keeps one Gaussian per pixel with normalised weight 1: F = f_j and
    # dL/da_j = 0 exactly (the normalisation removes a_j), while the yardstick
    # of its cancelling parts stays positive
    gf, ga, gc, sf, sa, sc = oracle.backward(pr, fpos, 1, pix, gpos, with_scales=True)
    sel = sf > 0
    assert (np.abs(ga[sel]) <= 1e-12 * sa[sel]).all() and (sa[sel] > 0).all()


def test_cosine_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(10)
    F = rng.normal(size=(20, 7))
    t = rng.normal(size=(20, 7))
    mask = rng.uniform(size=20) < 0.7
    F[3] = 0.0
    L, g = oracle.cosine_loss(F, t, mask)
    for p in range(20):
        for c in range(7):
            if p == 3:
                continue
            Fp, Fm = F.copy(), F.copy()
            Fp[p, c] += 1e-6
            Fm[p, c] -= 1e-6
            fd = (oracle.cosine_loss(Fp, t, mask)[0] - oracle.cosine_loss(Fm, t, mask)[0]) / 2e-6
            np.testing.assert_allclose(g[p, c], fd, atol=1e-8)
    # cos of identical directions is 1, opposite is -1
    L1, _ = oracle.cosine_loss(t * 3.0, t, np.ones(20, bool))
    L2, _ = oracle.cosine_loss(-t, t, np.ones(20, bool))
    assert abs(L1) < 1e-12 and abs(L2 - 2.0) < 1e-12


# ---------------------------------------------------------------- storage formats
def _f32_sample(rng, n):
    bits = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 448.0, 464.0, 480.0,
                        2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -11, 1e-30, 65504.0,
                        np.float32(3.3895314e38)], np.float32)
    return np.concatenate([x, special, rng.normal(0, 50, n).astype(np.float32)])


def test_bf16_encode_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = _f32_sample(rng, 1 << 20)
    ours = oracle.bf16_encode(x)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    fin = np.isfinite(x)
    np.testing.assert_array_equal(ours[fin], ref[fin])
    assert np.isnan(oracle.bf16_decode(ours[np.isnan(x)])).all()
    np.testing.assert_array_equal(oracle.bf16_decode(ours[fin]),
                                  torch.from_numpy(ref[fin].view(np.int16)).view(torch.bfloat16)
                                  .float().numpy().astype(np.float64))


def test_fp8_e4m3_matches_torch_within_range():
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    dec = oracle.fp8_decode(codes)
    ref = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).float().numpy()
    nan = np.isnan(ref)
    assert set(np.nonzero(nan)[0].tolist()) == {0x7f, 0xff}
    np.testing.assert_array_equal(dec[~nan], ref[~nan].astype(np.float64))
    assert np.isnan(dec[nan]).all()
    rng = np.random.default_rng(12)
    x = _f32_sample(rng, 1 << 20)
    x = x[np.isfinite(x) & (np.abs(x) < 464.0)]
    ours = oracle.fp8_encode(x)
    ref = torch.from_numpy(x.copy()).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_fp8_saturation_by_definition():
    x = np.array([448.0, 463.9, 464.0, 479.0, 1e6, np.inf, -np.inf, -500.0, np.nan], np.float32)
    got = oracle.fp8_encode(x)
    assert list(got[:8]) == [0x7e, 0x7e, 0x7e, 0x7e, 0x7e, 0x7e, 0xfe, 0xfe]
    assert got[8] in (0x7f, 0xff)


def test_fp8_rows_round_trip_error_bound():
    """Per-row scaling: decoded rows are within half an E4M3 step (2^-4 relative) of the input."""
    rng = np.random.default_rng(13)
    f = scenes.unit_features(rng, 300, 64)
    f[0] = 0.0
    codes, scale = oracle.fp8_quantize_rows(f)
    assert scale[0] == 1.0 and (codes[0] == 0).all()
    mx = np.abs(f).max(axis=1)
    np.testing.assert_array_equal(scale[1:], (mx[1:] / np.float32(448.0)).astype(np.float32))
    back = oracle.fp8_dequantize_rows(codes, scale)
    err = np.abs(back - f)
    # normal range: relative 2^-4; subnormal range: absolute 2^-10 * scale
    bound = np.maximum(np.abs(f) * 2.0 ** -4, 2.0 ** -10 * scale[:, None]) * 1.0001
    assert (err <= bound).all()


def test_cosine_loss_through_the_render_matches_finite_differences():
    """The composition the fused loss + backward computes: the cosine loss of
    the rendered map, differentiated through Algorithm 1 into the features and
    the opacities, against central differences of the whole FP64 pipeline."""
    rng = np.random.default_rng(12)
    gs = scenes.room_gaussians(rng, 20000)
    cam = scenes.room_camera(24, 24)
    pr_all = oracle.project(gs, cam.as_array())
    near = np.nonzero(pr_all.valid & (np.abs(pr_all.mean2d[:, 0] - 12) < 16) &
                      (np.abs(pr_all.mean2d[:, 1] - 12) < 16))[0][:150]
    sub = scenes.Gaussians(gs.mean[near], gs.log_scale[near], gs.quat[near], gs.opacity[near])
    pr = oracle.project(sub, cam.as_array())
    C, K = 5, 4
    f = rng.normal(size=(len(near), C))
    pix = oracle.all_pixels(24, 24)
    tgt = rng.normal(size=(len(pix), C))

    def loss(p, feat):
        r = oracle.render(p, feat, K, pix, want_dense=False)
        L, gmap = oracle.cosine_loss(r.out_q, tgt, r.cnt > 0)
        return L, gmap, r

    L0, gmap, r0 = loss(pr, f)
    gf, ga, _ = oracle.backward(pr, f, K, pix, gmap)
    for i in rng.choice(len(near), 8, replace=False):
        for c in (0, 3):
            fp, fm = f.copy(), f.copy()
            fp[i, c] += 1e-5
            fm[i, c] -= 1e-5
            fd = (loss(pr, fp)[0] - loss(pr, fm)[0]) / 2e-5
            assert abs(gf[i, c] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, c, gf[i, c], fd)
    checked = 0
    for i in np.argsort(-np.abs(ga))[:12]:
        h = 1e-7 * abs(pr.alpha[i])
        vals, same = [], True
        for s in (+1, -1):
            p2 = oracle.Projected(pr.mean2d, pr.conic, pr.cov2d, pr.depth, pr.alpha.copy(), pr.valid)
            p2.alpha[i] += s * h
            L, _, r = loss(p2, f)
            vals.append(L)
            same &= np.array_equal(r.ids, r0.ids)
        if not same:
            continue  # the perturbation moved a selection boundary
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(ga[i] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(ga).max()), (i, ga[i], fd)
        checked += 1
    assert checked >= 6


# ---------------------------------------------------------------- contrastive loss (Eq. 2)
def test_contrastive_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(31)
    P, C, M = 40, 12, 5
    F = rng.normal(size=(P, C))
    F[3] = 0.0                                   # |F| <= eps: constant normaliser
    T = rng.normal(size=(M, C))
    mid = rng.integers(-1, M, P)
    L, g = oracle.contrastive_loss(F, T, mid)
    h = 1e-6
    for p in (0, 1, 2, 5, 7, 11):
        for c in (0, 4, 11):
            Fp, Fm = F.copy(), F.copy()
            Fp[p, c] += h
            Fm[p, c] -= h
            fd = (oracle.contrastive_loss(Fp, T, mid)[0] - oracle.contrastive_loss(Fm, T, mid)[0]) / (2 * h)
            assert abs(fd - g[p, c]) <= 1e-6 * max(1.0, abs(fd)), (p, c, fd, g[p, c])
    # pixels outside every mask neither count nor get a gradient
    assert (g[mid < 0] == 0).all()


def test_contrastive_loss_scale_invariance_and_two_masks():
    """Cosine similarity ignores the length of F: L(cF) = L(F) and
    F . dL/dF_p = 0 on every pixel.  With two masks the denominator of Eq. 2
    holds the other mask alone, so the pixel's term is s_other - s_own."""
    rng = np.random.default_rng(32)
    P, C = 30, 9
    F = rng.normal(size=(P, C))
    T = rng.normal(size=(4, C))
    mid = rng.integers(0, 4, P)
    L, g = oracle.contrastive_loss(F, T, mid)
    L2, _ = oracle.contrastive_loss(3.7 * F, T, mid)
    assert abs(L - L2) <= 1e-13
    np.testing.assert_allclose((F * g).sum(axis=1), 0.0, atol=1e-15)
    T2 = T[:2]
    mid2 = rng.integers(0, 2, P)
    L, _ = oracle.contrastive_loss(F, T2, mid2)
    cosv = (F @ T2.T) / (np.linalg.norm(F, axis=1)[:, None] * np.linalg.norm(T2, axis=1)[None, :])
    want = np.mean([cosv[p, 1 - mid2[p]] - cosv[p, mid2[p]] for p in range(P)])
    assert abs(L - want) <= 1e-13
