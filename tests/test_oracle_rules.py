"""Pins of the oracle's other select rules: top-K (the comparison renderer of
Sec. 4.2 and the complexity table), Stratified-K (App. E) and the
Riemann-weight form of Algorithm 1 (App. C).

Top-K is pinned against a full stable sort of the Eq. 1 weights (the oracle
keeps a running set of K instead), against the dense blend when K covers the
whole walk, and at K = 1.  Stratified-K is pinned by its defining
properties, each checked with independent tools: pass 1's mean and standard
deviation equal numpy's over the dense walk's transmittances (numpy cumprod),
the boundaries are equally spaced in scipy's normal CDF over [0, 1], the
selection equals the closed form "visited and the count of boundaries above T
grows", and with fewer than two blended Gaussians it is Algorithm 1.  The
Riemann-weight form (App. C) is pinned to Algorithm 1's selection, to a numpy
count of the boundaries crossed, to special cases, and to App. C's own error
bound M / (2 (K + 1)) on a smooth integrand.
"""
import numpy as np
import pytest

import oracle
from paper_2512_20927_gb300 import scenes

sp = pytest.importorskip("scipy.special")


def _dense_weights(a, T_min):
    """Eq. 1 weights of the walk and how many entries it blends (numpy)."""
    T = np.concatenate([[1.0], np.cumprod(1.0 - a)])
    n = len(a)
    if T_min > 0:
        below = np.nonzero(T[1:] < T_min)[0]
        n = int(below[0]) if below.size else len(a)
    return T[:n] * a[:n], n, T[1:n + 1]


def _random_alphas(rng, n):
    a = np.exp(rng.uniform(np.log(1.0 / 255), np.log(0.99), n))
    a[rng.random(n) < 0.1] = 0.99
    return a


# --------------------------------------------------------------------------- top-K
@pytest.mark.parametrize("K", [1, 2, 4, 8, 16, 32])
def test_topk_equals_a_full_stable_sort(K):
    rng = np.random.default_rng(K)
    for trial in range(300):
        n = int(rng.integers(0, 80))
        a = _random_alphas(rng, n)
        if trial % 5 == 0 and n > 3:          # equal weights: the earlier entry wins
            a[:] = 0.01
        T_min = 1e-4 if trial % 2 else 0.0
        sel, w, nused = oracle.topk_list(a, K, T_min)
        wd, n_ref, _ = _dense_weights(a, T_min)
        assert nused == n_ref
        order = np.argsort(-wd, kind="stable")[:K]
        want = np.zeros(n, bool)
        want[order] = True
        np.testing.assert_array_equal(sel, want)
        np.testing.assert_allclose(w[sel], wd[want[:n_ref]], rtol=1e-15)
        assert (w[~sel] == 0).all()


def test_topk_render_with_k_covering_the_walk_is_the_normalised_dense_blend():
    g, f = scenes.tiny_scene(seed=1, n=400, channels=6)
    cam = scenes.tiny_camera(40, 40)
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(40, 40)
    dense = oracle.render(pr, f, 8, pix, T_min=1e-4)
    K = 32
    rr = oracle.render_rule(pr, f, oracle.RULE_TOPK, K, pix, T_min=1e-4)
    # pixels whose dense walk blends at most K Gaussians keep all of them
    small = (rr.n_proc <= K) & (rr.n_proc > 0)
    assert small.sum() > 100
    want = dense.out_dense[small] / (1.0 - dense.t_final[small])[:, None]
    np.testing.assert_allclose(rr.out[small], want, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(rr.cnt[small], rr.n_proc[small])
    none = rr.n_proc == 0
    assert (rr.out[none] == 0).all() and (rr.cnt[none] == 0).all()


def test_topk_k1_renders_the_largest_weight_gaussian():
    g, f = scenes.tiny_scene(seed=2, n=400, channels=6)
    cam = scenes.tiny_camera(40, 40)
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(40, 40)
    rr = oracle.render_rule(pr, f, oracle.RULE_TOPK, 1, pix, T_min=1e-4)
    has = rr.cnt == 1
    assert has.sum() > 100 and (rr.cnt <= 1).all()
    np.testing.assert_array_equal(rr.out[has], f[rr.ids[has, 0]].astype(np.float64))
    np.testing.assert_allclose(rr.wq[has, 0], 1.0, rtol=0, atol=1e-15)


def test_topk_weights_and_ids_invariants():
    g, f = scenes.tiny_scene(seed=3, n=600, channels=4)
    cam = scenes.tiny_camera(48, 48)
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(48, 48)
    K = 4
    rr = oracle.render_rule(pr, f, oracle.RULE_TOPK, K, pix, T_min=1e-4)
    ref = oracle.render(pr, None, K, pix, want_q=False, want_dense=False, max_members=256)
    assert (rr.cnt <= K).all()
    for p in range(len(pix)):
        c = rr.cnt[p]
        if c == 0:
            continue
        assert abs(rr.wq[p, :c].sum() - 1.0) <= 1e-12 and (rr.wq[p, :c] > 0).all()
        mem = list(ref.members[p][ref.members[p] >= 0])
        pos = [mem.index(i) for i in rr.ids[p, :c]]
        assert pos == sorted(pos)                   # depth order, a subsequence of I(p)
        assert (rr.ids[p, c:] == -1).all()


# --------------------------------------------------------------------------- Stratified-K
@pytest.mark.parametrize("K", [1, 4, 8, 16, 40])
def test_stratified_statistics_and_boundary_spacing(K):
    rng = np.random.default_rng(50 + K)
    tested = 0
    for trial in range(200):
        n = int(rng.integers(2, 90))
        a = _random_alphas(rng, n)
        T_min = 1e-4 if trial % 2 else 0.0
        sel, w, tq, nproc, tau, (mu, sigma, nb) = oracle.stratified_list(a, K, T_min)
        _, n_ref, Ts = _dense_weights(a, T_min)
        assert nb == n_ref
        if nb < 2:
            np.testing.assert_allclose(tau, 1.0 - np.arange(1, K + 1) / (K + 1), rtol=0, atol=0)
            continue
        np.testing.assert_allclose(mu, Ts.mean(), rtol=1e-13)
        np.testing.assert_allclose(sigma, Ts.std(), rtol=1e-9, atol=1e-300)
        tested += 1
        # equally spaced in the normal CDF between Phi(-mu/s) and Phi((1-mu)/s)
        ulo, uhi = sp.ndtr(-mu / sigma), sp.ndtr((1.0 - mu) / sigma)
        u = sp.ndtr((tau - mu) / sigma)
        want = ulo + (uhi - ulo) * (1.0 - np.arange(1, K + 1) / (K + 1))
        np.testing.assert_allclose(u, want, rtol=0, atol=1e-12)
        assert (np.diff(tau) < 0).all() and tau[0] < 1.0 and tau[-1] > 0.0
    assert tested > 100


@pytest.mark.parametrize("K", [1, 4, 8, 16])
def test_stratified_selection_matches_the_closed_form(K):
    """Pass 2 written a second way: entry i is kept iff every earlier test
    transmittance stayed >= tau_K and the number of boundaries above T grows
    at i."""
    rng = np.random.default_rng(70 + K)
    for trial in range(300):
        n = int(rng.integers(0, 60))
        a = _random_alphas(rng, n)
        sel, w, tq, nproc, tau, _ = oracle.stratified_list(a, K, 1e-4)
        T = np.concatenate([[1.0], np.cumprod(1.0 - a)])
        cnt = lambda t: int((t < tau).sum())  # noqa: E731
        want = np.zeros(n, bool)
        visited = True
        for i in range(n):
            want[i] = visited and cnt(T[i + 1]) > cnt(T[i])
            if visited and T[i + 1] < tau[-1]:
                visited = False
                assert nproc == i + 1
        np.testing.assert_array_equal(sel, want)
        # weights: T^Q alpha' over the kept subset, telescoping to 1 - T^Q
        np.testing.assert_allclose(w.sum(), 1.0 - tq, rtol=1e-12, atol=1e-15)
        kept = a[sel]
        Tq = np.concatenate([[1.0], np.cumprod(1.0 - kept)])
        np.testing.assert_allclose(w[sel], Tq[:-1] * kept, rtol=1e-13)


def test_stratified_with_one_blended_gaussian_is_algorithm_1():
    rng = np.random.default_rng(8)
    for _ in range(200):
        K = int(rng.integers(1, 20))
        n = int(rng.integers(1, 30))
        a = _random_alphas(rng, n)
        T_min = (1.0 - a[0]) * 0.999 * (1.0 - a[1]) if n > 1 else 1e-4   # only the first blends
        sel, w, tq, nproc, tau, (_, _, nb) = oracle.stratified_list(a, K, T_min)
        if nb != 1:
            continue
        s2, w2, tq2, np2 = oracle.qrender_list(a, K)
        np.testing.assert_array_equal(sel, s2)
        np.testing.assert_allclose(w, w2, rtol=0, atol=0)
        assert nproc == np2 and tq == tq2


def test_stratified_render_invariants():
    g, f = scenes.tiny_scene(seed=5, n=600, channels=4)
    cam = scenes.tiny_camera(48, 48)
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(48, 48)
    K = 8
    rr = oracle.render_rule(pr, f, oracle.RULE_STRATIFIED, K, pix, T_min=1e-4)
    assert (rr.cnt <= K).all() and (rr.cnt > 0).sum() > 200
    for p in np.nonzero(rr.cnt > 0)[0]:
        c = rr.cnt[p]
        assert abs(rr.wq[p, :c].sum() - 1.0) <= 1e-12
        np.testing.assert_allclose(rr.out[p], rr.wq[p, :c] @ f[rr.ids[p, :c]].astype(np.float64),
                                   rtol=1e-12, atol=1e-12)
        assert (np.diff(rr.tau[p]) <= 0).all()


# ----------------------------------------------------------------------- Riemann weights
@pytest.mark.parametrize("K", [1, 2, 4, 8, 16, 32])
def test_riemann_selection_is_algorithm_1_and_weights_count_crossings(K):
    """App. C's right Riemann sum: the selection is Algorithm 1's, and each
    kept Gaussian weighs the number of boundaries 1 - j/(K+1) that the
    transmittance crosses at it -- written here with numpy's cumprod and a
    direct count, independently of the oracle's walk."""
    rng = np.random.default_rng(90 + K)
    bounds = 1.0 - np.arange(1, K + 1) / (K + 1)
    for trial in range(300):
        n = int(rng.integers(0, 60))
        a = _random_alphas(rng, n)
        sel, w, nproc = oracle.riemann_list(a, K)
        s1, _, _, np1 = oracle.qrender_list(a, K)
        np.testing.assert_array_equal(sel, s1)
        assert nproc == np1
        T = np.concatenate([[1.0], np.cumprod(1.0 - a)])
        crossed = lambda t: int((t < bounds).sum())  # noqa: E731
        want = np.zeros(n)
        for i in range(nproc):
            want[i] = crossed(T[i + 1]) - crossed(T[i])
        np.testing.assert_array_equal(w[sel], want[sel])
        assert (w[~sel] == 0).all()
        # every boundary crossed before the walk stops is counted once
        assert w.sum() == crossed(T[nproc]) if nproc else w.sum() == 0
        if nproc < n or (n and T[n] < 1.0 / (K + 1)):
            assert w.sum() == K


def test_riemann_special_cases():
    # K = 1: one boundary, one kept Gaussian with weight 1 (Algorithm 1's as well)
    a = np.array([0.2, 0.3, 0.5, 0.9])
    sel, w, _ = oracle.riemann_list(a, 1)
    assert sel.sum() == 1 and w[sel][0] == 1.0
    # one Gaussian crossing every boundary at once takes all K counts
    sel, w, nproc = oracle.riemann_list(np.array([0.95, 0.5]), 8)
    assert sel.tolist() == [True, False] and w[0] == 8.0 and nproc == 1
    # equal steps of one segment each: uniform weights
    K = 4
    T = 1.0 - (np.arange(1, K + 1) + 0.5) / (K + 1)       # one boundary between steps
    a = 1.0 - T / np.concatenate([[1.0], T[:-1]])
    sel, w, _ = oracle.riemann_list(a, K)
    assert sel.all() and (w == 1.0).all()


def test_riemann_render_invariants():
    """Rendered with the rule: weights k_j / sum k, summing to 1, rational with
    the boundaries crossed as denominator; ids equal Algorithm 1's."""
    g, f = scenes.tiny_scene(seed=6, n=600, channels=4)
    cam = scenes.tiny_camera(48, 48)
    pr = oracle.project(g, cam.as_array())
    pix = oracle.all_pixels(48, 48)
    K = 8
    rr = oracle.render_rule(pr, f, oracle.RULE_RIEMANN, K, pix, T_min=0.0)
    ref = oracle.render(pr, f, K, pix, T_min=0.0)
    np.testing.assert_array_equal(rr.ids, ref.ids)
    np.testing.assert_array_equal(rr.cnt, ref.cnt)
    assert (rr.cnt > 0).sum() > 200
    for p in np.nonzero(rr.cnt > 0)[0]:
        c = rr.cnt[p]
        ws = rr.wq[p, :c]
        assert abs(ws.sum() - 1.0) <= 1e-12
        # some total D <= K of crossed boundaries makes every weight a whole count >= 1
        ok = [D for D in range(1, K + 1)
              if np.allclose(ws * D, np.round(ws * D), atol=1e-9) and (np.round(ws * D) >= 1).all()]
        assert ok, ws
        np.testing.assert_allclose(rr.out[p], ws @ f[rr.ids[p, :c]].astype(np.float64),
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("K", [1, 2, 4, 8, 16, 32])
def test_riemann_within_app_c_error_bound(K):
    """App. C's theorem for the right-Riemann reading: with c(u) the feature
    of the Gaussian covering transmittance u and |c'| <= M, one sample per
    segment of width 1/(K+1), normalised by the width covered, lies within
    M / (2 (K + 1)) of the mean of c over that width.  A list of many small
    steps (each at most delta) carrying features g(u) = (sin 3u, cos 2u, u^2)
    at the step's midpoint makes c a step approximation of g, so the oracle's
    Riemann estimate must be within M / (2 (K + 1)) + M delta of the exact
    mean of g over [u_D, 1] (closed-form antiderivatives), u_D the last
    boundary crossed."""
    n = 4000
    T = np.concatenate([[1.0], 1.0 - (1.0 - 1e-3) * np.arange(1, n + 1) / n])
    a = 1.0 - T[1:] / T[:-1]
    mid = 0.5 * (T[1:] + T[:-1])
    g = np.stack([np.sin(3 * mid), np.cos(2 * mid), mid ** 2], 1)
    M = np.array([3.0, 2.0, 2.0])
    delta = (1.0 - 1e-3) / n
    sel, w, _ = oracle.riemann_list(a, K)
    D = w.sum()
    assert D == K                       # the walk ends below 1/(K+1) > 1e-3
    R = (w[:, None] * g).sum(0) / D
    lo = 1.0 - D / (K + 1)
    G = lambda u: np.stack([-np.cos(3 * u) / 3, np.sin(2 * u) / 2, u ** 3 / 3], -1)
    mean = (G(1.0) - G(lo)) / (1.0 - lo)
    err = np.abs(R - mean)
    assert (err <= M / (2 * (K + 1)) + M * delta + 1e-12).all(), (K, err)
    # the bound is met with the sample at each segment's crossing, not with a
    # sample one segment late (a misplaced crossing count breaks it at K >= 4)
    if K >= 4:
        idx = np.nonzero(sel)[0]
        late = g[np.minimum(idx + int(1.0 / ((K + 1) * delta)), n - 1)]
        R_late = (w[idx, None] * late).sum(0) / D
        assert (np.abs(R_late - mean) > M / (2 * (K + 1)) * 0.5).any()
