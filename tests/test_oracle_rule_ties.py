"""Pins of the near-tie classification of the top-K and Stratified-K rules
(``classify_rule_ties`` in qr_oracle.c), as for Algorithm 1's classifier:
every candidate list is also walked by an FP32 emulation of the kernels'
arithmetic (rules.cu), with alpha*G perturbed inside the error model, the
transmittance and weight products rounded to nearest or by a directed-rounding
adversary, and -- for Stratified-K -- the normal CDF and its inverse off by up
to 5 units in the last place (the documented accuracy of CUDA's normcdff and
normcdfinvf).  Wherever the FP32 walk keeps another sequence of Gaussians than
the FP64 oracle, the classifier must have flagged the list (RULE_TIE_BITS);
lists far from every threshold are rarely flagged.
"""
import numpy as np
import pytest

import oracle
from oracle import compare

sp = pytest.importorskip("scipy.special")

U = 2.0 ** -24
AMIN = oracle.ALPHA_MIN_F32
AMAX = oracle.ALPHA_MAX_F32
f32 = np.float32
BITS = compare.RULE_TIE_BITS


def _rel(qabs):
    return oracle.DEFAULT_TIE_EPS * (1.0 + qabs) + 4.0 * U


def _rnd(x, mode):
    """FP32 of an exact FP64 value: nearest (mode 0) or one ulp up / down."""
    r = f32(x)
    if mode > 0 and float(r) < x:
        r = np.nextafter(r, f32(np.inf))
    elif mode < 0 and float(r) > x:
        r = np.nextafter(r, f32(-np.inf))
    return r


def _ulps(x, k):
    x = f32(x)
    return f32(float(x) + k * float(np.spacing(x)))


def _members(depth, ids, g, delta):
    order = np.lexsort((ids, depth.astype(f32)))
    a = [min(f32(AMAX), f32(g[i] * (1.0 + delta[i]))) for i in order]
    return [(int(ids[i]), a_) for i, a_ in zip(order, a) if a_ >= f32(AMIN)]


def fp32_topk(depth, ids, g, K, T_min, delta, mode):
    T = f32(1.0)
    kept = []                          # (weight, position, id)
    for pos, (gid, a) in enumerate(_members(depth, ids, g, delta)):
        Tt = _rnd(float(T) * float(_rnd(1.0 - float(a), mode)), mode)
        if T_min > 0 and Tt < f32(T_min):
            break
        w = _rnd(float(T) * float(a), mode)
        T = Tt
        if len(kept) < K:
            kept.append((w, pos, gid))
        else:
            s = min(range(K), key=lambda j: (kept[j][0], -kept[j][1]))
            if w > kept[s][0]:
                kept[s] = (w, pos, gid)
    return tuple(gid for _, _, gid in sorted(kept, key=lambda e: e[1]))


def fp32_stratified(depth, ids, g, K, T_min, delta, mode, rng):
    mem = _members(depth, ids, g, delta)
    T = f32(1.0)
    Ts = []
    for gid, a in mem:
        Tt = _rnd(float(T) * float(_rnd(1.0 - float(a), mode)), mode)
        if T_min > 0 and Tt < f32(T_min):
            break
        T = Tt
        Ts.append(float(T))
    n = len(Ts)
    if n >= 2:
        S1, S2 = sum(Ts), sum(t * t for t in Ts)
        mu64 = S1 / n
        mu = f32(mu64)
        sigma = f32(np.sqrt(max(S2 / n - mu64 * mu64, 0.0)))
        zlo = f32(-float(mu) / float(sigma))
        zhi = f32(float(f32(1.0 - float(mu))) / float(sigma))
        e = rng.integers(-5, 6, size=K + 2)
        ulo = _ulps(sp.ndtr(float(zlo)), e[0])
        uhi = _ulps(sp.ndtr(float(zhi)), e[1])
        d = f32(float(uhi) - float(ulo))
        tau = []
        for k in range(1, K + 1):
            c = f32(float(K + 1 - k) / float(K + 1))
            uk = f32(float(d) * float(c) + float(ulo))
            zk = _ulps(sp.ndtri(float(uk)), e[1 + k])
            tau.append(f32(float(sigma) * float(zk) + float(mu)))
    else:
        tau = [f32(float(K + 1 - k) / float(K + 1)) for k in range(1, K + 1)]
    T, TQ, k = f32(1.0), f32(1.0), 0
    kept = []
    for gid, a in mem:
        Tt = _rnd(float(T) * float(_rnd(1.0 - float(a), mode)), mode)
        if k < K and Tt < tau[k]:
            kept.append(gid)
            k += 1
            while k < K and Tt < tau[k]:
                k += 1
        if Tt < tau[K - 1]:
            break
        T = Tt
    return tuple(kept)


def random_list(rng, n):
    depth = np.sort(rng.uniform(1.0, 5.0, n))
    for i in range(1, n):
        if rng.random() < 0.08:
            depth[i] = depth[i - 1] * (1.0 + rng.choice([0.0, 1.0, 3.0, 1e3]) * U)
    ids = rng.permutation(n * 3)[:n].astype(np.int64)
    g = np.exp(rng.uniform(np.log(2e-3), np.log(0.7), n))
    kind = rng.random(n)
    g[kind < 0.1] = AMAX * (1.0 + rng.uniform(-1, 1, (kind < 0.1).sum()) * 1e-6)
    nm = (kind >= 0.1) & (kind < 0.18)
    g[nm] = AMIN * (1.0 + rng.uniform(-1, 1, nm.sum()) * 10.0 ** rng.uniform(-7.5, -3, nm.sum()))
    qabs = np.exp(rng.uniform(np.log(1e-3), np.log(30.0), n))
    return depth, ids, g, qabs


def topk_tie_list(rng, K, eps):
    """Members whose (K+1)-th largest weight equals the K-th times (1 + eps)."""
    n = int(rng.integers(K + 2, K + 12))
    a = np.exp(rng.uniform(np.log(0.01), np.log(0.2), n))
    T = np.concatenate([[1.0], np.cumprod(1.0 - a)])
    w = T[:-1] * a
    order = np.argsort(-w, kind="stable")
    i, j = int(order[K - 1]), int(order[K])      # K-th and (K+1)-th
    a[j] = w[i] * (1.0 + eps) / T[j]
    if not (AMIN * 1.01 < a[j] < 0.9):
        return None
    return (np.arange(1, n + 1, dtype=np.float64), np.arange(n, dtype=np.int64), a,
            np.zeros(n))


def stratified_tie_list(rng, K, eps, T_min):
    """Members whose pass-2 test transmittance at one entry sits at a
    boundary tau_k times (1 + eps) (fixed point: moving the entry moves tau)."""
    n = int(rng.integers(3, 30))
    a = np.exp(rng.uniform(np.log(0.02), np.log(0.3), n))
    depth, ids, q = np.arange(1, n + 1, dtype=np.float64), np.arange(n, dtype=np.int64), np.zeros(n)
    sel, w, tq, nproc, tau, _ = oracle.stratified_list(a, K, T_min)
    if nproc < 1:
        return None
    i = int(rng.integers(0, nproc))
    k = int(rng.integers(0, K))
    for _ in range(6):
        Tprev = float(np.prod(1.0 - a[:i]))
        ai = 1.0 - tau[k] * (1.0 + eps) / Tprev
        if not (AMIN * 1.01 < ai < 0.9):
            return None
        a[i] = ai
        _, _, _, _, tau, _ = oracle.stratified_list(a, K, T_min)
    return depth, ids, a, q


@pytest.mark.parametrize("K", [1, 2, 4, 8, 16])
def test_topk_classifier_is_sound(K):
    rng = np.random.default_rng(300 + K)
    cases = [random_list(rng, int(rng.integers(1, 40))) for _ in range(250)]
    for eps in np.concatenate([-np.logspace(-8, -3, 11), np.logspace(-8, -3, 11)]):
        for _ in range(4):
            c = topk_tie_list(rng, K, eps)
            if c is not None:
                cases.append(c)
    flips = 0
    for depth, ids, g, qabs in cases:
        T_min = float(f32(1e-4)) if rng.random() < 0.5 else 0.0
        flags, kept64, _ = oracle.classify_rule_candidates(depth, ids, g, qabs, oracle.RULE_TOPK,
                                                           K, T_min=T_min, alpha_min=AMIN,
                                                           alpha_max=AMAX)
        rel = _rel(qabs)
        draws = [np.zeros_like(g), rel, -rel] + [rng.uniform(-1, 1, g.size) * rel
                                                 for _ in range(6)]
        changed = any(fp32_topk(depth, ids, g, K, T_min, d, mode) != tuple(kept64)
                      for d in draws for mode in (0, 1, -1))
        flips += changed
        if changed:
            assert flags & BITS, (K, flags, depth, ids, g, qabs)
    assert flips > 0


@pytest.mark.parametrize("K", [1, 4, 8, 16])
def test_stratified_classifier_is_sound(K):
    rng = np.random.default_rng(400 + K)
    T_min = float(f32(1e-4))
    cases = [random_list(rng, int(rng.integers(1, 40))) for _ in range(150)]
    for eps in np.concatenate([-np.logspace(-8, -3, 11), np.logspace(-8, -3, 11)]):
        for _ in range(3):
            c = stratified_tie_list(rng, K, eps, T_min)
            if c is not None:
                cases.append(c)
    flips = 0
    for depth, ids, g, qabs in cases:
        flags, kept64, _ = oracle.classify_rule_candidates(depth, ids, g, qabs,
                                                           oracle.RULE_STRATIFIED, K, T_min=T_min,
                                                           alpha_min=AMIN, alpha_max=AMAX)
        rel = _rel(qabs)
        draws = [np.zeros_like(g), rel, -rel] + [rng.uniform(-1, 1, g.size) * rel
                                                 for _ in range(3)]
        changed = any(fp32_stratified(depth, ids, g, K, T_min, d, mode, rng) != tuple(kept64)
                      for d in draws for mode in (0, 1, -1))
        flips += changed
        if changed:
            assert flags & BITS, (K, flags, depth, ids, g, qabs)
    assert flips > 0


@pytest.mark.parametrize("rule", [oracle.RULE_TOPK, oracle.RULE_STRATIFIED])
def test_rule_classifier_leaves_most_clean_lists_alone(rule):
    """Lists with distinct depths and alpha*G far from alpha_min and
    alpha_max: only a small fraction can sit within the FP32 error of a
    ranking or boundary decision."""
    rng = np.random.default_rng(500 + rule)
    flagged = total = 0
    for _ in range(400):
        n = int(rng.integers(1, 40))
        depth = np.sort(rng.uniform(1.0, 5.0, n)) + np.arange(n) * 1e-3
        ids = np.arange(n, dtype=np.int64)
        g = np.exp(rng.uniform(np.log(0.01), np.log(0.6), n))
        flags, _, _ = oracle.classify_rule_candidates(depth, ids, g, np.full(n, 1.0), rule, 8,
                                                      T_min=float(f32(1e-4)), alpha_min=AMIN,
                                                      alpha_max=AMAX)
        total += 1
        flagged += bool(flags & BITS)
    assert flagged <= 0.02 * total, (flagged, total)
