"""Pins of the oracle's near-tie classifier (``classify_ties`` in qr_oracle.c).

The GPU evaluates alpha' and the transmittance products in FP32; the FP64
oracle flags a pixel as a near tie where a decision of Algorithm 1 (Sec. 4.2)
or of the dense Eq. 1 walk is closer to its threshold than that FP32 error
can reach, and the parity tests excuse exactly the flagged pixels from the
exact-id check.  The classifier is pinned here against an FP32 emulation of
the GPU's arithmetic written independently in numpy:

  (i)   soundness: every candidate list is walked in FP32 with each alpha*G
        perturbed by a relative error inside the model's bound
        (tie_eps (1 + qabs) + 4u); wherever the FP32 walk keeps another
        sequence of Gaussians than the FP64 walk, the classifier must have
        flagged the list;
  (ii)  tightness: lists whose every margin (test transmittance to each
        boundary, alpha*G to alpha_min, depth gaps, T to T_min) is at least
        ten times the model's bound are never flagged;
  (iii) hand-built lists with a decision at (1 +- eps) of its threshold are
        flagged for small eps and not for large eps, for each check, and only
        up to the entry where the walk stops.

Beside round-to-nearest, the transmittance products are also taken with every
operation rounded up (or down) by up to one ulp, an adversary that bounds the
accumulated rounding of any walk.  The FP32 emulation follows the kernels'
arithmetic: alpha' =
min(alpha_max, fl32(alpha*G)), membership alpha' >= alpha_min, T_test =
fl32(T * fl32(1 - alpha')), boundaries fl32((K-k)/(K+1)), stop below
fl32(1/(K+1)), list order by (FP32 depth, id), non-members leaving T unchanged.
"""
import numpy as np
import pytest

import oracle

U = 2.0 ** -24
AMIN = oracle.ALPHA_MIN_F32
AMAX = oracle.ALPHA_MAX_F32
TIE_EPS = oracle.DEFAULT_TIE_EPS
f32 = np.float32


def _rel(qabs):
    return TIE_EPS * (1.0 + qabs) + 4.0 * U


# --------------------------------------------------------------------------- definitions
def fp64_walks(depth, ids, g, K, T_min):
    """Kept ids of Algorithm 1 and blended ids of the dense walk, in FP64."""
    a = np.minimum(AMAX, g)
    mem = a >= AMIN
    order = np.lexsort((ids[mem], depth[mem]))
    al, il = a[mem][order], ids[mem][order]
    T, k, kept = 1.0, 0, []
    for i in range(len(al)):
        Tt = T * (1.0 - al[i])
        if Tt < 1.0 - (k + 1) / (K + 1):
            kept.append(int(il[i]))
            k += 1
            while Tt < 1.0 - (k + 1) / (K + 1):
                k += 1
        if Tt < 1.0 / (K + 1):
            break
        T = Tt
    T, blended = 1.0, []
    for i in range(len(al)):
        Tt = T * (1.0 - al[i])
        if T_min > 0.0 and Tt < T_min:
            break
        blended.append(int(il[i]))
        T = Tt
    return tuple(kept), tuple(blended)


def _round(x64, mode):
    """FP32 value of an exact FP64 result: round to nearest (the GPU), or
    always up / always down -- an adversary whose every operation is off by
    up to one ulp, which bounds any sequence of round-to-nearest errors."""
    r = x64.astype(f32)
    if mode == 0:
        return r
    if mode > 0:
        return np.where(r.astype(np.float64) < x64, np.nextafter(r, f32(np.inf)), r)
    return np.where(r.astype(np.float64) > x64, np.nextafter(r, f32(-np.inf)), r)


def fp32_walks(depth, ids, g, K, T_min, delta, mode=0):
    """The same walks as the GPU takes them, for R perturbations at once.

    delta [R, n]: relative errors of alpha*G; mode: rounding of the
    transmittance products (0 nearest, +1 up, -1 down).  Returns lists of R
    tuples."""
    R, n = delta.shape
    order = np.lexsort((ids, depth.astype(f32)))
    gp = (g[None, :] * (1.0 + delta))[:, order].astype(f32)
    a = np.minimum(f32(AMAX), gp)
    mem = a >= f32(AMIN)
    a = np.where(mem, a, f32(0.0))            # a non-member leaves T exactly unchanged
    il = ids[order]
    one = f32(1.0)
    thr_tab = np.array([f32(K - k) / f32(K + 1) for k in range(K)] + [-1.0], f32)
    stop = f32(1.0) / f32(K + 1)
    T = np.ones(R, f32)
    k = np.zeros(R, np.int64)
    done = np.zeros(R, bool)
    kept = np.zeros((R, n), bool)
    def mul(Tv, ai):        # fl32(T * fl32(1 - a)); both FP64 steps are exact
        om = _round(1.0 - ai.astype(np.float64), mode)
        return _round(Tv.astype(np.float64) * om.astype(np.float64), mode)
    for i in range(n):
        Tt = mul(T, a[:, i])
        live = ~done & mem[:, i]
        ev = live & (Tt < thr_tab[k])
        kept[:, i] = ev
        for _ in range(K + 1):                 # advance k past every boundary above T_test
            adv = ev & (Tt < thr_tab[k])
            if not adv.any():
                break
            k = np.where(adv, k + 1, k)
        done = done | (live & (Tt < stop))
        T = np.where(live & ~(Tt < stop), Tt, T)
    Td = np.ones(R, f32)
    dd = np.zeros(R, bool)
    blend = np.zeros((R, n), bool)
    tmin = f32(T_min)
    for i in range(n):
        Tt = mul(Td, a[:, i])
        live = ~dd & mem[:, i]
        brk = live & (T_min > 0.0) & (Tt < tmin)
        dd = dd | brk
        use = live & ~brk
        blend[:, i] = use
        Td = np.where(use, Tt, Td)
    return ([tuple(int(x) for x in il[kept[r]]) for r in range(R)],
            [tuple(int(x) for x in il[blend[r]]) for r in range(R)])


def perturbations(rng, qabs, R):
    rel = _rel(qabs)[None, :]
    d = rng.uniform(-1.0, 1.0, size=(R, qabs.size)) * rel
    d[0] = rel[0]                    # the extremes of the model
    d[1] = -rel[0]
    d[2] = 0.0
    return d


# --------------------------------------------------------------------------- list generators
def random_list(rng, n):
    depth = np.sort(rng.uniform(1.0, 5.0, n))
    # some neighbours at (nearly) the same depth
    for i in range(1, n):
        if rng.random() < 0.1:
            depth[i] = depth[i - 1] * (1.0 + rng.choice([0.0, 1.0, 3.0, 10.0, 1e3]) * U)
    ids = rng.permutation(n * 3)[:n].astype(np.int64)
    kind = rng.random(n)
    g = np.exp(rng.uniform(np.log(2e-3), np.log(0.6), n))
    near_clamp = kind < 0.15
    g[near_clamp] = AMAX * (1.0 + rng.uniform(-1, 1, near_clamp.sum()) *
                            10.0 ** rng.uniform(-7.5, -1.5, near_clamp.sum()))
    near_min = (kind >= 0.15) & (kind < 0.25)
    g[near_min] = AMIN * (1.0 + rng.uniform(-1, 1, near_min.sum()) *
                          10.0 ** rng.uniform(-7.5, -2.0, near_min.sum()))
    qabs = np.exp(rng.uniform(np.log(1e-3), np.log(50.0), n))
    return depth, ids, g, qabs


def boundary_list(rng, K, eps):
    """Random members whose test transmittance at a random step sits at
    tau_k (1 + eps) for a boundary tau_k = (K-k)/(K+1) it reaches."""
    n = int(rng.integers(2, 12))
    a = np.exp(rng.uniform(np.log(0.01), np.log(0.3), n))
    T = np.cumprod(1.0 - a)
    i = int(rng.integers(0, n))
    Tprev = 1.0 if i == 0 else T[i - 1]
    taus = [(K - k) / (K + 1) for k in range(K + 1)][:K]
    below = [t for t in taus if t < Tprev * 0.999]
    if not below:
        return None
    tau = below[0] if rng.random() < 0.6 else below[int(rng.integers(0, len(below)))]
    ai = 1.0 - tau * (1.0 + eps) / Tprev
    if not (AMIN * 1.01 < ai < 0.95):
        return None
    a[i] = ai
    depth = np.arange(1, n + 1, dtype=np.float64)
    ids = np.arange(n, dtype=np.int64)
    return depth, ids, a.copy(), np.zeros(n)


def small_alpha_list(rng, K, eps):
    """A long list of small alpha' values, where the FP32 roundings of the
    transmittance products (not the alpha' errors) decide: the test
    transmittance at its last entry sits at the stop boundary 1/(K+1) times
    (1 + eps)."""
    n = int(rng.integers(100, 400))
    a = rng.uniform(0.004, 0.012, n)
    T = np.cumprod(1.0 - a)
    tau = 1.0 / (K + 1)
    j = int(np.argmax(T < tau))
    if T[j] >= tau or j == 0:
        return None
    a[j] = 1.0 - tau * (1.0 + eps) / T[j - 1]
    if not (AMIN * 1.01 < a[j] < 0.95):
        return None
    n = min(j + 3, n)
    return (np.arange(1, n + 1, dtype=np.float64), np.arange(n, dtype=np.int64), a[:n].copy(),
            np.zeros(n))


def clamp_list(rng):
    """Two members at the alpha_max clamp whose product lands near T_min: the
    second one's alpha*G sits within a few error bounds of alpha_max, so the
    FP32 clamp may fall either way (Eq. 1's alpha' = min(alpha_max, alpha G)).
    Returns the list and the T_min that puts the decision at (1 + eps)."""
    qabs = np.array([0.0, float(np.exp(rng.uniform(np.log(1.0), np.log(400.0))))])
    rel = _rel(qabs[1])
    g = np.array([2.0, AMAX * (1.0 + rng.uniform(-3.0, 3.0) * rel)])
    T2 = (1.0 - AMAX) * (1.0 - min(AMAX, g[1]))
    T_min = T2 * (1.0 + rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-7.0, -1.5))
    return (np.array([1.0, 2.0]), np.array([0, 1], np.int64), g, qabs), T_min


# --------------------------------------------------------------------------- (i) soundness
@pytest.mark.parametrize("K", [1, 4, 8, 16, 32])
def test_classifier_flags_every_list_the_fp32_walk_can_change(K):
    rng = np.random.default_rng(100 + K)
    checked = flips = 0
    cases = []
    for _ in range(400):
        cases.append(random_list(rng, int(rng.integers(1, 40))))
    for eps in np.concatenate([-np.logspace(-9, -4, 11), np.logspace(-9, -4, 11)]):
        for _ in range(12):
            c = boundary_list(rng, K, eps)
            if c is not None:
                cases.append(c)
    for eps in np.concatenate([-np.logspace(-7.5, -4, 14), np.logspace(-7.5, -4, 14)]):
        for _ in range(4):
            c = small_alpha_list(rng, K, eps)
            if c is not None:
                cases.append(c)
    cases = [(c, None) for c in cases]
    for _ in range(200):
        c, tm = clamp_list(rng)
        cases.append((c, float(f32(tm))))
    for (depth, ids, g, qabs), T_min in cases:
        if T_min is None:
            T_min = float(f32(1e-4)) if rng.random() < 0.5 else 0.0
        flags, _, _ = oracle.classify_candidates(depth, ids, g, qabs, K, T_min=T_min,
                                                 alpha_min=AMIN, alpha_max=AMAX)
        kept64, blend64 = fp64_walks(depth, ids, g, K, T_min)
        kept32, blend32 = fp32_walks(depth, ids, g, K, T_min, perturbations(rng, qabs, 24))
        for mode in (1, -1):
            k2, b2 = fp32_walks(depth, ids, g, K, T_min, perturbations(rng, qabs, 6), mode)
            kept32 += k2
            blend32 += b2
        checked += 1
        q_flip = any(k != kept64 for k in kept32)
        d_flip = any(b != blend64 for b in blend32)
        flips += q_flip
        if q_flip:
            assert flags & (1 | 2 | 4), (K, flags, depth, ids, g, qabs)
        if d_flip:
            assert flags & (8 | 64 | 128), (K, flags, depth, ids, g, qabs)
    # the generators do reach the thresholds: some lists change under FP32
    assert flips > 0 and checked > 300


# --------------------------------------------------------------------------- (ii) tightness
def _margins_ok(depth, ids, g, qabs, K, T_min, factor=10.0):
    """Every margin of the list at least `factor` times the model's bound,
    recomputed here from the stated model (not from the classifier)."""
    rel = _rel(qabs)
    pos = g > 0
    if (np.abs(np.log(g[pos] / AMIN)) <= factor * 4.0 * rel[pos]).any():
        return False
    a = np.minimum(AMAX, g)
    mem = a >= AMIN
    order = np.lexsort((ids[mem], depth[mem]))
    al, zl, rl, gl = a[mem][order], depth[mem][order], rel[mem][order], g[mem][order]
    if len(zl) > 1 and (np.abs(np.diff(zl)) <= factor * 4.0 * U * np.abs(zl[:-1])).any():
        return False
    T, E = 1.0, 0.0
    taus = np.array([1.0 - (j + 1) / (K + 1) for j in range(K)])
    for i in range(len(al)):
        ea = 0.0 if gl[i] >= AMAX * (1.0 + 2.0 * rl[i]) else rl[i] * al[i] / (1.0 - al[i])
        E += ea + 2.0 * U
        Tt = T * (1.0 - al[i])
        bound = (2.0 * E + 2.0 * U)
        if (np.abs(Tt - taus) <= factor * bound * taus).any():
            return False
        if T_min > 0 and abs(Tt - T_min) <= factor * bound * T_min:
            return False
        T = Tt
    return True


@pytest.mark.parametrize("K", [1, 4, 8, 16, 32])
def test_classifier_leaves_well_separated_lists_alone(K):
    rng = np.random.default_rng(200 + K)
    tested = 0
    for _ in range(600):
        n = int(rng.integers(1, 40))
        depth = np.sort(rng.uniform(1.0, 5.0, n))
        ids = rng.permutation(n).astype(np.int64)
        g = np.exp(rng.uniform(np.log(2e-3), np.log(1.5), n))
        qabs = np.exp(rng.uniform(np.log(1e-3), np.log(50.0), n))
        T_min = float(f32(1e-4)) if rng.random() < 0.5 else 0.0
        if not _margins_ok(depth, ids, g, qabs, K, T_min):
            continue
        tested += 1
        flags, _, _ = oracle.classify_candidates(depth, ids, g, qabs, K, T_min=T_min,
                                                 alpha_min=AMIN, alpha_max=AMAX)
        assert flags == 0, (K, flags, depth, ids, g, qabs)
    assert tested > 300


# --------------------------------------------------------------------------- (iii) hand-built
def _flags(depth, g, K, qabs=None, T_min=0.0, ids=None):
    depth = np.asarray(depth, np.float64)
    g = np.asarray(g, np.float64)
    ids = np.arange(len(depth), dtype=np.int64) if ids is None else np.asarray(ids, np.int64)
    qabs = np.zeros(len(depth)) if qabs is None else np.asarray(qabs, np.float64)
    return oracle.classify_candidates(depth, ids, g, qabs, K, T_min=T_min, alpha_min=AMIN,
                                      alpha_max=AMAX)


@pytest.mark.parametrize("K", [1, 4, 8])
def test_boundary_check_flags_small_margins_only(K):
    # one member whose test transmittance is tau_1 (1 + eps), tau_1 = K / (K + 1)
    # (the stop boundary 1/2 for K = 1), then members that end the walk
    tau = K / (K + 1)
    for eps, want in ((0.0, True), (1e-9, True), (-1e-9, True), (2e-7, True), (-2e-7, True),
                      (1e-4, False), (-1e-4, False), (1e-2, False)):
        a1 = 1.0 - tau * (1.0 + eps)
        flags, nproc, _ = _flags([1.0, 2.0, 3.0], [a1, 0.9, 0.9], K)
        assert bool(flags & 1) == want, (K, eps, flags)
        assert flags & ~1 == 0


def test_boundary_check_stops_at_the_last_visited_entry():
    K = 4
    # T_test after entry 0 is 0.5 (no boundary near), entry 1 takes T far below
    # 1/(K+1) and ends the walk; entry 2's test transmittance would sit on a
    # boundary but is never visited, so it must not flag
    a0 = 0.5
    a1 = 1.0 - 0.1 / 0.5
    tau = 3.0 / 5.0
    # entry 2 puts T_test exactly at a boundary relative to T = 0.1 if it were visited
    a2 = 1.0 - (0.1 * tau) / 0.1
    flags, nproc, _ = _flags([1.0, 2.0, 3.0], [a0, a1, a2], K)
    assert nproc == 2 and flags == 0
    # the same near-tie moved to the stopping entry does flag
    a1_tie = 1.0 - (1.0 / (K + 1)) * (1.0 - 1e-9) / 0.5
    flags, nproc, _ = _flags([1.0, 2.0, 3.0], [a0, a1_tie, a2], K)
    assert nproc == 2 and flags & 1


def test_alpha_min_border_check():
    K = 4
    # a candidate at alpha*G = alpha_min (1 + eps) in front of the stop
    for eps, want in ((0.0, True), (1e-8, True), (-1e-8, True), (1e-3, False), (-1e-3, False)):
        flags, _, _ = _flags([1.0, 2.0, 3.0], [0.3, AMIN * (1.0 + eps), 0.9], K)
        assert bool(flags & 2) == want, (eps, flags)
        assert bool(flags & 64) == want, (eps, flags)    # the dense walk passes it too
    # behind the stopping point it cannot matter to Algorithm 1
    flags, nproc, _ = _flags([1.0, 2.0, 3.0], [0.3, 0.95, AMIN], K)
    assert nproc == 2 and not flags & 2
    # but it does to the dense walk that blends to the end of the list
    assert flags & 64


def test_equal_depth_check():
    K = 4
    for rel, want in ((0.0, True), (U, True), (3 * U, True), (1e-5, False)):
        flags, _, _ = _flags([1.0, 1.0 * (1.0 + rel), 2.0], [0.1, 0.2, 0.9], K)
        assert bool(flags & 4) == want, (rel, flags)
        assert bool(flags & 128) == want, (rel, flags)
    # equal depths behind the stop: only the dense walk can see them
    flags, nproc, _ = _flags([1.0, 2.0, 3.0, 3.0], [0.1, 0.95, 0.2, 0.3], K)
    assert nproc == 2 and not flags & 4 and flags & 128


def test_t_min_check():
    K = 4
    T_min = 1e-2
    # two members: after the first T = 0.5; the second's test transmittance is
    # T_min (1 + eps)
    for eps, want in ((0.0, True), (1e-9, True), (-1e-9, True), (1e-3, False)):
        a1 = 1.0 - T_min * (1.0 + eps) / 0.5
        flags, _, nused = _flags([1.0, 2.0], [0.5, a1], K, T_min=T_min)
        assert bool(flags & 8) == want, (eps, flags)
