"""Parity metrics between the CUDA path and the FP64 oracle (test infrastructure only).

Feature error of a pixel (a mixed relative metric; component-wise relative
error is ill-posed for mixed-sign features near zero):

    err_p = max_c |F_gpu[p,c] - F_ref[p,c]| / max(sum_j |w_j| max_c |f_j,c|, 1e-30)

where the sum runs over the Gaussians the oracle blended at p.  Selection
parity is exact (integer ids) on every pixel the oracle does not flag as a
near tie; flagged pixels are counted and reported.
"""
from __future__ import annotations

import numpy as np

Q_TIE_BITS = 1 | 2 | 4
DENSE_TIE_BITS = 8 | 16 | 64 | 128
RULE_TIE_BITS = 1 | 2 | 4 | 8        # top-K and Stratified-K (or_render_rule)


def blend(ids, weights, counts, feat) -> np.ndarray:
    """The blend of Algorithm 1 by definition, FP64: out[p] = sum_{j<cnt} w[p,j] f[ids[p,j]]."""
    ids = np.asarray(ids)
    w = np.asarray(weights, np.float64)
    f = np.asarray(feat, np.float64)
    cnt = np.asarray(counts).astype(np.int64)
    K = ids.shape[1]
    mask = np.arange(K)[None, :] < cnt[:, None]
    safe = np.where(mask, ids, 0)
    return np.einsum("pk,pkc->pc", np.where(mask, w, 0.0), f[safe])


def blend_scale(ids, weights, counts, feat) -> np.ndarray:
    ids = np.asarray(ids)
    w = np.abs(np.asarray(weights, np.float64))
    cnt = np.asarray(counts).astype(np.int64)
    rowmax = np.abs(np.asarray(feat, np.float64)).max(axis=1)
    mask = np.arange(ids.shape[1])[None, :] < cnt[:, None]
    return (np.where(mask, w, 0.0) * rowmax[np.where(mask, ids, 0)]).sum(axis=1)


def feature_error(F_gpu, F_ref, scale) -> np.ndarray:
    d = np.abs(np.asarray(F_gpu, np.float64) - np.asarray(F_ref, np.float64)).max(axis=1)
    return d / np.maximum(np.asarray(scale, np.float64), 1e-30)


def selection_report(ids_gpu, w_gpu, cnt_gpu, ref, tie_bits: int = Q_TIE_BITS) -> dict:
    """Compare the per-pixel selections; returns counts and the weight error on matching pixels."""
    ids_gpu = np.asarray(ids_gpu)
    cnt_gpu = np.asarray(cnt_gpu).astype(np.int64)
    tie = (np.asarray(ref.tie) & tie_bits) != 0
    same = (ids_gpu == ref.ids).all(axis=1) & (cnt_gpu == ref.cnt)
    wrel = np.abs(np.asarray(w_gpu, np.float64) - ref.wq)
    wmax = float(wrel[same].max()) if same.any() else 0.0
    return {
        "pixels": int(len(tie)),
        "tie_pixels": int(tie.sum()),
        "mismatch_nontie": int((~same & ~tie).sum()),
        "mismatch_tie": int((~same & tie).sum()),
        "weight_abs_err_max": wmax,
        "same": same,
        "tie": tie,
    }
