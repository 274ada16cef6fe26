"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import compare
from paper_2512_20927_gb300 import scenes


def run_gpu(g, feat, cam, K, dense=True, params_kw=None, max_isect=None, feat_dev=None):
    import torch
    from paper_2512_20927_gb300 import qrender as q
    gdev = q.gaussians_to_device(g)
    if feat_dev is None and feat is not None:
        feat_dev = torch.from_numpy(np.ascontiguousarray(feat, np.float32)).cuda()
    params = q.default_params(K, **(params_kw or {}))
    res = q.render_frame(gdev, feat_dev, cam, K=K, params=params, max_isect=max_isect,
                         dense=dense)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in res.items()
           if k != "frame"}
    out["frame"] = res["frame"]
    return out


def run_oracle(g, feat, cam, K, pixels=None, T_min=1e-4, max_members=0, params_kw=None):
    pk = params_kw or {}
    pr = oracle.project(g, cam.as_array(), dilation=pk.get("dilation", oracle.DEFAULT_DILATION))
    pix = oracle.all_pixels(cam.width, cam.height) if pixels is None else pixels
    ref = oracle.render(pr, feat, K, pix, T_min=float(np.float32(T_min)),
                        alpha_min=oracle.ALPHA_MIN_F32, alpha_max=oracle.ALPHA_MAX_F32,
                        max_members=max_members)
    return pr, pix, ref


def pixel_index(pix, width):
    return pix[:, 1].astype(np.int64) * width + pix[:, 0]


def check_frame(gpu, ref, pix, width, feat, tol_feat, tol_dense=None, max_tie_frac=0.02,
                label=""):
    """Assert selection and feature parity; return a report dict."""
    idx = pixel_index(pix, width)
    rep = compare.selection_report(gpu["ids"][idx], gpu["weights"][idx], gpu["counts"][idx], ref)
    same, tie = rep.pop("same"), rep.pop("tie")
    assert rep["mismatch_nontie"] == 0, (label, rep)
    assert rep["tie_pixels"] <= max_tie_frac * rep["pixels"] + 2, (label, rep)
    if feat is not None and "out" in gpu:
        err = compare.feature_error(gpu["out"][idx], ref.out_q, ref.scale_q)
        rep["feat_err_max"] = float(err[same].max()) if same.any() else 0.0
        rep["feat_err_mean"] = float(err[same].mean()) if same.any() else 0.0
        assert rep["feat_err_max"] <= tol_feat, (label, rep)
        # pixels without any quantile Gaussian render exactly zero
        none = ref.cnt == 0
        assert (gpu["out"][idx][none & same] == 0).all()
    if tol_dense is not None and "dense" in gpu:
        dtie = (ref.tie & compare.DENSE_TIE_BITS) != 0
        derr = compare.feature_error(gpu["dense"][idx], ref.out_dense, ref.scale_dense)
        ok = ~dtie
        rep["dense_tie_pixels"] = int(dtie.sum())
        rep["dense_err_max"] = float(derr[ok].max()) if ok.any() else 0.0
        rep["dense_err_mean"] = float(derr[ok].mean()) if ok.any() else 0.0
        assert rep["dense_err_max"] <= tol_dense, (label, rep)
        tf_err = np.abs(gpu["T_final"][idx] - ref.t_final)[ok]
        rep["t_final_err_max"] = float(tf_err.max()) if ok.any() else 0.0
    return rep


def sample_pixels(width, height, n, seed=0):
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, width, n)
    ys = rng.integers(0, height, n)
    # always include the corners and the ragged last row/column
    extra = np.array([[0, 0], [width - 1, 0], [0, height - 1], [width - 1, height - 1]])
    return np.concatenate([np.stack([xs, ys], 1), extra]).astype(np.int32)


def small_room(n=20000, seed=0, channels=64):
    g, f = scenes.room_scene(seed=seed, n=n, channels=channels)
    return g, f


def check_relevance(got, fmap, qbits, kernel="tma"):
    """Scores of the relevance GEMM against FP64.  Every kernel is within the
    BF16 bound 2^-8 * sum |a b| of the exact product of the FP32 map and the
    BF16 queries.  The TMA kernel reads the map as TF32 (at least 10 mantissa
    bits): within 2^-10 * sum |a b|.  The register-staged kernel rounds the map
    to BF16 like the oracle's encoder: equal to the FP64 product of the
    BF16-rounded map up to FP32 accumulation (1e-4 * sum |a b|)."""
    got = np.asarray(got, np.float64)
    b = oracle.bf16_decode(qbits)
    exact = oracle.relevance(fmap, b)
    mag = np.abs(np.asarray(fmap, np.float64)) @ np.abs(b).T
    err = np.abs(got - exact)
    assert (err <= 2.0 ** -8 * mag + 1e-6).all(), (err / (mag + 1e-30)).max()
    if kernel == "tma":
        assert (err <= 2.0 ** -10 * mag + 1e-6).all(), (err / (mag + 1e-30)).max()
    else:
        a = oracle.bf16_decode(oracle.bf16_encode(fmap))
        ref = oracle.relevance(a, b)
        assert (np.abs(got - ref) <= 1e-4 * mag + 1e-30).all(), np.abs(got - ref).max()
