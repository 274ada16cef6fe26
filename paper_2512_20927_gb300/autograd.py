"""torch.autograd.Function over the C ABI: Q-Render forward (qr_render steps)
and its hand-written backward (qr_backward).  Marshalling only; no PyTorch
math on the rendering path."""
from __future__ import annotations

import torch

from . import qrender as q


class QuantileRenderFunction(torch.autograd.Function):
    """out[H, W, C] = Q-Render of the Gaussians' features.

    Differentiable in `features` and `opacity` (activated).  Means, scales and
    rotations only move the selection and the projection; their gradients are
    not part of this operator (the paper's network predicts the features)."""

    @staticmethod
    def forward(ctx, mean, log_scale, quat, opacity, features, feat_scale, camera, params,
                max_isect):
        feat = features if feat_scale is None else (features, feat_scale)
        res = q.render_frame((mean, log_scale, quat, opacity), feat, camera, K=params.K,
                             params=params, max_isect=max_isect)
        ctx.frame = res["frame"]
        ctx.save_for_backward(features, feat_scale, res["ids"], res["weights"], res["counts"])
        ctx.mark_non_differentiable(res["ids"], res["counts"])
        fr = res["frame"]
        return res["out"].view(fr.height, fr.width, features.shape[1]), res["counts"]

    @staticmethod
    def backward(ctx, grad_out, grad_counts):
        features, feat_scale, ids, weights, counts = ctx.saved_tensors
        P = ids.shape[0]
        g = grad_out.reshape(P, -1).float().contiguous()
        gf, ga, _ = q.qr_backward(ctx.frame, features, feat_scale, ids, weights, counts, g,
                                  want_conic=False)
        gfeat = gf.to(features.dtype) if ctx.needs_input_grad[4] else None
        gop = ga if ctx.needs_input_grad[3] else None
        return None, None, None, gop, gfeat, None, None, None, None


def quantile_render(mean, log_scale, quat, opacity, features, camera, K=8, feat_scale=None,
                    params=None, max_isect=None):
    """Differentiable Q-Render of one view: returns (map [H, W, C] float32, counts [P])."""
    params = params or q.default_params(K)
    return QuantileRenderFunction.apply(mean, log_scale, quat, opacity, features, feat_scale,
                                        camera, params, max_isect)
