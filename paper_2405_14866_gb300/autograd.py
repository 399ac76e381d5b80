"""torch.autograd.Function over the differentiable rasterizer (A3..A8).

Tele-Aloha Sec. 4.2 trains the encoder and decoder through R_G, so the
rasterizer must return gradients for the 2D means, conics, opacities and
features.  Forward = tsplat_rasterize with the backward state saved;
backward = tsplat_backward (transmittance recomputed, not stored per step).
"""
from __future__ import annotations

import torch

from .api import Context


class SplatFn(torch.autograd.Function):
    """F, A = SplatFn.apply(mean2d (N,2), conic (N,3), opac (N,), feat (N,C),
    depth (N,), radius (N,) int32, width, height, params, context).

    `context` (an api.Context) holds the saved state until backward; use one
    context per forward that is still waiting for its backward."""

    @staticmethod
    def forward(ctx, mean2d, conic, opac, feat, depth, radius, width, height, params, context: Context):
        F, A = context.rasterize(mean2d.detach().contiguous(), conic.detach().contiguous(),
                                 opac.detach().contiguous(), depth.detach().contiguous(), radius.contiguous(),
                                 feat.detach().contiguous(), width, height, params, save=True)
        ctx.context = context
        ctx.n, ctx.C = feat.shape
        ctx.hw = (height, width)
        ctx.feat_dtype = feat.dtype
        return F, A

    @staticmethod
    def backward(ctx, dF, dA):
        if dF is None:  # the library reads a whole C x H x W gradient
            dF = torch.zeros((ctx.C, *ctx.hw), device="cuda")
        dm, dc, do, df = ctx.context.backward(dF.contiguous(), None if dA is None else dA.contiguous(),
                                              n=ctx.n, C=ctx.C)
        return dm, dc, do, df.to(ctx.feat_dtype), None, None, None, None, None, None
