"""SRWCR as a ``torch.autograd.Function``.

forward(c)   runs the fused warp + statistics kernel and the FP64 per-region
             finalisation (value of Eq. 9); it keeps only c and the small
             per-region tables inside the engine, never the warped image.
backward(gD) runs the adjoint kernel, which recomputes the warp from c and
             turns dD/dB (Eq. 19) into dD/dc (Eqs. 16-17), scaled by gD.

The engine holds one set of tables per pyramid level.  If another
evaluation at the same level ran between this forward and its backward, the
backward first re-runs the forward for its own c so the tables match.
"""
from __future__ import annotations

import torch

from . import SRWCR


class SRWCRFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c: torch.Tensor, engine: SRWCR, level: int = 0):
        c = c.detach().contiguous()
        D = torch.empty((), dtype=torch.float64, device=c.device)
        gen = engine.forward(c, D, level)
        ctx.save_for_backward(c)
        ctx.engine, ctx.level, ctx.gen = engine, level, gen
        return D

    @staticmethod
    def backward(ctx, gD: torch.Tensor):
        (c,) = ctx.saved_tensors
        engine, level = ctx.engine, ctx.level
        if engine.generation(level) != ctx.gen:
            scratch = torch.empty((), dtype=torch.float64, device=c.device)
            engine.forward(c, scratch, level)
        g = torch.empty_like(c)
        scale = gD.detach().to(torch.float32).reshape(1).contiguous()
        engine.backward(c, scale, g, level)
        return g, None, None


def srwcr(c: torch.Tensor, engine: SRWCR, level: int = 0) -> torch.Tensor:
    """Differentiable SRWCR value D(c) (float64 scalar tensor)."""
    return SRWCRFunction.apply(c, engine, level)
