"""Differentiable rendering: a torch.autograd.Function over the C ABI.

forward  -> rt_render (FP32 march)
backward -> rt_render_adjoint seeded with the incoming cube gradient (fused reverse march,
            FP64 gradient accumulation, cast to the dtype of the inputs)
"""

from __future__ import annotations

import torch

from . import _rt


class _Fields:
    def __init__(self, T, n, vt, hlo, hhi):
        self.T, self.n_h2, self.vturb, self.h_lo, self.h_hi = T, n, vt, hlo, hhi

    def tensors(self):
        return self.T, self.n_h2, self.vturb, self.h_lo, self.h_hi


class RenderFn(torch.autograd.Function):
    """cube = render(T, n_H2, v_turb, h_lo, h_hi) for a fixed problem geometry/view/line."""

    @staticmethod
    def forward(ctx, T, n, vt, hlo, hhi, problem):
        ts = [x.detach().contiguous().float() for x in (T, n, vt, hlo, hhi)]
        ctx.save_for_backward(*ts)
        ctx.problem = problem
        return _rt.rt_render(problem, _Fields(*ts))

    @staticmethod
    def backward(ctx, grad_cube):
        ts = ctx.saved_tensors
        _, g = _rt.rt_render_adjoint(ctx.problem, _Fields(*ts),
                                     dL_dcube=grad_cube.contiguous().float(), cube_out=None)
        outs = [g[k].to(t.dtype) for k, t in zip(("T", "n_h2", "vturb", "h_lo", "h_hi"), ts)]
        return (*outs, None)


def render(problem, T, n, vt, hlo, hhi):
    """Differentiable forward render (CUDA tensors, float32 fields)."""
    return RenderFn.apply(T, n, vt, hlo, hhi, problem)
