"""Differentiable rendering: torch.autograd.Functions over the C ABI.

RenderFn: forward  -> rt_render (FP32 march)
          backward -> rt_render_adjoint seeded with the incoming cube gradient (fused reverse
                      march, FP64 gradient accumulation, cast to the dtype of the inputs)
FieldChainFn: forward  -> rt_field_chain (T -> n_H2, h_lo, h_hi)
              backward -> rt_field_chain_adjoint
PressureVphiFn: forward  -> rt_pressure_vphi (n_H2, T -> v_phi)
                backward -> rt_pressure_vphi_adjoint
Render3Fn: forward  -> rt_render3d / rt_render_sph (3-D Cartesian or spherical grid)
           backward -> rt_render3d_adjoint / rt_render_sph_adjoint
so that with n, h_lo, h_hi = field_chain(problem, chain, T), vphi = pressure_vphi(problem, n, T)
and cube = render(problem, T, n, vt, h_lo, h_hi, vphi) a loss differentiates with respect to T
through the march, the rotation and the chain.
"""

from __future__ import annotations

import torch

from . import _rt


class _Fields:
    def __init__(self, T, n, vt, hlo, hhi, vphi=None):
        self.T, self.n_h2, self.vturb, self.h_lo, self.h_hi = T, n, vt, hlo, hhi
        self.vphi = vphi

    def tensors(self):
        return self.T, self.n_h2, self.vturb, self.h_lo, self.h_hi


class RenderFn(torch.autograd.Function):
    """cube = render(T, n_H2, v_turb, h_lo, h_hi[, v_phi]) for a fixed problem geometry/view/
    line (v_phi: an optional rotation field, Keplerian rotation when None)."""

    @staticmethod
    def forward(ctx, T, n, vt, hlo, hhi, vphi, problem):
        ins = (T, n, vt, hlo, hhi) + ((vphi,) if vphi is not None else ())
        ts = [x.detach().contiguous().float() for x in ins]
        ctx.save_for_backward(*ts)
        ctx.problem = problem
        return _rt.rt_render(problem, _Fields(*ts))

    @staticmethod
    def backward(ctx, grad_cube):
        ts = ctx.saved_tensors
        _, g = _rt.rt_render_adjoint(ctx.problem, _Fields(*ts),
                                     dL_dcube=grad_cube.contiguous().float(), cube_out=None)
        keys = ("T", "n_h2", "vturb", "h_lo", "h_hi", "vphi")[:len(ts)]
        outs = [g[k].to(t.dtype) for k, t in zip(keys, ts)]
        if len(ts) == 5:
            outs.append(None)
        return (*outs, None)


def render(problem, T, n, vt, hlo, hhi, vphi=None):
    """Differentiable forward render (CUDA tensors, float32 fields; vphi an optional rotation
    field)."""
    return RenderFn.apply(T, n, vt, hlo, hhi, vphi, problem)


class FieldChainFn(torch.autograd.Function):
    """(n_H2, h_lo, h_hi) = chain(T) for a fixed grid and chain parameters."""

    @staticmethod
    def forward(ctx, T, problem, chain):
        Tf = T.detach().contiguous().float()
        ctx.save_for_backward(Tf)
        ctx.problem, ctx.chain, ctx.dtype = problem, chain, T.dtype
        out = _rt.rt_field_chain(problem, Tf, chain, column=False)
        return out["n_h2"], out["h_lo"], out["h_hi"]

    @staticmethod
    def backward(ctx, g_n, g_lo, g_hi):
        (Tf,) = ctx.saved_tensors
        as64 = lambda g: g.contiguous().double() if g is not None else None
        gT = _rt.rt_field_chain_adjoint(ctx.problem, Tf, ctx.chain, as64(g_n), as64(g_lo),
                                        as64(g_hi))
        return gT.to(ctx.dtype), None, None


def field_chain(problem, chain, T):
    """Differentiable field chain: (n_H2, h_lo, h_hi) from the temperature grid T (CUDA)."""
    return FieldChainFn.apply(T, problem, chain)


class PressureVphiFn(torch.autograd.Function):
    """v_phi = rotation(n_H2, T) (pressure-corrected, km/s) for a fixed grid and line."""

    @staticmethod
    def forward(ctx, n, T, problem):
        nf, Tf = n.detach().contiguous().float(), T.detach().contiguous().float()
        ctx.save_for_backward(nf, Tf)
        ctx.problem, ctx.dtypes = problem, (n.dtype, T.dtype)
        return _rt.rt_pressure_vphi(problem, nf, Tf)

    @staticmethod
    def backward(ctx, g_v):
        nf, Tf = ctx.saved_tensors
        gn, gT = _rt.rt_pressure_vphi_adjoint(ctx.problem, nf, Tf, g_v.contiguous().double())
        return gn.to(ctx.dtypes[0]), gT.to(ctx.dtypes[1]), None


def pressure_vphi(problem, n, T):
    """Differentiable pressure-corrected rotation [nz][nr] km/s from n_H2 and T (CUDA)."""
    return PressureVphiFn.apply(n, T, problem)


class _Grid3Fields:
    def __init__(self, keys, ts):
        for k, t in zip(keys, ts):
            setattr(self, k, t)


class Render3Fn(torch.autograd.Function):
    """cube = render through a 3-D grid of the problem (problem.g3: Cartesian, fields T, n_H2,
    v_turb, X_CO, v_x, v_y, v_z; problem.gs: spherical, fields T, n_H2, v_turb, X_CO, v_r,
    v_theta, v_phi), for a fixed geometry, view and line: forward rt_render3d / rt_render_sph,
    backward rt_render3d_adjoint / rt_render_sph_adjoint seeded with the incoming cube
    gradient."""

    @staticmethod
    def forward(ctx, problem, *fields):
        ts = [x.detach().contiguous().float() for x in fields]
        ctx.save_for_backward(*ts)
        ctx.problem = problem
        if getattr(problem, "gs", None) is not None:
            return _rt.rt_render_sph(problem, _Grid3Fields(_rt.DeviceGridSph.FIELDS, ts))
        return _rt.rt_render3d(problem, _Grid3Fields(_rt.DeviceGrid3.FIELDS, ts))

    @staticmethod
    def backward(ctx, grad_cube):
        ts = ctx.saved_tensors
        sph = getattr(ctx.problem, "gs", None) is not None
        keys = _rt.DeviceGridSph.FIELDS if sph else _rt.DeviceGrid3.FIELDS
        adjoint = _rt.rt_render_sph_adjoint if sph else _rt.rt_render3d_adjoint
        _, g = adjoint(ctx.problem, _Grid3Fields(keys, ts),
                       dL_dcube=grad_cube.contiguous().float(), cube_out=None)
        return (None, *[g[k].to(t.dtype) for k, t in zip(keys, ts)])


def render3(problem, *fields):
    """Differentiable forward render through the problem's 3-D grid: the seven node fields in
    the order of DeviceGrid3.FIELDS (Cartesian) or DeviceGridSph.FIELDS (spherical), CUDA
    float32 tensors in the grid's node order."""
    return Render3Fn.apply(problem, *fields)
