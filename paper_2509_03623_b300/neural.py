"""The neural field in FP32 on the GPU, for comparison with the tensor-core BF16 path.

The network (Fourier features, Linear layers, SiLU) is built from torch operations, i.e.
plain cuBLAS FP32 GEMMs with TF32 disabled; its outputs drive the library's march through
rt_sample_coords / rt_render_modulated. The product path is rt_render_mlp.
"""

from __future__ import annotations

import math

from . import _rt


def mlp_fp32(net, xy):
    """Network outputs [..., 4] for inputs xy [..., 2] in FP32 (no TF32)."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        shp = xy.shape[:-1]
        x = xy.reshape(-1, 2)
        ph = x @ net.B.T
        ph = ph - torch.round(ph)
        h = torch.cat([torch.sin(2 * math.pi * ph), torch.cos(2 * math.pi * ph)], 1)
        for l, (W, b) in enumerate(zip(net.W, net.b)):
            h = torch.addmm(b, h, W.T)
            if l < len(net.W) - 1:
                h = torch.nn.functional.silu(h)
        return h.reshape(*shp, -1)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def render_mlp_fp32(problem, fields, net, out=None, stream=None):
    """Forward render with the FP32 network (comparison path)."""
    xy = _rt.rt_sample_coords(problem, fields, stream=stream)
    mod = mlp_fp32(net, xy)
    return _rt.rt_render_modulated(problem, fields, mod, net.h_scale, out=out, stream=stream)
