"""Tensor-core neural-field network (tcgen05, BF16 operands, FP32 accumulation) against the
FP64 oracle network and a torch emulation of the same BF16 roundings."""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.test_forward_gpu import rt  # noqa: F401

pytestmark = pytest.mark.gpu


def bf16_emulation(torch, w, x):
    """Same network with the kernel's roundings: features, weights and hidden activations in
    BF16, products accumulated in FP32, exact SiLU."""
    xt = torch.tensor(x, dtype=torch.float32)
    B = torch.tensor(w.B, dtype=torch.float32)
    ph = xt @ B.T
    ph = ph - torch.round(ph)
    h = torch.cat([torch.sin(2 * np.pi * ph), torch.cos(2 * np.pi * ph)], 1)
    h = h.to(torch.bfloat16).float()
    for l, (W, b) in enumerate(zip(w.W, w.b)):
        Wt = torch.tensor(W).to(torch.bfloat16).float()
        h = h @ Wt.T + torch.tensor(b)
        if l < len(w.W) - 1:
            h = torch.nn.functional.silu(h).to(torch.bfloat16).float()
    return h.numpy()


@pytest.mark.parametrize("n", [1, 127, 128, 5000, 100_003])
def test_mlp_bf16_vs_oracle_and_emulation(rt, orc, n):
    import torch
    w = synth.mlp_weights(3)
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, size=(n, 2)).astype(np.float32)
    net = rt.DeviceMLP(w)
    out = rt.rt_mlp_eval(net, torch.tensor(x, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    assert rt.rt_mlp_status() == 0
    ref = orc.mlp_eval(w, x.astype(np.float64))
    emu = bf16_emulation(torch, w, x)
    scale = np.abs(ref).max()
    err_emu = np.abs(out - emu).max() / scale
    err_ref = np.abs(out - ref).max() / scale
    print(f"n={n}: output scale {scale:.3e}, max err vs BF16 emulation {err_emu:.2e}, "
          f"vs FP64 {err_ref:.2e}")
    assert err_emu < 2e-2   # differences: hardware tanh in SiLU, FP32 accumulation order
    assert err_ref < 5e-2   # BF16 rounding of weights, features and activations
