"""Reverse mode through the neural field on the GPU (tensor-core network backward and the
fused march adjoint with the network's modulation) vs the FP64 oracle.

Tolerances are those of 16-bit tensor-core operands: every weight, activation and delta is
rounded to FP16 (11-bit significand) or BF16 (8-bit) before each MMA, with FP32 accumulation,
so a gradient entry that sums many products carries a relative error of a few units of the
16-bit rounding; compared per array as max |gpu - oracle| / max |oracle| (scaled error).
"""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu

SCALED_TOL = {"f16": 4e-3, "bf16": 2.5e-2}


def scaled_err(got, ref):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    m = np.abs(ref).max()
    return float(np.abs(got - ref).max() / m) if m > 0 else float(np.abs(got).max())


def net_weights(seed=7):
    w = synth.mlp_weights(seed)
    rng = np.random.default_rng(seed)
    w.b = [rng.uniform(-0.1, 0.1, size=b.shape).astype(np.float32) for b in w.b]
    return w


@pytest.mark.parametrize("prec", ["f16", "bf16"])
# sizes around the backward's 64-sample tiles and a CTA's pair of tile groups, and one with
# several tiles per group (both groups accumulating into the same weight gradients)
@pytest.mark.parametrize("n", [1, 63, 64, 65, 128, 129, 300, 5000, 40001])
def test_mlp_backward_vs_oracle(rt, orc, prec, n):
    """Random inputs (ragged last tile, a single input, several tiles per CTA) and random
    output gradients spanning a wide dynamic range (the kernel scales them to FP16 range)."""
    import torch
    w = net_weights()
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, size=(n, 2))
    gout = rng.standard_normal((n, 4)) * 1e-9   # far below FP16's smallest normal
    dW_ref, db_ref = orc.mlp_grad(w, x.astype(np.float32), gout.astype(np.float32))
    net = rt.DeviceMLP(w, precision=prec)
    dW, db = rt.rt_mlp_backward(net, torch.tensor(x, dtype=torch.float32, device="cuda"),
                                torch.tensor(gout, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert rt.rt_mlp_status() == 0
    errs = [scaled_err(dW[l].cpu().numpy(), dW_ref[l]) for l in range(5)]
    errs += [scaled_err(db[l].cpu().numpy(), db_ref[l]) for l in range(5)]
    print(f"mlp backward {prec} n={n}: W {errs[:5]} b {errs[5:]}")
    assert max(errs) <= SCALED_TOL[prec], errs


def small_neural_problem(seed=0):
    return synth.config_small(seed).replace(nx=24, ny=20, n_samples=64)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_render_mlp_adjoint_vs_oracle(rt, orc, prec):
    import torch
    p = small_neural_problem(3)
    w = net_weights(5)
    rng = np.random.default_rng(8)
    G = rng.standard_normal((p.nch, p.ny, p.nx))
    cube_ref, g_ref = orc.render_mlp_adjoint(p, w, G)
    dd = rt.DeviceDisk(p)
    net = rt.DeviceMLP(w, precision=prec)
    cube, g, (dW, db) = rt.rt_render_mlp_adjoint(
        p, dd, net, dL_dcube=torch.tensor(G, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert rt.rt_mlp_status() == 0
    c = cube.cpu().numpy()
    cube_err = scaled_err(c, cube_ref)
    node = {k: scaled_err(g[k].cpu().numpy(), g_ref[k]) for k in ("T", "n_h2", "vturb", "h_lo", "h_hi")}
    werr = [scaled_err(dW[l].cpu().numpy(), g_ref["W"][l]) for l in range(5)]
    berr = [scaled_err(db[l].cpu().numpy(), g_ref["b"][l]) for l in range(5)]
    print(f"neural adjoint {prec}: cube {cube_err:.2e} nodes {node} W {werr} b {berr}")
    assert cube_err <= SCALED_TOL[prec]
    assert max(node.values()) <= SCALED_TOL[prec], node
    assert max(werr + berr) <= SCALED_TOL[prec], (werr, berr)


def test_render_mlp_adjoint_target_mode_and_loss(rt, orc):
    """Fused loss target: the loss value and the gradients match the dL/dcube seed form."""
    import torch
    p = small_neural_problem(4)
    w = net_weights(6)
    dd = rt.DeviceDisk(p)
    net = rt.DeviceMLP(w, precision="f16")
    cube = rt.rt_render_mlp(p, dd, net)
    tgt = (cube * 1.03 + 1e-3 * cube.abs().max()).contiguous()
    c1, g1, (dW1, db1) = rt.rt_render_mlp_adjoint(p, dd, net, target=tgt)
    c2, g2, (dW2, db2) = rt.rt_render_mlp_adjoint(p, dd, net, dL_dcube=2.0 * (c1 - tgt))
    torch.cuda.synchronize()
    loss = float(((c1.double() - tgt.double()) ** 2).sum())
    assert float(g1["loss"].item()) == pytest.approx(loss, rel=1e-5)
    for l in range(5):
        assert scaled_err(dW1[l].cpu().numpy(), dW2[l].cpu().numpy()) <= 1e-6
    for k in ("T", "n_h2", "h_lo"):
        assert scaled_err(g1[k].cpu().numpy(), g2[k].cpu().numpy()) <= 1e-6
