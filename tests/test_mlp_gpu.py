"""Tensor-core neural-field network (tcgen05, FP32 accumulation) against the FP64 oracle
network: FP16 operands (one pass, checked against a torch emulation of the same roundings as
well) and BF16 operands (split product: BF16 main product, FP8 E5M2 correction products, FP32
SiLU, FP32 output layer)."""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.test_forward_gpu import rt  # noqa: F401

pytestmark = pytest.mark.gpu


def emulation(torch, w, x, dt):
    """Same network with the kernel's roundings: features, weights and hidden activations in
    the 16-bit format dt, products accumulated in FP32, exact SiLU."""
    xt = torch.tensor(x, dtype=torch.float32)
    B = torch.tensor(w.B, dtype=torch.float32)
    ph = xt @ B.T
    ph = ph - torch.round(ph)
    h = torch.cat([torch.sin(2 * np.pi * ph), torch.cos(2 * np.pi * ph)], 1)
    h = h.to(dt).float()
    for l, (W, b) in enumerate(zip(w.W, w.b)):
        Wt = torch.tensor(W).to(dt).float()
        h = h @ Wt.T + torch.tensor(b)
        if l < len(w.W) - 1:
            h = torch.nn.functional.silu(h).to(dt).float()
    return h.numpy()


# sizes around the tiles (FP16: 128 samples, BF16: 64) and a CTA's three tile groups
@pytest.mark.parametrize("prec,n", [("f16", 1), ("f16", 127), ("f16", 128), ("f16", 385),
                                    ("f16", 5000), ("f16", 100_003),
                                    ("bf16", 1), ("bf16", 63), ("bf16", 64), ("bf16", 65),
                                    ("bf16", 128), ("bf16", 191), ("bf16", 193),
                                    ("bf16", 100_003)])
def test_mlp_tensor_cores_vs_oracle_and_emulation(rt, orc, prec, n):
    import torch
    w = synth.mlp_weights(3)
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, size=(n, 2)).astype(np.float32)
    net = rt.DeviceMLP(w, precision=prec)
    out = rt.rt_mlp_eval(net, torch.tensor(x, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    assert rt.rt_mlp_status() == 0
    ref = orc.mlp_eval(w, x.astype(np.float64))
    scale = np.abs(ref).max()
    err_ref = np.abs(out - ref).max() / scale
    if prec == "f16":
        # 16-bit roundings of weights, features and activations; hardware tanh in SiLU
        emu = emulation(torch, w, x, torch.float16)
        err_emu = np.abs(out - emu).max() / scale
        print(f"f16 n={n}: output scale {scale:.3e}, max err vs emulation {err_emu:.2e}, "
              f"vs FP64 {err_ref:.2e}")
        assert err_emu < 2e-3 and err_ref < 2e-3
    else:
        # split BF16 operands: the BF16 roundings of the main product are corrected by the
        # products W a_lo and W_lo a, themselves ~2^-8 of it and formed with E5M2 factors
        # (2^-3 relative), so about 2^-11 of each term remains, largely averaging out over the
        # 128-term products; with the hardware tanh of SiLU and FP32 accumulation the outputs
        # stay within a few 1e-4 of FP64 (the workload's bar is 3e-3)
        print(f"bf16 n={n}: output scale {scale:.3e}, max err vs FP64 {err_ref:.2e}")
        assert err_ref < 1e-3


def neural_case(seed=0, **kw):
    p = synth.config_neural(seed).replace(**kw)
    return p, synth.mlp_weights(seed + 7)


@pytest.mark.parametrize("kw", [
    dict(nx=40, ny=36, v_kms=np.linspace(-6, 6, 24), n_samples=96),
    dict(nx=33, ny=29, v_kms=np.linspace(-5, 5, 40), n_samples=100, incl_deg=70.0),
])
def test_render_mlp_vs_oracle(rt, orc, kw):
    """Tensor-core neural-field render vs the FP64 oracle: FP16 and BF16 operands within 3e-3
    per voxel above 1e-3 of the peak (the tolerance of the 16-bit network path); the FP32
    network through the same march within 1e-4."""
    import torch
    from paper_2509_03623_b300 import neural
    from tests.cubecheck import assert_cube_close
    p, w = neural_case(1, **kw)
    dd = rt.DeviceDisk(p)
    ref = orc.render_mlp(p, w)
    f16 = rt.rt_render_mlp(p, dd, rt.DeviceMLP(w, precision="f16")).cpu().numpy()
    bf16 = rt.rt_render_mlp(p, dd, rt.DeviceMLP(w, precision="bf16")).cpu().numpy()
    fp32 = neural.render_mlp_fp32(p, dd, rt.DeviceMLP(w)).cpu().numpy()
    torch.cuda.synchronize()
    assert rt.rt_mlp_status() == 0
    e16 = assert_cube_close(f16, ref, rtol=3e-3, small_abs=3e-6, label="f16 mlp")
    eb = assert_cube_close(bf16, ref, rtol=3e-3, small_abs=3e-6, label="bf16 mlp")
    e32 = assert_cube_close(fp32, ref, rtol=1e-4, label="fp32 mlp")
    print(f"mlp render {list(kw)}: f16 {e16}, bf16 {eb}, fp32 {e32}")
    # the network matters: a zero network gives a different cube
    plain = rt.rt_render(p, dd).cpu().numpy()
    assert np.abs(plain - ref).max() > 1e-2 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_render_mlp_neural_workload_sampled(rt, orc, prec):
    """512x512 px, 128 channels, 256 samples (the neural-field workload) in the launch
    configuration of the benchmark; the oracle computes 48 sampled spectra; 3e-3 per voxel
    above 1e-3 of the peak for either operand format."""
    import torch
    p, w = neural_case(2)
    dd = rt.DeviceDisk(p)
    net = rt.DeviceMLP(w, precision=prec)
    cube = rt.rt_render_mlp(p, dd, net).cpu().numpy()
    torch.cuda.synchronize()
    flux = cube.sum(axis=0).ravel()
    rng = np.random.default_rng(3)
    pix = np.unique(np.concatenate([np.argsort(flux)[::-1][:32],
                                    rng.choice(p.nx * p.ny, 16, replace=False)]))
    ref = orc.render_mlp(p, w, pix=pix)
    got = cube.reshape(p.nch, -1)[:, pix].T
    peak = np.abs(ref).max()
    big = np.abs(ref) > 1e-3 * peak
    rel = np.abs(got - ref)[big] / np.abs(ref)[big]
    print(f"neural workload {prec}: {big.sum()} voxels, max rel {rel.max():.3e}")
    assert big.sum() > 500 and rel.max() <= 3e-3
