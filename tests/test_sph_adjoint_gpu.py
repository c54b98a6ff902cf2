"""Fused CUDA adjoint through the 3-D spherical grid (rt_render_sph_adjoint) vs the FP64
oracle's reverse mode (orc_render_adjoint3, pinned by central differences of the oracle's
forward march): gradients of every node field (T, n_H2, v_turb, CO abundance, v_r, v_theta,
v_phi), the rendered cube and the in-kernel loss, on seeded spherical grids in every lane
layout (2, 4, 8 and 16 lanes per ray), with equally and unequally spaced channels, Mach-number
turbulence, a dL/dcube seed and a target cube, a mid-size grid, and the degenerate calls.
Gradient criterion as for the other adjoints: 3e-4 of the field's largest entry everywhere,
3e-3 relative on entries above 1 % of it."""

import dataclasses

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.cubecheck import assert_cube_close
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu

FIELDS = ("T", "n_h2", "vturb", "x_co", "vr", "vth", "vph")


def grad_errors(got, ref):
    out = {}
    for k in FIELDS:
        g, r = np.asarray(got[k]), np.asarray(ref[k])
        m = np.abs(r).max()
        if m == 0:
            out[k] = (float(np.abs(g).max()), 0.0)
            continue
        big = np.abs(r) >= 1e-2 * m
        out[k] = (float(np.abs(g - r).max() / m),
                  float((np.abs(g - r)[big] / np.abs(r[big])).max()))
    return out


def assert_grads_close(got, ref, atol=3e-4, rtol=3e-3, label=""):
    e = grad_errors(got, ref)
    for k, (a, r) in e.items():
        assert a <= atol and r <= rtol, f"{label} {k}: scaled err {a:.2e}, rel err {r:.2e} ({e})"
    return e


def to_np(g):
    return {k: g[k].cpu().numpy() for k in g}


def sphere(seed, nsph, **kw):
    """A seeded spherical grid with broadened lines and thinned gas, so that every field
    carries gradient."""
    mach = kw.pop("mach", False)
    p = synth.sphere3d(seed, nsph=nsph, **kw)
    g = p.gs
    g = dataclasses.replace(g, vturb=np.full_like(g.vturb, 0.6 if mach else 0.15),
                            n_h2=g.n_h2 * 0.05)
    return p.replace(gs=g, vturb_mach=1 if mach else 0)


CASES = [
    dict(seed=0, nsph=(20, 10, 16), nx=32, ny=28, nch=16, n_samples=96),              # 4 x 4
    dict(seed=1, nsph=(17, 9, 13), nx=20, ny=24, nch=40, n_samples=80, incl=60.0,
         pa=35.0),                                                                    # 8 x 8
    dict(seed=2, nsph=(15, 8, 7), nx=18, ny=16, nch=6, n_samples=70, incl=20.0,
         mach=True, r_log=0, r_in=0.0),                                               # 2 x 4
    dict(seed=3, nsph=(13, 8, 9), nx=12, ny=10, nch=100, n_samples=64, vmax=8.0),     # 16 x 8
]


@pytest.mark.parametrize("case", CASES)
def test_sph_adjoint_vs_oracle(rt, orc, case):
    import torch
    p = sphere(**case)
    w = np.random.default_rng(31 + case["seed"]).standard_normal((p.nch, p.ny, p.nx))
    ref_cube, ref = orc.render_adjoint3(p, w)
    dl = torch.tensor(w, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render_sph_adjoint(p, dL_dcube=dl)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="sph adjoint cube")
    e = assert_grads_close(to_np(g), ref, label=f"sph {case}")
    print(f"sph adjoint {case}: {e}")


def test_sph_adjoint_unequal_channels_and_target(rt, orc):
    import torch
    p = sphere(4, (14, 9, 10), nx=22, ny=18, nch=12, n_samples=72)
    rng = np.random.default_rng(6)
    p = p.replace(v_kms=np.sort(rng.uniform(-6.0, 6.0, p.nch)))
    ref_cube = orc.render(p)
    target = ref_cube * (1.0 + 0.05 * rng.standard_normal(ref_cube.shape))
    _, ref = orc.render_adjoint3(p, 2.0 * (ref_cube - target))
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render_sph_adjoint(p, target=tgt)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="sph unequal channels cube")
    assert_grads_close(to_np(g), ref, label="sph target seed")
    want = float(((ref_cube - target) ** 2).sum())
    assert float(g["loss"].item()) == pytest.approx(want, rel=1e-3)


def test_sph_adjoint_mid_size(rt, orc):
    """A 64 x 24 x 48 grid (r log-spaced 20-600 au, the workload's theta range) at 64^2 px,
    32 channels and 256 samples, in the 8-lanes x 8-channels layout the workload uses."""
    import torch
    p = synth.sphere3d(7, nsph=(64, 24, 48), nx=64, ny=64, nch=32, n_samples=256, incl=47.0,
                       pa=133.0)
    w = np.random.default_rng(41).standard_normal((p.nch, p.ny, p.nx))
    ref_cube, ref = orc.render_adjoint3(p, w)
    dl = torch.tensor(w, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render_sph_adjoint(p, dL_dcube=dl)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="sph mid-size cube")
    e = assert_grads_close(to_np(g), ref, label="sph mid-size")
    print(f"sph adjoint mid-size: {e}")


def test_sph_adjoint_degenerate_calls(rt):
    import torch
    p = sphere(5, (6, 5, 4), nx=8, ny=6, nch=5, n_samples=20)
    dl = torch.zeros((p.nch, p.ny, p.nx), dtype=torch.float32, device="cuda")
    with pytest.raises(rt.RTError):
        rt.rt_render_sph_adjoint(p)
    with pytest.raises(rt.RTError):
        rt.rt_render_sph_adjoint(p, dL_dcube=dl, target=dl)
    cube, g = rt.rt_render_sph_adjoint(p.replace(ny=0), cube_out=None)
    torch.cuda.synchronize()
    assert cube is None
    for k in FIELDS + ("loss",):
        assert float(g[k].abs().max()) == 0.0
    cube, g = rt.rt_render_sph_adjoint(p, dL_dcube=dl)
    fwd = rt.rt_render_sph(p)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), fwd.cpu().numpy().astype(np.float64), rtol=1e-5,
                      label="sph adjoint cube vs forward")
    for k in FIELDS:
        assert float(g[k].abs().max()) == 0.0


@pytest.mark.parametrize("grid", ["box", "sph"])
def test_render3_autograd(rt, grid):
    """torch autograd through Render3Fn: the gradients of L = sum(w * cube) with respect to the
    seven node fields equal the fused adjoint's (same kernel, same seed), and the cube equals
    the forward render."""
    import torch
    from paper_2509_03623_b300 import autograd
    if grid == "box":
        p = synth.box3d(8, n3=(14, 12, 9), nx=20, ny=18, nch=16, n_samples=64)
        dg, keys, adjoint, render = (rt.DeviceGrid3(p), rt.DeviceGrid3.FIELDS,
                                     rt.rt_render3d_adjoint, rt.rt_render3d)
    else:
        p = sphere(8, (14, 9, 10), nx=20, ny=18, nch=16, n_samples=64)
        dg, keys, adjoint, render = (rt.DeviceGridSph(p), rt.DeviceGridSph.FIELDS,
                                     rt.rt_render_sph_adjoint, rt.rt_render_sph)
    fields = [getattr(dg, k).clone().requires_grad_(True) for k in keys]
    w = torch.randn((p.nch, p.ny, p.nx), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    cube = autograd.render3(p, *fields)
    (cube * w).sum().backward()
    _, g = adjoint(p, dg, dL_dcube=w.contiguous(), cube_out=None)
    ref = render(p, dg)
    torch.cuda.synchronize()
    assert torch.equal(cube.detach(), ref)
    for k, f in zip(keys, fields):
        a, b = f.grad.double(), g[k]
        scale = float(b.abs().max())
        assert float((a - b).abs().max()) <= 1e-5 * max(scale, 1e-300), k
