"""Pressure-corrected rotation (next row f3) on the GPU vs the FP64 oracle: the node field
from rt_pressure_vphi, and the march driven by a rotation field (node-array and corner-quad
paths).

Tolerance of the node field, from FP32 arithmetic: the pressure term differences n T at
neighbouring nodes, whose relative change per node is >= ~1e-2 on these grids, so each
difference carries ~6e-8 / 1e-2 = 6e-6 relative error; the term itself is <~3 % of the
Keplerian v^2, and the Keplerian term carries a few 1e-7. Compared on v_phi^2 (which is what
the formula produces; v_phi = sqrt(v_phi^2) amplifies errors where the pressure term nearly
cancels gravity): |dv^2| <= 1e-5 of the node's Keplerian v^2.
"""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.cubecheck import assert_cube_close
from tests.test_forward_gpu import gpu_cube, rt  # noqa: F401  (module fixture)
from tests.test_oracle_vphi import kepler_kms

pytestmark = pytest.mark.gpu

GM_SUN = 1.3271244e26
AU_CM = 1.495978707e13


def kepler2(p):
    r = p.r_nodes()[None, :] * AU_CM
    z = p.zr_nodes()[:, None] * r
    return GM_SUN * p.mstar_msun * r * r / (r * r + z * z) ** 1.5 / 1e10  # km^2 s^-2


@pytest.mark.parametrize("which", ["small", "observation", "linear"])
def test_rotation_field_vs_oracle(rt, orc, which):
    import torch
    p = {"small": synth.config_small(6), "observation": synth.config_observation(1),
         "linear": synth.config_small(7).replace(r_log=0)}[which]
    n32 = np.ascontiguousarray(p.n_h2, dtype=np.float32)
    T32 = np.ascontiguousarray(p.T, dtype=np.float32)
    v = rt.rt_pressure_vphi(p, torch.tensor(n32, device="cuda"), torch.tensor(T32, device="cuda"))
    torch.cuda.synchronize()
    got = v.cpu().numpy().astype(np.float64)
    ref = orc.pressure_vphi(p, n32.astype(np.float64), T32.astype(np.float64))
    err = np.abs(got ** 2 - ref ** 2) / kepler2(p)
    print(f"rotation {which}: max |dv^2| / v_K^2 = {err.max():.2e}, "
          f"sub-Keplerian by up to {1 - (ref / np.sqrt(kepler2(p))).min():.3f}")
    assert err.max() <= 1e-5


def test_render_with_rotation_field(rt, orc):
    p = synth.config_small(8)
    vphi = orc.pressure_vphi(p).astype(np.float32).astype(np.float64)
    q = p.replace(vphi=vphi)
    assert_cube_close(gpu_cube(rt, q), orc.render(q), label="rotation field")
    # the pressure term is visible: the cube differs from the Keplerian render
    kep = orc.render(p)
    assert np.abs(orc.render(q) - kep).max() > 1e-3 * np.abs(kep).max()


def test_render_with_rotation_field_corner_quads(rt, orc):
    """4.19 M samples: the rotation field is read from the fourth corner quad. The disk is
    the observation grid (512x256, 64 channels, rings) without the per-node log-normal
    noise: with that noise the pressure term differs node to node by tens of per cent and
    clamps some nodes to v_phi = 0, so v_los jumps by km/s inside a cell and the FP32 sample
    positions (about one rounding of 600 au) move it by 1e-4 km/s, ~1e-3 of a line width:
    such fields are outside the 1e-4 parity criterion by construction, not by the march."""
    p = synth.disk(2, nr=512, nz=256, nx=128, ny=128, nch=64, vmax=6.0, n_samples=256,
                   incl=47.0, pa=133.0, rings=3)
    vphi = orc.pressure_vphi(p).astype(np.float32).astype(np.float64)
    q = p.replace(vphi=vphi)
    assert_cube_close(gpu_cube(rt, q), orc.render(q), label="rotation field, corner quads")


def vphi_adjoint_case(rt, orc, p, seed):
    """GPU adjoint with a rotation field vs the oracle's (orc_render_adjoint_vphi), seeded with
    dL/dcube = 2 (I - I*) against a fixed target."""
    import torch
    from tests.test_adjoint_gpu import assert_grads_close, loss_target
    tgt = loss_target(orc, p, seed)
    cube_ref = orc.render(p)
    dl = 2.0 * (cube_ref - tgt)
    _, g_ref = orc.render_adjoint_vphi(p, dl)
    dd = rt.DeviceDisk(p)
    _, g = rt.rt_render_adjoint(p, dd, dL_dcube=torch.tensor(dl.astype(np.float32), device="cuda"),
                                cube_out=None)
    got = {k: g[k].cpu().numpy() for k in ("T", "n_h2", "vturb", "h_lo", "h_hi", "vphi")}
    return assert_grads_close(got, g_ref, label="rotation field")


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_with_rotation_field_vs_oracle(rt, orc, seed):
    """64x32 grid, 64^2 px, 16 channels, 128 samples, the pressure-corrected rotation of the
    disk as the field (node-array path)."""
    p = synth.config_small(seed)
    q = p.replace(vphi=orc.pressure_vphi(p).astype(np.float32).astype(np.float64))
    print("rotation-field adjoint", vphi_adjoint_case(rt, orc, q, seed))


def test_adjoint_with_rotation_field_corner_quads(rt, orc):
    """A grid large enough for the corner quads (four per cell with a rotation field), 64
    channels; the smooth disk of the forward test above."""
    p = synth.disk(2, nr=256, nz=128, nx=96, ny=96, nch=64, vmax=6.0, n_samples=512,
                   incl=47.0, pa=133.0, rings=3)
    q = p.replace(vphi=orc.pressure_vphi(p).astype(np.float32).astype(np.float64))
    print("rotation-field adjoint, corner quads", vphi_adjoint_case(rt, orc, q, 2))


def test_adjoint_with_rotation_field_needs_its_gradient_output(rt):
    import torch
    from paper_2509_03623_b300 import _rt
    p = synth.config_small(0)
    q = p.replace(vphi=np.full((p.nz, p.nr), 3.0))
    dd = rt.DeviceDisk(q)
    grads = {k: torch.zeros(tuple(t.shape), dtype=torch.float64, device="cuda")
             for k, t in zip(("T", "n_h2", "vturb", "h_lo", "h_hi"), dd.tensors())}
    with pytest.raises(rt.RTError, match="dvphi"):
        rt.rt_render_adjoint_noalloc(q, dd, None, grads,
                                     dL_dcube=torch.zeros((q.nch, q.ny, q.nx), device="cuda"))


def test_autograd_render_with_rotation_field(rt, orc):
    """RenderFn with a rotation field: the rotation field's gradient (and the others) equal
    those of the explicit adjoint call."""
    import torch
    from paper_2509_03623_b300 import autograd
    p = synth.config_small(3)
    q = p.replace(vphi=orc.pressure_vphi(p).astype(np.float32).astype(np.float64))
    dd = rt.DeviceDisk(q)
    ins = [t.clone().requires_grad_(True) for t in dd.tensors()]
    vp = dd.vphi.clone().requires_grad_(True)
    cube = autograd.render(q, *ins, vphi=vp)
    w = torch.randn(tuple(cube.shape), device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    (cube * w).sum().backward()
    _, g = rt.rt_render_adjoint(q, dd, dL_dcube=w.contiguous(), cube_out=None)
    for got, k in zip(ins + [vp], ("T", "n_h2", "vturb", "h_lo", "h_hi", "vphi")):
        want = g[k].float()
        scale = float(want.abs().max())
        assert scale > 0, k
        assert float((got.grad - want).abs().max()) <= 1e-5 * scale, k


@pytest.mark.parametrize("r_log,nr,nz", [(1, 64, 32), (0, 33, 17), (1, 512, 256)])
def test_rotation_reverse_mode_vs_oracle(rt, orc, r_log, nr, nz):
    """rt_pressure_vphi_adjoint vs orc_pressure_vphi_adjoint from the same float32 fields. The
    kernel evaluates the pressure term in FP32 (differences of n T: ~1e-6 relative of the
    term), so entries above 1 % of the largest agree to 1e-3 relative and all to 1e-5 of it."""
    import torch
    p = synth.config_small(4).replace(nr=nr, nz=nz, r_log=r_log, r_in_au=30.0, r_out_au=600.0)
    rng = np.random.default_rng(nr + nz)
    # node-to-node noise scaled with the node count, so the pressure term (differences over
    # the node spacing) stays a correction: near the clamp v_phi -> 0 the derivative grows as
    # 1 / v_phi and FP32 against FP64 differences there say nothing about the kernel
    amp = 0.05 * min(1.0, 32.0 / nr)
    n = (1e7 * np.exp(rng.uniform(-amp, amp, (nz, nr)))).astype(np.float32)
    T = (30.0 * np.exp(rng.uniform(-amp, amp, (nz, nr)))).astype(np.float32)
    v = orc.pressure_vphi(p, n.astype(np.float64), T.astype(np.float64))
    assert np.all(v > 0.5 * kepler_kms(p)), "a node near the clamp"
    g = rng.standard_normal((nz, nr))
    gn, gT = rt.rt_pressure_vphi_adjoint(p, torch.tensor(n, device="cuda"),
                                         torch.tensor(T, device="cuda"),
                                         torch.tensor(g, device="cuda"))
    rn, rT = orc.pressure_vphi_adjoint(p, g, n.astype(np.float64), T.astype(np.float64))
    for got, ref, k in ((gn.cpu().numpy(), rn, "n"), (gT.cpu().numpy(), rT, "T")):
        scale = np.abs(ref).max()
        assert scale > 0, k
        assert np.abs(got - ref).max() <= 1e-5 * scale, k
        big = np.abs(ref) >= 0.01 * scale
        assert (np.abs(got - ref)[big] / np.abs(ref)[big]).max() <= 1e-3, k
