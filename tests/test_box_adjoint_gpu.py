"""Fused CUDA adjoint through the 3-D Cartesian grid (rt_render3d_adjoint) vs the FP64
oracle's reverse mode (orc_render_adjoint3, pinned by central differences of the oracle's
forward march): gradients of every node field, the rendered cube and the in-kernel loss, on
seeded boxes in every lane layout (2, 4, 8 and 16 lanes per ray), with equally and unequally
spaced channels, Mach-number turbulence, a dL/dcube seed and a target cube, plus the
degenerate calls. Gradient criterion as for the axisymmetric adjoint: 3e-4 of the field's
largest entry everywhere, 3e-3 relative on entries above 1 % of it."""

import dataclasses

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.cubecheck import assert_cube_close
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu

FIELDS = ("T", "n_h2", "vturb", "x_co", "vy", "vz")


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


def box(seed, n3, **kw):
    """A seeded box with broadened lines and thinned gas, so that every field carries
    gradient."""
    mach = kw.pop("mach", False)
    p = synth.box3d(seed, n3=n3, **kw)
    g = p.g3
    g = dataclasses.replace(g, vturb=np.full_like(g.vturb, 0.6 if mach else 0.15),
                            n_h2=g.n_h2 * 0.05)
    return p.replace(g3=g, vturb_mach=1 if mach else 0)


CASES = [
    dict(seed=0, n3=(24, 20, 12), nx=32, ny=28, nch=16, n_samples=96),            # 4 lanes x 4
    dict(seed=1, n3=(17, 23, 11), nx=20, ny=24, nch=40, n_samples=80, incl=60.0,
         pa=35.0),                                                                # 8 lanes x 8
    dict(seed=2, n3=(15, 13, 9), nx=18, ny=16, nch=6, n_samples=70, incl=20.0,
         mach=True),                                                              # 2 lanes x 4
    dict(seed=3, n3=(13, 12, 8), nx=12, ny=10, nch=100, n_samples=64, vmax=8.0),  # 16 lanes x 8
]


@pytest.mark.parametrize("case", CASES)
def test_box_adjoint_vs_oracle(rt, orc, case):
    import torch
    p = box(**case)
    w = np.random.default_rng(11 + case["seed"]).standard_normal((p.nch, p.ny, p.nx))
    ref_cube, ref = orc.render_adjoint3(p, w)
    dl = torch.tensor(w, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render3d_adjoint(p, dL_dcube=dl)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="box adjoint cube")
    got = to_np(g)
    assert np.all(got["vx"] == 0.0)
    e = assert_grads_close(got, ref, label=f"box {case}")
    print(f"box adjoint {case}: {e}")


def test_box_adjoint_unequal_channels_and_target(rt, orc):
    """Unequally spaced channels (every channel block marched: no window) and the loss formed
    in the kernel against a target cube: the gradients equal the oracle's reverse mode seeded
    with 2 (cube - target), and the loss its sum of squares."""
    import torch
    p = box(4, (14, 16, 10), nx=22, ny=18, nch=12, n_samples=72)
    rng = np.random.default_rng(5)
    v = np.sort(rng.uniform(-6.0, 6.0, p.nch))
    p = p.replace(v_kms=v)
    ref_cube = orc.render(p)
    target = ref_cube * (1.0 + 0.05 * rng.standard_normal(ref_cube.shape))
    _, ref = orc.render_adjoint3(p, 2.0 * (ref_cube - target))
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render3d_adjoint(p, target=tgt)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="unequal channels cube")
    assert_grads_close(to_np(g), ref, label="target seed")
    want = float(((ref_cube - target) ** 2).sum())
    assert float(g["loss"].item()) == pytest.approx(want, rel=1e-3)


def test_box_adjoint_degenerate_calls(rt):
    import torch
    p = box(5, (6, 5, 4), nx=8, ny=6, nch=5, n_samples=20)
    dl = torch.zeros((p.nch, p.ny, p.nx), dtype=torch.float32, device="cuda")
    with pytest.raises(rt.RTError):
        rt.rt_render3d_adjoint(p)  # neither seed
    with pytest.raises(rt.RTError):
        rt.rt_render3d_adjoint(p, dL_dcube=dl, target=dl)  # both
    # no pixels: every gradient is zero, no kernel runs
    q = p.replace(nx=0)
    cube, g = rt.rt_render3d_adjoint(q, cube_out=None)
    torch.cuda.synchronize()
    assert cube is None
    for k in ("T", "n_h2", "vturb", "x_co", "vx", "vy", "vz", "loss"):
        assert float(g[k].abs().max()) == 0.0
    # a zero seed gives zero gradients and the forward render's cube (the two kernels group
    # the optical-depth sums in batches of different lengths: rounding apart)
    cube, g = rt.rt_render3d_adjoint(p, dL_dcube=dl)
    fwd = rt.rt_render3d(p)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), fwd.cpu().numpy().astype(np.float64), rtol=1e-5,
                      label="adjoint cube vs forward")
    for k in ("T", "n_h2", "vturb", "x_co", "vx", "vy", "vz"):
        assert float(g[k].abs().max()) == 0.0


def test_box_adjoint_workload_scale(rt, orc):
    """The benchmark's 3-D workload at full size (128^3 nodes, 256^2 px, 64 channels, 256
    samples; the 8-lanes x 8-channels layout the benchmark times), every gradient entry
    against the oracle's reverse mode, with a seeded dL/dcube."""
    import torch
    p = synth.config_box(0)
    w = np.random.default_rng(21).standard_normal((p.nch, p.ny, p.nx))
    ref_cube, ref = orc.render_adjoint3(p, w)
    dl = torch.tensor(w, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render3d_adjoint(p, dL_dcube=dl)
    torch.cuda.synchronize()
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="box workload cube")
    e = assert_grads_close(to_np(g), ref, label="box workload")
    print(f"box adjoint workload: {e}")
