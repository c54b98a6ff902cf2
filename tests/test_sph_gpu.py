"""3-D spherical grid march (next row f4) on the GPU vs the FP64 oracle: full cubes of seeded
spherical grids (odd node counts, a linear radial grid from the centre over the full
colatitude range, a single azimuth node, position angle, Jy units and background, rays that
miss), and the node count of the paper's runtime benchmark (512 x 96 x 256) at 256^2 px, 64
channels and 512 samples on sampled pixels, in the launch configuration the benchmark times.
Same parity criterion as the axisymmetric forward (1e-4 relative above 1e-3 of the peak,
3e-7 of the peak below)."""

import math

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.cubecheck import assert_cube_close
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def gpu_cube_sph(rt, p):
    import torch
    out = rt.rt_render_sph(p)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", [
    dict(seed=0, nsph=(48, 24, 32)),
    dict(seed=1, nsph=(37, 19, 23), nx=40, ny=24, nch=20, incl=60.0, pa=35.0),
    dict(seed=2, nsph=(29, 41, 17), r_log=0, r_in=0.0, th_range=(0.0, math.pi), nx=31,
         ny=33, n_samples=100, incl=15.0),
    dict(seed=3, nsph=(40, 16, 1), nx=24, ny=24, incl=75.0, pa=-20.0),
])
def test_sph_full_cube(rt, orc, case):
    kw = dict(nsph=(32, 16, 24), nx=32, ny=32, nch=16, n_samples=128)
    kw.update(case)
    p = synth.sphere3d(**kw)
    e = assert_cube_close(gpu_cube_sph(rt, p), orc.render(p), label=str(case))
    print(f"sph {case}: {e}")


def test_sph_units_background_and_misses(rt, orc):
    p = synth.sphere3d(3, nsph=(24, 12, 16), nx=20, ny=20, nch=12, n_samples=96, incl=50.0)
    q = p.replace(units=1, I0=2e-3, half_fov_au=900.0)   # rays outside the sphere keep I0
    assert_cube_close(gpu_cube_sph(rt, q), orc.render(q), label="Jy + I0")


def test_sph_workload_scale(rt, orc):
    """512 x 96 x 256 nodes, 256^2 px, 64 channels, 512 samples (33.5 M samples): the
    brightest pixels and random ones."""
    p = synth.config_sph(0)
    g = gpu_cube_sph(rt, p)
    rng = np.random.default_rng(1)
    flux = g.sum(axis=0).ravel()
    pix = np.unique(np.concatenate([np.argsort(flux)[::-1][:24],
                                    rng.choice(p.nx * p.ny, 24, replace=False)]))
    ref = orc.render_pixels(p, pix)
    got = g.reshape(p.nch, -1)[:, pix].T
    assert_cube_close(got, ref, label="spherical workload")


@pytest.mark.parametrize("bad", [dict(th1=3.5), dict(nr=1), dict(r_in=-1.0),
                                 dict(r_log=1, r_in=0.0)])
def test_sph_rejects_bad_grid(rt, bad):
    p = synth.sphere3d(0, nsph=(4, 4, 4), nx=8, ny=8, nch=4, n_samples=16)
    g = p.gs
    kw = {k: getattr(g, k) for k in ("nr", "nth", "nph", "r_log", "r_in", "r_out", "th0",
                                     "th1", "T", "n_h2", "vturb", "x_co", "vr", "vth", "vph")}
    kw.update(bad)
    if "nr" in bad:  # keep the arrays consistent with the node counts
        for k in ("T", "n_h2", "vturb", "x_co", "vr", "vth", "vph"):
            kw[k] = np.ascontiguousarray(kw[k][:, :, :bad["nr"]])
    with pytest.raises(rt.RTError):
        rt.rt_render_sph(p.replace(gs=synth.GridSph(**kw)))


def test_sph_mach_turbulence(rt, orc):
    """Turbulence given as a Mach number (the paper's form) on the spherical grid."""
    p = synth.sphere3d(5, nsph=(30, 14, 20), nx=24, ny=24, nch=16, n_samples=96, incl=55.0)
    g = p.gs
    gs = synth.GridSph(g.nr, g.nth, g.nph, g.r_log, g.r_in, g.r_out, g.th0, g.th1, g.T, g.n_h2,
                       np.full_like(g.T, 0.3), g.x_co, g.vr, g.vth, g.vph)
    q = p.replace(gs=gs, vturb_mach=1)
    assert_cube_close(gpu_cube_sph(rt, q), orc.render(q), label="sph Mach")
