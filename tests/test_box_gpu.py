"""3-D Cartesian grid march (next row f4) on the GPU vs the FP64 oracle: full cubes of
seeded 3-D boxes (odd node counts, unequal extents, rays that miss, position angle, Jy units
and background) and a box at 4.2 M samples in the launch configuration the benchmark times.
Same parity criterion as the axisymmetric forward (1e-4 relative above 1e-3 of the peak,
3e-7 of the peak below)."""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.cubecheck import assert_cube_close
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def gpu_cube3(rt, p):
    import torch
    out = rt.rt_render3d(p)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


# The rotation flips sign across the central cells (tens of km/s, >100 line widths, within
# one cell on the coarse grids), so 1e-6 of a cell in the interpolation weights would move
# line-wing intensities by ~1e-4: the kernel measures positions from the node nearest the box
# centre, where FP32 coordinates are finest. The coarse 33x27x19 case checks that.
@pytest.mark.parametrize("case", [
    dict(seed=0, n3=(64, 64, 32)),
    dict(seed=1, n3=(65, 53, 37), nx=40, ny=24, nch=20, incl=60.0, pa=35.0),
    dict(seed=2, n3=(41, 97, 33), half_xy=400.0, half_z=200.0, n_samples=100, incl=15.0),
    dict(seed=1, n3=(33, 27, 19), nx=40, ny=24, nch=20, incl=60.0, pa=35.0),
])
def test_box_full_cube(rt, orc, case):
    kw = dict(n3=(32, 32, 16), nx=32, ny=32, nch=16, n_samples=128)
    kw.update(case)
    p = synth.box3d(**kw)
    e = assert_cube_close(gpu_cube3(rt, p), orc.render(p), label=str(case))
    print(f"box {case}: {e}")


def test_box_units_background_and_misses(rt, orc):
    p = synth.box3d(3, n3=(24, 24, 12), nx=20, ny=20, nch=12, n_samples=96, incl=50.0)
    q = p.replace(units=1, I0=2e-3, half_fov_au=900.0)   # rays outside the box keep I0
    assert_cube_close(gpu_cube3(rt, q), orc.render(q), label="Jy + I0")


def test_box_workload_scale(rt, orc):
    """128^3 nodes, 128^2 px, 64 channels, 256 samples (4.2 M samples): sampled pixels."""
    p = synth.config_box(0).replace(nx=128, ny=128)
    g = gpu_cube3(rt, p)
    rng = np.random.default_rng(1)
    flux = g.sum(axis=0).ravel()
    pix = np.unique(np.concatenate([np.argsort(flux)[::-1][:40],
                                    rng.choice(p.nx * p.ny, 40, replace=False)]))
    ref = orc.render_pixels(p, pix)
    got = g.reshape(p.nch, -1)[:, pix].T
    assert_cube_close(got, ref, label="box workload")


def test_box_rejects_bad_grid(rt):
    import torch
    p = synth.box3d(0, n3=(4, 4, 4), nx=8, ny=8, nch=4, n_samples=16)
    g3 = p.g3
    bad = synth.Grid3(g3.nx, g3.ny, g3.nz, (10.0, -10.0) + tuple(g3.extent[2:]), g3.T, g3.n_h2,
                      g3.vturb, g3.x_co, g3.vx, g3.vy, g3.vz)
    with pytest.raises(rt.RTError):
        rt.rt_render3d(p.replace(g3=bad))
