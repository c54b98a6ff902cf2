"""The allocation-free adjoint entry point (rt_render_adjoint_noalloc) gives the same cube
and gradients as rt_render_adjoint.

Callers that cannot allocate device memory while running (their own memory manager already
holds the device, or they run under a fixed memory budget) use this entry point; its scratch
(checkpoints and replicated gradient accumulators) is a fixed array inside the library, shared
by every call.
The test calls it twice in a row through the C ABI, so the second call runs on the array the
first call left behind, and compares both calls with the allocating entry point. This file is collected last
so that a run stopping at the first failure has already run every other test.
"""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.test_adjoint_gpu import assert_grads_close, loss_target, to_np
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def _alloc_outputs(torch, p):
    shp = (p.nz, p.nr)
    g = {k: torch.empty(shp, dtype=torch.float64, device="cuda") for k in ("T", "n_h2", "vturb")}
    g.update({k: torch.empty(p.nr, dtype=torch.float64, device="cuda") for k in ("h_lo", "h_hi")})
    g["loss"] = torch.empty(1, dtype=torch.float64, device="cuda")
    return g, torch.empty((p.nch, p.ny, p.nx), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("mode", ["target", "dL_dcube"])
def test_noalloc_matches_allocating_adjoint_twice(rt, orc, mode):
    import torch
    p = synth.config_small(31).replace(n_samples=200)   # ragged last batch
    dd = rt.DeviceDisk(p)
    tgt = torch.tensor(loss_target(orc, p, 31), dtype=torch.float32, device="cuda")
    if mode == "target":
        kw = dict(target=tgt)
    else:
        w = np.random.default_rng(1).standard_normal((p.nch, p.ny, p.nx))
        kw = dict(dL_dcube=torch.tensor(w, dtype=torch.float32, device="cuda"))
    ref_cube, ref = rt.rt_render_adjoint(p, dd, **kw)
    ref_np = to_np(ref)
    for call in range(2):
        grads, cube = _alloc_outputs(torch, p)
        for t in list(grads.values()) + [cube]:
            t.fill_(float("nan"))          # outputs must be fully written by the call
        rt.rt_render_adjoint_noalloc(p, dd, cube, grads, **kw)
        torch.cuda.synchronize()
        assert_grads_close(to_np(grads), ref_np, label=f"no-alloc call {call}")
        c, rc = cube.cpu().numpy(), ref_cube.cpu().numpy()
        np.testing.assert_allclose(c, rc, rtol=1e-6, atol=1e-7 * np.abs(rc).max())
        if mode == "target":
            assert float(grads["loss"].item()) == pytest.approx(float(ref["loss"].item()), rel=1e-9)


def test_noalloc_large_grid_without_room_for_copies(rt):
    """A 1024x512 grid: one copy of the node gradients (8.4 MB) leaves no room for a second
    in the fixed array, so the kernel adds straight into the FP64 outputs. The allocating
    call sums FP32 per-block copies (a few hundred terms each) in FP64, so the two agree to
    the FP32 rounding of those partial sums: 1e-6 of the largest entry."""
    import torch
    p = synth.disk(33, nr=1024, nz=512, nx=24, ny=24, nch=16, n_samples=128)
    dd = rt.DeviceDisk(p)
    w = np.random.default_rng(2).standard_normal((p.nch, p.ny, p.nx))
    dl = torch.tensor(w, dtype=torch.float32, device="cuda")
    _, ref = rt.rt_render_adjoint(p, dd, dL_dcube=dl)
    grads, cube = _alloc_outputs(torch, p)
    for t in grads.values():
        t.fill_(float("nan"))
    rt.rt_render_adjoint_noalloc(p, dd, cube, grads, dL_dcube=dl)
    torch.cuda.synchronize()
    for k in ("T", "n_h2", "vturb", "h_lo", "h_hi"):
        a, b = grads[k].cpu().numpy(), ref[k].cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max(), err_msg=k)


def test_noalloc_rejects_oversized_problem(rt):
    import torch
    p = synth.config_small(32).replace(nx=8, ny=8, v_kms=np.linspace(-5, 5, 200),
                                       n_samples=1 << 20)
    dd = rt.DeviceDisk(p)
    grads, cube = _alloc_outputs(torch, p)
    with pytest.raises(rt.RTError, match="fixed"):
        rt.rt_render_adjoint_noalloc(p, dd, cube, grads,
                                     dL_dcube=torch.zeros_like(cube))


def test_noalloc_with_corner_quads(rt, orc):
    """128x128 pixels x 256 samples = 2^22 samples on the 64x32 grid: enough samples for the
    corner quads of the fields to be packed, so the fixed array holds them next to the
    checkpoints and the surface and grid copies. Two calls in a row, against the allocating
    adjoint (which is checked against the oracle elsewhere)."""
    import torch
    p = synth.config_small(34).replace(nx=128, ny=128, n_samples=256)
    assert rt.rt_render_launch_count(p) == 2, "expected the corner-quad packing pass"
    dd = rt.DeviceDisk(p)
    w = np.random.default_rng(3).standard_normal((p.nch, p.ny, p.nx))
    dl = torch.tensor(w, dtype=torch.float32, device="cuda")
    ref_cube, ref = rt.rt_render_adjoint(p, dd, dL_dcube=dl)
    ref_np = to_np(ref)
    for call in range(2):
        grads, cube = _alloc_outputs(torch, p)
        for t in list(grads.values()) + [cube]:
            t.fill_(float("nan"))
        rt.rt_render_adjoint_noalloc(p, dd, cube, grads, dL_dcube=dl)
        torch.cuda.synchronize()
        assert_grads_close(to_np(grads), ref_np, label=f"no-alloc corner quads, call {call}")
        c, rc = cube.cpu().numpy(), ref_cube.cpu().numpy()
        np.testing.assert_allclose(c, rc, rtol=1e-6, atol=1e-7 * np.abs(rc).max())
