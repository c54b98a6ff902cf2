"""3-D renders from node records packed once (rt_pack_nodes3 + rt_render3d_packed /
rt_render_sph_packed): bit-identical to the renders that pack per call, for several views,
channel sets and image sizes from one packing, on the Cartesian and the spherical grid; bad
record pointers are rejected on the host."""

import ctypes as C

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid", ["box", "sph"])
def test_packed_renders_equal_unpacked(rt, grid):
    import torch
    if grid == "box":
        p = synth.box3d(3, n3=(33, 27, 19), nx=40, ny=24, nch=20, n_samples=100, incl=60.0,
                        pa=35.0)
        dg, render = rt.DeviceGrid3(p), rt.rt_render3d
    else:
        p = synth.sphere3d(4, nsph=(40, 16, 24), nx=36, ny=28, nch=24, n_samples=120,
                           incl=47.0, pa=133.0)
        dg, render = rt.DeviceGridSph(p), rt.rt_render_sph
    rec = rt.rt_pack_nodes3(p, dg)
    views = [p, p.replace(v_kms=np.linspace(-3.0, 3.0, 40)), p.replace(nx=64, ny=48),
             p.replace(incl_deg=20.0, pa_deg=-70.0, n_samples=64),
             p.replace(vturb_mach=1, v_kms=np.linspace(-6.0, 6.0, 7))]
    for q in views:
        a = rt.rt_render_packed(q, rec)
        b = render(q, dg)
        torch.cuda.synchronize()
        assert torch.equal(a, b), (grid, q.nx, q.nch, q.incl_deg)
        assert float(b.abs().max()) > 0


def test_packed_rejects_bad_records(rt):
    import torch
    p = synth.box3d(5, n3=(9, 8, 7), nx=8, ny=6, nch=5, n_samples=20)
    dg = rt.DeviceGrid3(p)
    nodes = 9 * 8 * 7
    f = rt.rt_fields3(*(getattr(dg, k).data_ptr() for k in rt.DeviceGrid3.FIELDS), 0)
    buf = torch.empty(8 * nodes + 4, dtype=torch.float32, device="cuda")
    L = rt.lib()
    assert L.rt_pack_nodes3(C.byref(f), nodes, C.c_void_p(buf.data_ptr() + 4), None) == -1
    assert b"aligned" in L.rt_last_error()
    assert L.rt_pack_nodes3(C.byref(f), nodes, None, None) == -1
    assert L.rt_pack_nodes3(C.byref(f), 0, C.c_void_p(buf.data_ptr()), None) == -1
    with pytest.raises(ValueError):
        rt.rt_render_packed(p, buf[: 8 * nodes - 8])  # records of another grid size


@pytest.mark.parametrize("grid", ["box", "sph"])
def test_packed_adjoints_equal_unpacked(rt, grid):
    """The 3-D adjoints from records packed once: the same cube bit for bit and the same
    gradients up to the order of the FP32 reductions (1e-6 of each field's largest entry)."""
    import torch
    if grid == "box":
        p = synth.box3d(6, n3=(21, 17, 13), nx=28, ny=24, nch=16, n_samples=80)
        dg, adjoint = rt.DeviceGrid3(p), rt.rt_render3d_adjoint
    else:
        p = synth.sphere3d(6, nsph=(24, 12, 16), nx=28, ny=24, nch=16, n_samples=96)
        dg, adjoint = rt.DeviceGridSph(p), rt.rt_render_sph_adjoint
    rec = rt.rt_pack_nodes3(p, dg)
    w = torch.randn((p.nch, p.ny, p.nx), device="cuda",
                    generator=torch.Generator("cuda").manual_seed(5))
    c0, g0 = adjoint(p, dg, dL_dcube=w)
    c1, g1 = rt.rt_render_adjoint_packed(p, rec, dL_dcube=w)
    torch.cuda.synchronize()
    assert torch.equal(c0, c1)
    for k in g0:
        if k == "loss":
            continue
        scale = float(g0[k].abs().max())
        assert float((g0[k] - g1[k]).abs().max()) <= 1e-6 * max(scale, 1e-300), k
