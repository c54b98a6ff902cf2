"""Field chain on the GPU (hydrostatic density, H2 column, CO-layer surfaces) vs the FP64
oracle on the same float32 temperature grid.

Tolerances from the FP32 arithmetic: the height integral I_j is a warp scan (depth
log2(32) plus one carry per 32-node chunk, ~13 roundings), so the exponent -I_j carries
about 13 x 2^-24 |I_j|; where the density is above 1e-6 of its column maximum |I_j| <= ~15,
giving ~1.2e-5 relative plus the expf/logf ulps; the normalisation and the column add a few
1e-6. Required: 1e-4 relative there, 1e-9 of the column maximum below it; surfaces to 1e-5
in z/r (a crossing moves by the relative error of N_H2 times N_H2 / |dN_H2/dw| < 0.1).
"""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.cubecheck import assert_cube_close
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def check_chain(got, ref, label=""):
    n, nr_ = got["n_h2"], ref["n_h2"]
    colmax = nr_.max(axis=0, keepdims=True)
    big = nr_ > 1e-6 * colmax
    rel = np.abs(n - nr_)[big] / nr_[big]
    assert rel.max() <= 1e-4, f"{label} n_h2 rel {rel.max():.2e}"
    assert (np.abs(n - nr_)[~big] <= 1e-9 * np.broadcast_to(colmax, n.shape)[~big]).all(), label
    if got["N_h2"] is not None:
        N, Nr = got["N_h2"], ref["N_h2"]
        bigN = Nr > 1e-6 * Nr[0:1]
        relN = np.abs(N - Nr)[bigN] / Nr[bigN]
        assert relN.max() <= 1e-4, f"{label} N_h2 rel {relN.max():.2e}"
    for k in ("h_lo", "h_hi"):
        d = np.abs(got[k] - ref[k]).max()
        assert d <= 1e-5, f"{label} {k} max diff {d:.2e}"
    return float(rel.max())


def run_both(rt, orc, p, T, chain, column=True):
    import torch
    T32 = np.ascontiguousarray(T, dtype=np.float32)
    out = rt.rt_field_chain(p, torch.tensor(T32, device="cuda"), chain, column=column)
    torch.cuda.synchronize()
    got = {k: (v.cpu().numpy().astype(np.float64) if v is not None else None)
           for k, v in out.items()}
    ref = orc.field_chain(p, chain, T32.astype(np.float64))
    return got, ref


def test_observation_grid(rt, orc):
    p = synth.config_observation(0)
    got, ref = run_both(rt, orc, p, p.T, synth.chain_params(p))
    print("chain obs grid: n rel", check_chain(got, ref, "obs"))


@pytest.mark.parametrize("nr,nz,r_log", [(7, 45, 1), (5, 33, 0), (3, 2, 1), (9, 32, 1),
                                         (6, 97, 1)])
def test_ragged_grids(rt, orc, nr, nz, r_log):
    p = synth.config_small(3)
    rng = np.random.default_rng(nr * 100 + nz)
    T = 12.0 + 50.0 * rng.random((nz, nr)) + 30.0 * np.linspace(0, 1, nz)[:, None]
    q = p.replace(nr=nr, nz=nz, r_log=r_log, T=T, n_h2=np.zeros((nz, nr)),
                  vturb=np.zeros((nz, nr)), h_lo=np.zeros(nr), h_hi=np.zeros(nr))
    got, ref = run_both(rt, orc, q, T, synth.chain_params(q), column=(nz != 45))
    check_chain(got, ref, f"{nr}x{nz}")


def test_surface_edge_cases(rt, orc):
    p = synth.config_small(4)
    nz, nr = p.nz, p.nr
    w = p.zr_nodes()[:, None]
    T = np.empty((nz, nr))
    T[:, :10] = 25.0 + 20.0 * w                  # warm from the midplane: h_lo = 0
    T[:, 10:20] = 8.0 + 5.0 * w                  # always frozen: h_lo = zr_max
    T[:, 20:] = 10.0 + 60.0 * w                  # crossing inside the column
    c = synth.chain_params(p)
    got, ref = run_both(rt, orc, p, T, c)
    check_chain(got, ref, "edges")
    assert np.all(got["h_lo"][:10] == 0.0) and np.all(got["h_lo"][10:20] == np.float32(p.zr_max))
    thin = synth.chain_params(p, m_gas_msun=1e-12)  # column never reaches N_dissoc: h_hi = 0
    got, ref = run_both(rt, orc, p, T, thin)
    check_chain(got, ref, "thin")
    assert np.all(got["h_hi"] == 0.0)


def test_rejects_bad_arguments(rt):
    import torch
    p = synth.config_small(0)
    T = torch.full((p.nz, p.nr), 30.0, device="cuda")
    with pytest.raises(rt.RTError):
        rt.rt_field_chain(p, T, synth.chain_params(p, gamma=2.5))
    with pytest.raises(rt.RTError):
        rt.rt_field_chain(p.replace(nz=1), torch.full((1, p.nr), 30.0, device="cuda"),
                          synth.chain_params(p))


def test_chain_then_render_matches_oracle_chain_then_render(rt, orc):
    """End to end: the density and CO layer from the chain, rendered; the oracle does both
    steps in FP64 from the same temperature grid."""
    import torch
    p = synth.config_small(5)
    c = synth.chain_params(p)
    T32 = np.ascontiguousarray(p.T, dtype=np.float32)
    out = rt.rt_field_chain(p, torch.tensor(T32, device="cuda"), c, column=False)
    dd = rt.DeviceDisk(p)
    dd.T = torch.tensor(T32, device="cuda")
    dd.n_h2, dd.h_lo, dd.h_hi = out["n_h2"], out["h_lo"], out["h_hi"]
    cube = rt.rt_render(p, dd).cpu().numpy()
    ref = orc.field_chain(p, c, T32.astype(np.float64))
    q = p.replace(T=T32.astype(np.float64), n_h2=ref["n_h2"], h_lo=ref["h_lo"], h_hi=ref["h_hi"])
    assert_cube_close(cube, orc.render(q), label="chain + render")


def adjoint_both(rt, orc, p, T, chain, gn, glo, ghi):
    import torch
    T32 = np.ascontiguousarray(T, dtype=np.float32)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda") \
        if a is not None else None
    got = rt.rt_field_chain_adjoint(p, torch.tensor(T32, device="cuda"), chain, dev(gn),
                                    dev(glo), dev(ghi))
    torch.cuda.synchronize()
    ref = orc.field_chain_adjoint(p, chain, T32.astype(np.float64), gn, glo, ghi)
    return got.cpu().numpy(), ref


def check_chain_grad(got, ref):
    """The kernel runs in FP32 with warp scans (depth 5 plus one carry per 32-node chunk, as
    in the forward chain): the exponent -I_j carries ~13 x 2^-24 |I_j| (|I_j| <= ~15 where the
    density matters), the normalisation and the column a few 1e-6, so entries above 1 % of the
    largest agree to 1e-4 relative and every entry to 1e-5 of the largest."""
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(got - ref).max() <= 1e-5 * scale
    big = np.abs(ref) >= 0.01 * scale
    assert (np.abs(got - ref)[big] / np.abs(ref)[big]).max() <= 1e-4


@pytest.mark.parametrize("which", ["all", "n", "lo", "hi"])
def test_chain_adjoint_matches_oracle(rt, orc, which):
    """The kernel (FP32) and the oracle (FP64) from the same float32 temperatures."""
    from tests.test_oracle_chain_adjoint import chain_problem
    p, rng = chain_problem(nr=37, nz=61, seed=7)
    c = synth.chain_params(p)
    nscale = orc.field_chain(p, c, p.T)["n_h2"].max()
    gn = rng.standard_normal((p.nz, p.nr)) / nscale if which in ("all", "n") else None
    glo = rng.standard_normal(p.nr) if which in ("all", "lo") else None
    ghi = rng.standard_normal(p.nr) if which in ("all", "hi") else None
    got, ref = adjoint_both(rt, orc, p, p.T, c, gn, glo, ghi)
    check_chain_grad(got, ref)


def test_chain_adjoint_observation_grid(rt, orc):
    """The 512 x 256 grid of the observation-scale workload (log radii, T over the whole
    freeze-out range)."""
    p = synth.config_observation(0)
    rng = np.random.default_rng(11)
    c = synth.chain_params(p)
    nscale = orc.field_chain(p, c, p.T)["n_h2"].max()
    got, ref = adjoint_both(rt, orc, p, p.T, c, rng.standard_normal((p.nz, p.nr)) / nscale,
                            rng.standard_normal(p.nr), rng.standard_normal(p.nr))
    check_chain_grad(got, ref)


def test_render_gradient_through_the_chain(rt, orc):
    """dL/dT of L = sum g * render(chain(T)) on the GPU (rt_field_chain, rt_render_adjoint,
    rt_field_chain_adjoint, plus the render's own dT) vs the oracle's composition of the same
    steps; the adjoint criterion of the render (3e-4 of the largest entry, 3e-3 relative
    above 1 % of it)."""
    import torch
    from tests.test_oracle_chain_adjoint import chain_problem
    p, rng = chain_problem(nr=48, nz=24, seed=9)
    p = p.replace(nx=24, ny=24, v_kms=np.linspace(-3.0, 3.0, 16), n_samples=96,
                  half_fov_au=330.0, vturb=np.full((24, 48), 0.05))
    c = synth.chain_params(p)
    T32 = np.ascontiguousarray(p.T, dtype=np.float32)
    Td = torch.tensor(T32, device="cuda")
    out = rt.rt_field_chain(p, Td, c, column=False)
    dd = rt.DeviceDisk(p)
    dd.T = Td
    dd.n_h2, dd.h_lo, dd.h_hi = out["n_h2"], out["h_lo"], out["h_hi"]
    cube = rt.rt_render(p, dd)
    g = rng.standard_normal(tuple(cube.shape)) / float(cube.abs().max())
    gd = torch.tensor(g.astype(np.float32), device="cuda")
    _, gr = rt.rt_render_adjoint(p, dd, dL_dcube=gd, cube_out=None)
    gT = gr["T"] + rt.rt_field_chain_adjoint(p, Td, c, gr["n_h2"], gr["h_lo"], gr["h_hi"])
    gT = gT.cpu().numpy()
    ref_f = orc.field_chain(p, c, T32.astype(np.float64))
    q = p.replace(T=T32.astype(np.float64), n_h2=ref_f["n_h2"], h_lo=ref_f["h_lo"],
                  h_hi=ref_f["h_hi"])
    _, rg = orc.render_adjoint(q, g.astype(np.float32).astype(np.float64))
    ref = rg["T"] + orc.field_chain_adjoint(p, c, T32.astype(np.float64), rg["n_h2"],
                                            rg["h_lo"], rg["h_hi"])
    scale = np.abs(ref).max()
    assert np.abs(gT - ref).max() <= 3e-4 * scale
    big = np.abs(ref) >= 0.01 * scale
    assert (np.abs(gT - ref)[big] / np.abs(ref)[big]).max() <= 3e-3


def test_autograd_through_the_chain(rt):
    """torch autograd over FieldChainFn and RenderFn gives the explicit composition's dL/dT."""
    import torch
    from paper_2509_03623_b300 import autograd
    from tests.test_oracle_chain_adjoint import chain_problem
    p, rng = chain_problem(nr=32, nz=16, seed=13)
    p = p.replace(nx=16, ny=16, v_kms=np.linspace(-3.0, 3.0, 8), n_samples=64,
                  half_fov_au=330.0, vturb=np.full((16, 32), 0.05))
    c = synth.chain_params(p)
    T = torch.tensor(np.ascontiguousarray(p.T, dtype=np.float32), device="cuda",
                     requires_grad=True)
    vt = torch.tensor(np.ascontiguousarray(p.vturb, dtype=np.float32), device="cuda")
    n, hlo, hhi = autograd.field_chain(p, c, T)
    cube = autograd.render(p, T, n, vt, hlo, hhi)
    g = torch.tensor(rng.standard_normal(tuple(cube.shape)).astype(np.float32),
                     device="cuda") / cube.detach().abs().max()
    (cube * g).sum().backward()
    # the explicit composition
    dd = rt.DeviceDisk(p)
    dd.T, dd.n_h2, dd.h_lo, dd.h_hi = T.detach(), n.detach(), hlo.detach(), hhi.detach()
    _, gr = rt.rt_render_adjoint(p, dd, dL_dcube=g.contiguous(), cube_out=None)
    want = gr["T"] + rt.rt_field_chain_adjoint(p, T.detach(), c, gr["n_h2"], gr["h_lo"],
                                               gr["h_hi"])
    got = T.grad.double()
    scale = float(want.abs().max())
    assert scale > 0
    assert float((got - want).abs().max()) <= 1e-5 * scale


def test_autograd_temperature_through_chain_rotation_and_render(rt, orc):
    """T -> chain -> (n_H2, surfaces) -> rotation(n_H2, T) -> render: dL/dT by torch autograd
    over the GPU steps vs the oracle's composition of its reverse modes (render with a rotation
    field, rotation, chain), on the same float32 fields; the adjoint criterion of the render."""
    import torch
    from paper_2509_03623_b300 import autograd
    from tests.test_oracle_chain_adjoint import chain_problem
    p, rng = chain_problem(nr=48, nz=24, seed=21)
    p = p.replace(nx=24, ny=24, v_kms=np.linspace(-4.0, 4.0, 16), n_samples=96,
                  half_fov_au=330.0, vturb=np.full((24, 48), 0.05))
    c = synth.chain_params(p)
    T = torch.tensor(np.ascontiguousarray(p.T, dtype=np.float32), device="cuda",
                     requires_grad=True)
    vt = torch.tensor(np.ascontiguousarray(p.vturb, dtype=np.float32), device="cuda")
    n, hlo, hhi = autograd.field_chain(p, c, T)
    vphi = autograd.pressure_vphi(p, n, T)
    cube = autograd.render(p, T, n, vt, hlo, hhi, vphi=vphi)
    g = rng.standard_normal(tuple(cube.shape)) / float(cube.detach().abs().max())
    gd = torch.tensor(g.astype(np.float32), device="cuda")
    (cube * gd).sum().backward()
    got = T.grad.double().cpu().numpy()
    # the oracle's composition from the same float32 intermediate fields
    T64 = p.T.astype(np.float32).astype(np.float64)
    f = orc.field_chain(p, c, T64)
    n32 = n.detach().cpu().numpy().astype(np.float64)
    v32 = vphi.detach().cpu().numpy().astype(np.float64)
    q = p.replace(T=T64, n_h2=n32, h_lo=hlo.detach().cpu().numpy().astype(np.float64),
                  h_hi=hhi.detach().cpu().numpy().astype(np.float64), vphi=v32)
    _, rg = orc.render_adjoint_vphi(q, g.astype(np.float32).astype(np.float64))
    gn_rot, gT_rot = orc.pressure_vphi_adjoint(p, rg["vphi"], n32, T64)
    ref = rg["T"] + gT_rot + orc.field_chain_adjoint(p, c, T64, rg["n_h2"] + gn_rot,
                                                    rg["h_lo"], rg["h_hi"])
    assert np.all(np.abs(f["n_h2"] - n32) <= 1e-4 * np.abs(f["n_h2"]).max())
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 3e-4 * scale
    big = np.abs(ref) >= 0.01 * scale
    assert (np.abs(got - ref)[big] / np.abs(ref)[big]).max() <= 3e-3
