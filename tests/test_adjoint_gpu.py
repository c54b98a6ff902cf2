"""Fused CUDA adjoint vs the FP64 oracle's reverse mode and vs central finite differences of
the oracle's forward march (through the C ABI)."""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.cubecheck import assert_cube_close
from tests.test_forward_gpu import rt  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu

FIELDS = ("T", "n_h2", "vturb", "h_lo", "h_hi")


def grad_errors(got, ref):
    """Per field: max |got - ref| / max |ref| and max relative error on entries >= 1% of max
    (the five node fields, and the rotation field where both sides have it)."""
    out = {}
    for k in FIELDS + (("vphi",) if "vphi" in got and "vphi" in ref else ()):
        g, r = np.asarray(got[k]), np.asarray(ref[k])
        m = np.abs(r).max()
        if m == 0:
            out[k] = (float(np.abs(g).max()), 0.0)
            continue
        big = np.abs(r) >= 1e-2 * m
        out[k] = (float(np.abs(g - r).max() / m), float((np.abs(g - r)[big] / np.abs(r[big])).max()))
    return out


def assert_grads_close(got, ref, atol=3e-4, rtol=3e-3, label=""):
    e = grad_errors(got, ref)
    for k, (a, r) in e.items():
        assert a <= atol and r <= rtol, f"{label} {k}: scaled err {a:.2e}, rel err {r:.2e} ({e})"
    return e


def to_np(g):
    return {k: g[k].cpu().numpy() for k in FIELDS}


def loss_target(orc, p, seed):
    """Sum-of-squares target: the oracle cube of the seed+1 disk plus 5% noise."""
    q = synth.config_small(seed + 1).replace(nx=p.nx, ny=p.ny, v_kms=p.v_kms,
                                             n_samples=p.n_samples)
    return synth.noisy_target(orc.render(q), seed + 2)


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_vs_oracle_adjoint(rt, orc, seed):
    """64x32 grid, 64^2 px, 16 channels, 128 samples; seed dL/dcube = 2 (I - I*)."""
    import torch
    p = synth.config_small(seed)
    ref_cube = orc.render(p)
    tgt = loss_target(orc, p, seed)
    dL = 2.0 * (ref_cube - tgt)
    _, g_ref = orc.render_adjoint(p, dL)
    cube, g = rt.rt_render_adjoint(p, dL_dcube=torch.tensor(dL, dtype=torch.float32,
                                                            device="cuda"))
    torch.cuda.synchronize()
    e = assert_grads_close(to_np(g), g_ref, label=f"seed {seed}")
    print(f"adjoint seed {seed}: {e}")
    # the adjoint's own forward pass and the forward kernel are two FP32 evaluations of the
    # same march (different lane layouts and operation order): both are held to the parity
    # criterion against the oracle, and to it against each other
    fwd = rt.rt_render(p).cpu().numpy()
    assert_cube_close(cube.cpu().numpy(), fwd, label="adjoint cube vs forward")
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="adjoint cube vs oracle")


def test_fused_loss_target_mode(rt, orc):
    import torch
    p = synth.config_small(3)
    tgt = loss_target(orc, p, 3)
    tgt_t = torch.tensor(tgt, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render_adjoint(p, target=tgt_t)
    torch.cuda.synchronize()
    c = cube.double().cpu().numpy()
    loss = float(((c - tgt.astype(np.float32).astype(np.float64)) ** 2).sum())
    assert float(g["loss"].item()) == pytest.approx(loss, rel=1e-5)
    _, g_ref = orc.render_adjoint(p, 2.0 * (orc.render(p) - tgt))
    assert_grads_close(to_np(g), g_ref, label="target mode")


@pytest.mark.parametrize("case", [
    dict(nx=29, ny=21, v_kms=np.linspace(-3.1, 4.0, 13), n_samples=100),  # ragged, partial seg
    dict(v_kms=np.linspace(-4, 4, 40), n_samples=200),                    # 16 lanes per ray
    dict(v_kms=np.array([-3.0, -0.3, 0.2, 0.25, 2.7]), n_samples=64),     # unequal, 2 lanes
    dict(v_kms=np.linspace(-5, 5, 128), nx=24, ny=24, n_samples=96),      # 32 lanes per ray
    dict(incl_deg=0.0, units=1, I0=0.02),                                 # face-on, Jy, I0
    dict(n_samples=1),
])
def test_adjoint_variants(rt, orc, case):
    import torch
    p = synth.config_small(21).replace(**case)
    rng = np.random.default_rng(4)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    _, g_ref = orc.render_adjoint(p, w)
    _, g = rt.rt_render_adjoint(p, dL_dcube=torch.tensor(w, dtype=torch.float32, device="cuda"),
                                cube_out=None)
    torch.cuda.synchronize()
    e = assert_grads_close(to_np(g), g_ref, label=str(list(case)))
    print(f"adjoint variant {list(case)}: {e}")


def test_adjoint_mach_mode_and_hard_edges(rt, orc):
    import torch
    p = synth.config_small(22)
    p = p.replace(vturb_mach=1, vturb=np.full_like(p.vturb, 0.3))
    rng = np.random.default_rng(5)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    _, g_ref = orc.render_adjoint(p, w)
    _, g = rt.rt_render_adjoint(p, dL_dcube=torch.tensor(w, dtype=torch.float32, device="cuda"))
    assert_grads_close(to_np(g), g_ref, label="mach")
    q = synth.config_small(23).replace(edge_w=0.0)
    _, g = rt.rt_render_adjoint(q, dL_dcube=torch.tensor(w, dtype=torch.float32, device="cuda"))
    assert float(g["h_lo"].abs().max()) == 0.0 and float(g["h_hi"].abs().max()) == 0.0


def test_adjoint_vs_central_differences(rt, orc):
    """32 random cells of T, n_H2, v_turb (|g| >= 2% of the field's largest) plus the four
    surface power-law parameters: GPU adjoint vs central differences (step 1e-3 relative) of
    the FP64 oracle's loss sum (I - I*)^2."""
    import torch
    p = synth.config_small(5)
    tgt = loss_target(orc, p, 5)

    def loss(q):
        return float(((orc.render(q) - tgt) ** 2).sum())

    tgt_t = torch.tensor(tgt, dtype=torch.float32, device="cuda")
    _, g = rt.rt_render_adjoint(p, target=tgt_t, cube_out=None)
    g = to_np(g)
    rng = np.random.default_rng(11)
    checked = 0
    for field, ncell in (("T", 12), ("n_h2", 12), ("vturb", 8)):
        flat = np.abs(g[field]).ravel()
        cand = np.flatnonzero(flat >= 0.02 * flat.max())
        for idx in rng.choice(cand, size=ncell, replace=False):
            arr = getattr(p, field)
            h = 1e-3 * abs(arr.flat[idx])
            a, b = arr.copy(), arr.copy()
            a.flat[idx] += h
            b.flat[idx] -= h
            fd = (loss(p.replace(**{field: a})) - loss(p.replace(**{field: b}))) / (2 * h)
            assert fd == pytest.approx(g[field].flat[idx], rel=3e-3), (field, int(idx))
            checked += 1
    assert checked == 32
    # surface power-law parameters (c, p) of both surfaces through rt_surface_powerlaw_grad
    r = p.r_nodes()
    c_lo, p_lo, c_hi, p_hi = p.surf
    dlo = rt.rt_surface_powerlaw_grad(p, torch.tensor(g["h_lo"], device="cuda"),
                                      torch.tensor(p.h_lo, device="cuda"), c_lo).cpu().numpy()
    dhi = rt.rt_surface_powerlaw_grad(p, torch.tensor(g["h_hi"], device="cuda"),
                                      torch.tensor(p.h_hi, device="cuda"), c_hi).cpu().numpy()

    def with_surf(cl, pl, ch, ph_):
        lo, hi = synth.surfaces(r, cl, pl, ch, ph_)
        return p.replace(h_lo=lo, h_hi=hi)

    d = 1e-3
    fd = [
        (loss(with_surf(c_lo * (1 + d), p_lo, c_hi, p_hi))
         - loss(with_surf(c_lo * (1 - d), p_lo, c_hi, p_hi))) / (2 * d * c_lo),
        (loss(with_surf(c_lo, p_lo + d, c_hi, p_hi)) - loss(with_surf(c_lo, p_lo - d, c_hi, p_hi)))
        / (2 * d),
        (loss(with_surf(c_lo, p_lo, c_hi * (1 + d), p_hi))
         - loss(with_surf(c_lo, p_lo, c_hi * (1 - d), p_hi))) / (2 * d * c_hi),
        (loss(with_surf(c_lo, p_lo, c_hi, p_hi + d)) - loss(with_surf(c_lo, p_lo, c_hi, p_hi - d)))
        / (2 * d),
    ]
    got = [dlo[0], dlo[1], dhi[0], dhi[1]]
    for a, b in zip(got, fd):
        assert a == pytest.approx(b, rel=3e-3)


def test_autograd_function(rt, orc):
    import torch
    from paper_2509_03623_b300 import autograd
    p = synth.config_small(6)
    dd = rt.DeviceDisk(p)
    ts = [t.clone().requires_grad_(True) for t in dd.tensors()]
    tgt = torch.tensor(loss_target(orc, p, 6), dtype=torch.float32, device="cuda")
    cube = autograd.render(p, *ts)
    loss = ((cube.double() - tgt.double()) ** 2).sum()
    loss.backward()
    _, g = rt.rt_render_adjoint(p, dd, target=tgt, cube_out=None)
    for t, k in zip(ts, FIELDS):
        ref = g[k].float()
        scale = float(ref.abs().max())
        assert float((t.grad - ref).abs().max()) <= 1e-3 * scale + 1e-30, k
    assert loss.item() == pytest.approx(float(g["loss"].item()), rel=1e-5)


def test_adjoint_corner_quads_vs_oracle(rt, orc):
    """The fused adjoint at 4.19 M samples (512x256 grid, 128^2 px, 256 samples, the 64
    channels of the observation workload) reads its fields from packed corner quads in all
    three passes; gradients vs the oracle under a random-sign seed."""
    import torch
    p = synth.config_observation(4).replace(nx=128, ny=128, n_samples=256)
    assert p.nx * p.ny * p.n_samples >= 1 << 22
    rng = np.random.default_rng(4)
    dL = rng.standard_normal((p.nch, p.ny, p.nx))
    ref_cube, g_ref = orc.render_adjoint(p, dL)
    cube, g = rt.rt_render_adjoint(p, dL_dcube=torch.tensor(dL, dtype=torch.float32,
                                                            device="cuda"))
    torch.cuda.synchronize()
    e = assert_grads_close(to_np(g), g_ref, label="corner quads")
    print(f"adjoint corner quads: {e}")
    assert_cube_close(cube.cpu().numpy(), ref_cube, label="adjoint cube (corner quads)")


def test_adjoint_work_counters(rt, orc):
    """rt_render_adjoint_work returns the results of rt_render_adjoint and counts its work:
    the samples with gas equal the forward march's count, the forward and reverse passes
    evaluate the same channel blocks, and nothing is recomputed between them."""
    import torch
    p = synth.config_small(8).replace(v_kms=np.linspace(-4, 4, 48))
    dd = rt.DeviceDisk(p)
    tgt = torch.tensor(loss_target(orc, p, 8), dtype=torch.float32, device="cuda")
    cube0, g0 = rt.rt_render_adjoint(p, dd, target=tgt)
    work = torch.zeros(4, dtype=torch.int64, device="cuda")
    cube1, g1 = rt.rt_render_adjoint(p, dd, target=tgt, work=work)
    _, phys, computed = rt.rt_render_work(p, dd)
    torch.cuda.synchronize()
    w = [int(x) for x in work.cpu()]
    assert np.array_equal(cube0.cpu().numpy(), cube1.cpu().numpy())
    assert_grads_close(to_np(g1), to_np(g0), atol=1e-6, rtol=1e-5, label="with counters")
    assert w[0] == phys > 0
    assert w[1] == w[3] > 0 and w[2] == 0
    assert w[1] <= p.nx * p.ny * p.n_samples * 64   # at most the dense count (64 = padded lanes)
    print(f"adjoint work {w}; forward march: {phys} samples, {computed} evaluations")


def edge_rays(orc, p, tol=1e-6):
    """[ny][nx] mask of the rays with a sample within `tol` (relative) of a hard edge of the
    gas: the wedge |z|/r = zr_max or the inner radius r = r_in."""
    ks = np.arange(p.n_samples) + 0.5
    out = np.zeros((p.ny, p.nx), dtype=bool)
    for iy in range(p.ny):
        for ix in range(p.nx):
            hit, s0, s1, P0, om = orc.ray(p, ix, iy)
            if not hit:
                continue
            s = s0 + ks * (s1 - s0) / p.n_samples
            x, y, z = (P0[a] + s * om[a] for a in range(3))
            r = np.hypot(x, y)
            zr = np.abs(z) / np.maximum(r, 1e-300)
            out[iy, ix] = bool(np.any(np.abs(zr - p.zr_max) <= tol * p.zr_max)
                               or np.any(np.abs(r - p.r_in_au) <= tol * p.r_in_au))
    return out


def test_adjoint_observation_workload(rt, orc):
    """The benchmark's forward+adjoint workload at full size (512x256 grid, 256^2 px, 64
    channels, 512 samples; the specialised 8-lanes x 8-channels kernel with corner quads, in
    the launch configuration the benchmark times), every gradient entry against the oracle's
    reverse mode. The seed is the benchmark's loss gradient 2 (cube - 1.05 cube) = -0.1 cube
    (at the oracle's cube), given to both sides. The gas ends at hard edges (|z|/r = zr_max,
    r = r_in): a sample within FP32 rounding of one may fall on the other side (the
    flip-tolerant reading of hard edges), which moves its ray by about 1/N_s and the gradient
    of a node of the wedge's thin top cell by about 1e-3, so those rays (0.25 % of the
    image) get a zero seed and stay out of the cube comparison."""
    import torch
    p = synth.config_observation(0)
    ref_cube = orc.render(p)
    keep = ~edge_rays(orc, p)
    assert keep.mean() > 0.99
    seed = -0.1 * ref_cube * keep[None]
    _, ref = orc.render_adjoint(p, seed)
    dl = torch.tensor(seed, dtype=torch.float32, device="cuda")
    cube, g = rt.rt_render_adjoint(p, dL_dcube=dl)
    torch.cuda.synchronize()
    got = cube.cpu().numpy()
    assert_cube_close(got[:, keep], ref_cube[:, keep], label="observation adjoint cube")
    e = assert_grads_close(to_np(g), ref, label="observation workload")
    print(f"observation workload adjoint: {e}")
