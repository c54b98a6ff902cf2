"""Pins of the FP64 oracle against closed forms, invariants, textbook limits and brute-force
quadrature (no GPU). Each test is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a unit factor) fails at least one.
"""

import math

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests import physics as ph


def uniform_problem(T=40.0, n=1e6, vt=0.1, *, nx=2, ny=1, hf=600.0, incl=90.0, pa=0.0,
                    mstar=0.0, v=(0.0,), ns=64, I0=0.0, zr_max=0.5, nr=8, nz=4, edge_w=0.0,
                    hlo=-1.0, hhi=10.0, units=0, dist=100.0):
    shape = (nz, nr)
    return synth.Problem(
        nr=nr, nz=nz, r_in_au=10.0, r_out_au=600.0, zr_max=zr_max, r_log=1,
        T=np.full(shape, T), n_h2=np.full(shape, n), vturb=np.full(shape, vt),
        h_lo=np.full(nr, hlo), h_hi=np.full(nr, hhi), edge_w=edge_w, incl_deg=incl,
        pa_deg=pa, mstar_msun=mstar, nx=nx, ny=ny, half_fov_au=hf,
        v_kms=np.asarray(v, dtype=float), n_samples=ns, I0=I0, units=units, dist_pc=dist)


# --------------------------------------------------------------------------------------
# P1 uniform slab: I = S (1 - e^-tau) + I0 e^-tau, exact for any number of samples
# --------------------------------------------------------------------------------------

def test_p1_uniform_slab_exact_any_ns(orc):
    # Edge-on midplane rays at x = +-300 au along y: gas everywhere on the chord.
    vals = [orc.render(uniform_problem(ns=ns))[0, 0, :] for ns in (1, 7, 64, 333)]
    for v in vals[1:]:
        np.testing.assert_allclose(v, vals[0], rtol=1e-12)
    assert vals[0][0] > 0


def test_p1_slab_source_is_planck_and_background_attenuation(orc):
    T = 37.0
    I_a = orc.render(uniform_problem(T=T, n=4e3, I0=0.0))[0, 0, 0]
    Ib = 2.5e-13
    I_b = orc.render(uniform_problem(T=T, n=4e3, I0=Ib))[0, 0, 0]
    trans = (I_b - I_a) / Ib
    assert 0.01 < trans < 0.99  # moderate optical depth: both terms matter
    S = I_a / (1.0 - trans)
    assert S == pytest.approx(ph.planck_nu(synth.CO21_NU0, T), rel=1e-11)


def test_p1_tau_linear_in_chord_and_density(orc):
    def tau(**kw):
        I0 = 1e-12
        a = orc.render(uniform_problem(I0=0.0, **kw))[0, 0, 0]
        b = orc.render(uniform_problem(I0=I0, **kw))[0, 0, 0]
        return -math.log((b - a) / I0)
    t300 = tau(n=2e3, hf=600.0)   # ray at x=300 au: chord 2 sqrt(600^2-300^2)
    t400 = tau(n=2e3, hf=800.0)   # ray at x=400 au
    assert t300 / t400 == pytest.approx(math.sqrt(600**2 - 300**2) / math.sqrt(600**2 - 400**2),
                                        rel=1e-10)
    assert tau(n=4e3, hf=600.0) / t300 == pytest.approx(2.0, rel=1e-10)


# --------------------------------------------------------------------------------------
# P6 optically thick isothermal: I -> B_nu0(T); P8 LTE identity j / beta = B_nu0(T)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("T", [8.0, 20.0, 65.0, 300.0])
def test_p6_thick_isothermal_planck(orc, T):
    I = orc.render(uniform_problem(T=T, n=1e12))[0, 0, 0]
    assert I == pytest.approx(ph.planck_nu(synth.CO21_NU0, T), rel=1e-12)


@pytest.mark.parametrize("T", [5.0, 19.0, 44.4, 150.0, 900.0])
def test_p8_lte_source_function(orc, T):
    p = uniform_problem(T=T, incl=30.0, mstar=1.0)
    d = orc.point(p, 120.0, 40.0, 3.0, 0.7)
    assert d["gas"]
    if d["beta"] > 1e-200:
        assert d["j"] / d["beta"] == pytest.approx(ph.planck_nu(synth.CO21_NU0, T), rel=1e-12)
    assert d["S"] == pytest.approx(ph.planck_nu(synth.CO21_NU0, T), rel=1e-12)


def test_p8_rayleigh_jeans_limit(orc):
    T = 2.0e4  # h nu / k T = 5.5e-4
    d = orc.point(uniform_problem(T=T), 100.0, 0.0, 1.0, 0.0)
    assert d["S"] == pytest.approx(ph.rayleigh_jeans(synth.CO21_NU0, T), rel=3e-4)


# --------------------------------------------------------------------------------------
# LTE populations: rigid-rotor partition function limits
# --------------------------------------------------------------------------------------

def test_partition_function_limits(orc):
    B = synth.CO21_NU0 / 4.0
    for T in (300.0, 1000.0, 3000.0):
        assert orc.partition(T, B) == pytest.approx(ph.rotor_Z_high_T(T, B), rel=2e-9)
    for T in (0.5, 1.0, 2.0):
        assert orc.partition(T, B) == pytest.approx(ph.rotor_Z_low_T(T, B, jmax=4), rel=1e-12)


def test_boltzmann_level_ratio(orc):
    # n_u / n_l = (g_u/g_l) exp(-h nu0 / kT) for a rigid rotor with B = nu0 / (2 J_u)
    T = 23.0
    d = orc.point(uniform_problem(T=T), 100.0, 0.0, 1.0, 0.0)
    ratio = 5.0 / 3.0 * math.exp(-ph.H * synth.CO21_NU0 / (ph.K * T))
    assert d["n_u"] / d["n_l"] == pytest.approx(ratio, rel=1e-12)
    Z = orc.partition(T, synth.CO21_NU0 / 4.0)
    n_co = 1e-4 * 1e6
    assert d["n_l"] == pytest.approx(n_co * 3.0 * math.exp(-2 * ph.H * synth.CO21_NU0 / 4 /
                                                         (ph.K * T)) / Z, rel=1e-12)


# --------------------------------------------------------------------------------------
# P7 profile: normalisation, centre (Doppler sign) and width
# --------------------------------------------------------------------------------------

def test_p7_profile_normalisation_centre_width(orc):
    p = uniform_problem(T=30.0, vt=0.2, incl=60.0, mstar=2.0)
    x, y, z = 150.0, 0.0, 0.0
    base = orc.point(p, x, y, z, 0.0)
    vlos, alpha = base["v_los_kms"], base["alpha_kms"]
    # receding side: x > 0 on the redshifted major axis, v_los = v_K sin i
    assert vlos == pytest.approx(ph.kepler_speed_kms(2.0, 150.0) * math.sin(math.radians(60)),
                                 rel=1e-12)
    assert alpha == pytest.approx(math.sqrt(2 * ph.K * 30.0 / (28.0101 * ph.AMU) / 1e10
                                            + 0.2 ** 2), rel=1e-12)
    vs = np.linspace(vlos - 12 * alpha, vlos + 12 * alpha, 801)
    phis = np.array([orc.point(p, x, y, z, v)["phi"] for v in vs])
    dnu = synth.CO21_NU0 * (vs[1] - vs[0]) * 1e5 / ph.C
    assert phis.sum() * dnu == pytest.approx(1.0, rel=1e-10)
    assert vs[np.argmax(phis)] == pytest.approx(vlos, abs=(vs[1] - vs[0]))
    pk = orc.point(p, x, y, z, vlos)["phi"]
    assert orc.point(p, x, y, z, vlos + alpha)["phi"] / pk == pytest.approx(math.exp(-1), rel=1e-9)
    assert pk == pytest.approx(ph.C / (synth.CO21_NU0 * alpha * 1e5 * math.sqrt(math.pi)),
                               rel=1e-9)


@pytest.mark.parametrize("T", [25.0, 80.0])
def test_p7_mach_mode_line_width_from_the_spectrum(orc, T):
    """Mach-mode line width (Methods, the alpha(x) and c_s equations): the turbulent speed is
    a Mach number times c_s with c_s^2 = 2kT/m_mol as printed, so
    alpha^2 = 2kT/m_CO + M^2 2kT/m_mol with m_CO = 28.0101 amu and m_mol = 2.37 m_H
    (m_H = 1.007825 amu). Measured from the rendered spectrum of an optically thin, static,
    isothermal slab: its line is the Gaussian exp(-v^2/alpha^2), whose second moment over a
    fine channel grid is alpha^2/2. Two temperatures and three Mach numbers fix both terms:
    a dropped factor 2 in c_s^2, the two masses swapped, or M entering linearly all fail."""
    m_co = 28.0101 * ph.AMU
    m_mol = 2.37 * 1.007825 * ph.AMU
    for M in (0.0, 0.5, 2.0):
        expect = (2 * ph.K * T / m_co + M * M * 2 * ph.K * T / m_mol) / 1e10   # km^2 s^-2
        a = math.sqrt(expect)
        v = np.linspace(-7 * a, 7 * a, 701)
        p = uniform_problem(T=T, n=1e-3, vt=M, v=v, ns=8)
        p = p.replace(vturb_mach=1)
        spec = orc.render(p)[:, 0, 0]
        assert spec.max() > 0
        m2 = float((v * v * spec).sum() / spec.sum())
        assert 2.0 * m2 == pytest.approx(expect, rel=1e-6), (T, M)
        # the same width at the sample itself
        assert orc.point(p, 300.0, 0.0, 0.0, 0.0)["alpha_kms"] ** 2 == pytest.approx(expect,
                                                                                    rel=1e-12)


def test_kepler_height_dependence(orc):
    p = uniform_problem(incl=90.0, mstar=1.0)
    v0 = orc.point(p, 200.0, 0.0, 0.0, 0.0)["v_los_kms"]
    v1 = orc.point(p, 200.0, 0.0, 60.0, 0.0)["v_los_kms"]
    # v_phi^2 / r = G M r / (r^2+z^2)^{3/2}  =>  v(z)/v(0) = (1 + z^2/r^2)^{-3/4}
    assert v1 / v0 == pytest.approx((1 + (60 / 200) ** 2) ** -0.75, rel=1e-12)
    # approaching side
    assert orc.point(p, -200.0, 0.0, 0.0, 0.0)["v_los_kms"] == pytest.approx(-v0, rel=1e-14)


# --------------------------------------------------------------------------------------
# P3 face-on symmetry, P4 inclined mirror symmetry, P5 PA rotation
# --------------------------------------------------------------------------------------

def test_p3_face_on_symmetry(orc):
    p = synth.config_small(3).replace(incl_deg=0.0, nx=24, ny=24, n_samples=48)
    cube = orc.render(p)
    assert cube.max() > 0
    # The profile is evaluated in frequency space as printed (nu_c - nu0(1 - dnu)), which
    # carries ~1e-9 relative rounding in the line wings even in FP64.
    tol = dict(rtol=1e-8, atol=1e-12 * cube.max())
    np.testing.assert_allclose(cube, cube[::-1], **tol)   # spectrum
    np.testing.assert_allclose(cube, cube.transpose(0, 2, 1), rtol=1e-14, atol=0)
    np.testing.assert_allclose(cube, cube[:, ::-1, :], rtol=1e-14, atol=0)
    np.testing.assert_allclose(cube, cube[:, :, ::-1], rtol=1e-14, atol=0)


def test_p4_inclined_mirror_symmetry(orc):
    p = synth.config_small(4).replace(nx=20, ny=16, n_samples=40, v_kms=np.linspace(-3, 3, 9))
    cube = orc.render(p)
    np.testing.assert_allclose(cube, cube[::-1, :, ::-1], rtol=1e-8, atol=1e-12 * cube.max())
    # and the disk is not face-on: the cube is not symmetric in velocity alone
    assert np.abs(cube - cube[::-1]).max() > 1e-3 * cube.max()


def test_p5_position_angle_rotation(orc):
    p = synth.config_small(5).replace(nx=18, ny=18, n_samples=40, v_kms=np.array([-1.0, 0.4]))
    a = orc.render(p.replace(pa_deg=0.0))
    b = orc.render(p.replace(pa_deg=90.0))
    n = p.nx
    ix = np.arange(n)
    # I_90(X, Y) = I_0(Y, -X): b[:, iy, ix] = a[:, n-1-ix, iy]
    expect = a[:, n - 1 - ix[None, :], ix[:, None]]
    np.testing.assert_allclose(b, expect, rtol=1e-9, atol=1e-12 * a.max())


# --------------------------------------------------------------------------------------
# P2 optically thin limit
# --------------------------------------------------------------------------------------

def test_p2_thin_limit_sum_j_ds(orc):
    p = synth.config_small(1).replace(nx=8, ny=8, n_samples=64)
    p = p.replace(n_h2=p.n_h2 * 1e-12)
    pix = np.array([3 * 8 + 4, 4 * 8 + 4, 2 * 8 + 6])
    spec = orc.render_pixels(p, pix)
    for k, q in enumerate(pix):
        ix, iy = int(q % 8), int(q // 8)
        hit, s0, s1, P0, om = orc.ray(p, ix, iy)
        assert hit
        ds = (s1 - s0) / p.n_samples
        for c, v in enumerate(p.v_kms):
            jsum, tau = 0.0, 0.0
            for i in range(p.n_samples):
                s = s0 + (i + 0.5) * ds
                d = orc.point(p, *(P0 + s * om), v)
                jsum += d["j"] * ds * ph.AU
                tau += d["beta"] * ds * ph.AU
            if jsum < 1e-250:  # far line wing: products underflow to denormals
                assert spec[k, c] < 1e-250
                continue
            assert tau < 1e-6
            # I = sum_k e^{-tau_k} S (1 - e^{-dtau_k}) = sum_k j_k ds (1 - O(tau))
            dev = spec[k, c] / jsum - 1.0
            assert -tau - 1e-12 <= dev <= 1e-12


# --------------------------------------------------------------------------------------
# P9 thin-limit flux conservation: image-integrated line flux = volume emission
# --------------------------------------------------------------------------------------

def test_p9_flux_conservation(orc):
    # Constant T, n in a wedge h_lo <= z/r <= h_hi (hard edges), face-on, tiny density:
    # sum_pix sum_ch I dnu dA = (h nu0 / 4 pi) n_u A_ul V, V = (4 pi / 3)(h_hi-h_lo)(r_out^3 - r_in^3)
    T, n, hlo, hhi = 80.0, 1e-6, 0.05, 0.2
    p = uniform_problem(T=T, n=n, vt=0.3, incl=0.0, mstar=0.5, nx=96, ny=96, hf=600.0,
                        ns=512, hlo=hlo, hhi=hhi, v=np.linspace(-2.0, 2.0, 61))
    cube = orc.render(p)
    dv = p.v_kms[1] - p.v_kms[0]
    dnu = synth.CO21_NU0 * dv * 1e5 / ph.C
    dA = (2 * 600.0 / 96 * ph.AU) ** 2
    flux = cube.sum() * dnu * dA
    B = synth.CO21_NU0 / 4.0
    Z = orc.partition(T, B)
    nu_ = 1e-4 * n * 5.0 * math.exp(-ph.H * B * 6 / (ph.K * T)) / Z
    V = 4 * math.pi / 3 * (hhi - hlo) * (600.0 ** 3 - 10.0 ** 3) * ph.AU ** 3
    expect = ph.H * synth.CO21_NU0 / (4 * math.pi) * nu_ * p.A_ul * V
    # face-on: the line is unshifted; the residual is the sky-plane and z quadrature of a
    # body with sharp edges (pixel ~ 12.5 au, ds ~ 1.2 au)
    assert flux == pytest.approx(expect, rel=2e-2)
    # refining the image grid moves the sum toward the volume integral
    p2 = p.replace(nx=192, ny=192)
    flux2 = orc.render(p2).sum() * dnu * (2 * 600.0 / 192 * ph.AU) ** 2
    assert abs(flux2 / expect - 1) < abs(flux / expect - 1)
    assert flux2 == pytest.approx(expect, rel=1e-2)


# --------------------------------------------------------------------------------------
# P10 brute-force quadrature of Eq. rt-int on a tiny smooth grid
# --------------------------------------------------------------------------------------

def test_p10_quadrature_convergence(orc):
    """The midpoint march converges to an independent fine quadrature of Eq. rt-int (nested
    trapezoid rules for tau(s) and the emission integral) along the exact ray."""
    from scipy import integrate
    p = synth.disk(7, nr=8, nz=4, nx=6, ny=6, nch=3, vmax=1.0, n_samples=64, incl=50.0,
                   pa=20.0)
    # moderate optical depth and a broad line so that the integrand is resolved
    p = p.replace(vturb=np.full_like(p.vturb, 0.4), n_h2=p.n_h2 * 2e-3)
    c, iy, ix = 0, 3, 2
    hit, s0, s1, P0, om = orc.ray(p, ix, iy)
    assert hit
    v = p.v_kms[c]
    ss = np.linspace(s0, s1, 40001)
    pts = [orc.point(p, *(P0 + s * om), v) for s in ss]
    bb = np.array([d["beta"] for d in pts]) * ph.AU
    jj = np.array([d["j"] for d in pts]) * ph.AU
    tau = integrate.cumulative_trapezoid(bb, ss, initial=0.0)
    I_ref = integrate.trapezoid(jj * np.exp(-tau), ss)
    assert 0.5 < tau[-1] < 5.0 and I_ref > 0
    pixel = iy * p.nx + ix
    errs = {}
    for ns in (32, 128, 1024, 4096):
        I = orc.render_pixels(p.replace(n_samples=ns), [pixel])[0, c]
        errs[ns] = abs(I - I_ref) / I_ref
    assert errs[4096] < 1e-5 and errs[1024] < 1e-4
    assert errs[4096] < errs[1024] < errs[128] < errs[32]


# --------------------------------------------------------------------------------------
# Units: Jy per pixel
# --------------------------------------------------------------------------------------

def test_units_jy_per_pixel(orc):
    p = synth.config_small(2).replace(nx=10, ny=10, n_samples=32)
    a = orc.render(p)
    b = orc.render(p.replace(units=1))
    pix_au = 2 * 1.1 * 600.0 / 10
    np.testing.assert_allclose(b, a * ph.pixel_solid_angle(pix_au, p.dist_pc) * 1e23,
                               rtol=1e-12, atol=1e-15 * b.max())


# --------------------------------------------------------------------------------------
# Geometry: chord and misses
# --------------------------------------------------------------------------------------

def test_chord_and_miss(orc):
    p = uniform_problem(incl=90.0, nx=2, ny=1, hf=600.0)
    hit, s0, s1, P0, om = orc.ray(p, 1, 0)
    assert hit and s1 - s0 == pytest.approx(2 * math.sqrt(600 ** 2 - 300 ** 2), rel=1e-13)
    # face-on ray outside r_out misses and returns the background
    q = uniform_problem(incl=0.0, nx=2, ny=2, hf=1000.0, I0=3e-14)   # pixels at r = 707 au
    assert not orc.ray(q, 0, 0)[0]
    np.testing.assert_allclose(orc.render(q), 3e-14, rtol=0)
    # face-on chord through the slab |z| <= zr_max r_out
    r = uniform_problem(incl=0.0, nx=2, ny=2, hf=400.0)
    hit, s0, s1, _, _ = orc.ray(r, 0, 0)
    assert hit and s1 - s0 == pytest.approx(2 * 0.5 * 600.0, rel=1e-13)


# --------------------------------------------------------------------------------------
# P12 neural field vs a library routine (torch fp64 Sequential)
# --------------------------------------------------------------------------------------

def test_p12_mlp_matches_torch(orc):
    torch = pytest.importorskip("torch")
    w = synth.mlp_weights(11)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, size=(257, 2))
    out = orc.mlp_eval(w, x)
    layers = []
    for l, (W, b) in enumerate(zip(w.W, w.b)):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W.astype(np.float64)))
            lin.bias.copy_(torch.from_numpy(b.astype(np.float64)))
        layers.append(lin)
        if l < len(w.W) - 1:
            layers.append(torch.nn.SiLU())
    net = torch.nn.Sequential(*layers)
    xt = torch.from_numpy(x)
    Bt = torch.from_numpy(w.B.astype(np.float64))
    proj = 2 * math.pi * xt @ Bt.T
    feats = torch.cat([torch.sin(proj), torch.cos(proj)], dim=1)
    ref = net(feats).detach().numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-13)


def test_p12_mlp_gradients_match_torch_autograd(orc):
    """Reverse mode of the oracle network vs torch FP64 autograd of the same Sequential."""
    torch = pytest.importorskip("torch")
    w = synth.mlp_weights(12)
    rng = np.random.default_rng(1)
    w.b = [rng.uniform(-0.1, 0.1, size=b.shape) for b in w.b]
    x = rng.uniform(0, 1, size=(93, 2))
    gout = rng.standard_normal((93, 4))
    dW, db = orc.mlp_grad(w, x, gout)
    layers = []
    for l, (W, b) in enumerate(zip(w.W, w.b)):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(np.asarray(W, dtype=np.float64)))
            lin.bias.copy_(torch.from_numpy(np.asarray(b, dtype=np.float64)))
        layers.append(lin)
        if l < len(w.W) - 1:
            layers.append(torch.nn.SiLU())
    net = torch.nn.Sequential(*layers)
    proj = 2 * math.pi * torch.from_numpy(x) @ torch.from_numpy(w.B.astype(np.float64)).T
    feats = torch.cat([torch.sin(proj), torch.cos(proj)], dim=1)
    (net(feats) * torch.from_numpy(gout)).sum().backward()
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for l, lin in enumerate(lins):
        np.testing.assert_allclose(dW[l], lin.weight.grad.numpy(), rtol=1e-11,
                                   atol=1e-13 * np.abs(dW[l]).max(), err_msg=f"W{l}")
        np.testing.assert_allclose(db[l], lin.bias.grad.numpy(), rtol=1e-11,
                                   atol=1e-13 * np.abs(db[l]).max(), err_msg=f"b{l}")


def test_mlp_render_zero_network_equals_grid_render(orc):
    p = synth.config_small(6).replace(nx=12, ny=12, n_samples=40)
    w = synth.mlp_weights(1, width=16, hidden=2)
    w.W[-1][:] = 0.0
    a = orc.render(p)
    b = orc.render_mlp(p, w)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=0)
    # a constant log-T offset o0 = c equals a grid render with T * e^c
    w.b[-1][:] = np.array([0.1, -0.2, 0.0, 0.0], dtype=np.float32)
    c = orc.render_mlp(p, w)
    q = p.replace(T=p.T * math.exp(np.float32(0.1)), n_h2=p.n_h2 * math.exp(np.float32(-0.2)))
    np.testing.assert_allclose(c, orc.render(q), rtol=1e-12, atol=1e-14 * a.max())


# --------------------------------------------------------------------------------------
# Field interpolation, outside-grid rule and the CO layer
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("r_log", [1, 0])
def test_bilinear_interpolation_reproduces_bilinear_fields(orc, r_log):
    """Bilinear interpolation in (grid r coordinate, z/r) is exact for fields that are
    bilinear in those coordinates; any swapped weight or index breaks this."""
    nr, nz = 9, 5
    p = uniform_problem(nr=nr, nz=nz, incl=30.0, mstar=1.0)
    p = p.replace(r_log=r_log)
    r = p.r_nodes()
    zr = p.zr_nodes()
    q = np.log(r) if r_log else r
    R, ZR = np.meshgrid(q, zr)

    def f(a, b, c, d, qq, zz):
        return a + b * qq + c * zz + d * qq * zz

    p = p.replace(T=f(30, 2.0, 17.0, -3.0, R, ZR), n_h2=f(1e5, 3e3, -2e4, 5e3, R, ZR),
                  vturb=f(0.1, 0.01, 0.2, -0.02, R, ZR))
    rng = np.random.default_rng(1)
    for _ in range(40):
        rr = rng.uniform(10.0, 600.0)
        z = rng.uniform(-0.5, 0.5) * rr
        phi = rng.uniform(0, 2 * math.pi)
        d = orc.point(p, rr * math.cos(phi), rr * math.sin(phi), z, 0.0)
        qq = math.log(rr) if r_log else rr
        zz = abs(z) / rr
        assert d["T"] == pytest.approx(f(30, 2.0, 17.0, -3.0, qq, zz), rel=1e-12)
        assert d["n_h2"] == pytest.approx(f(1e5, 3e3, -2e4, 5e3, qq, zz), rel=1e-12)
        assert d["vturb"] == pytest.approx(f(0.1, 0.01, 0.2, -0.02, qq, zz), rel=1e-12)


def test_outside_grid_has_no_gas(orc):
    p = uniform_problem(incl=30.0, mstar=1.0)
    assert orc.point(p, 9.9, 0.0, 0.0, 0.0)["gas"] is False       # r < r_in
    assert orc.point(p, 10.1, 0.0, 0.0, 0.0)["gas"] is True
    assert orc.point(p, 100.0, 0.0, 50.5, 0.0)["gas"] is False    # z/r > zr_max
    assert orc.point(p, 100.0, 0.0, -49.5, 0.0)["gas"] is True    # mirror symmetric


def test_co_layer_logistic_edges(orc):
    p = uniform_problem(incl=30.0, mstar=1.0, hlo=0.1, hhi=0.3, edge_w=0.01)
    for zr in (0.05, 0.1, 0.12, 0.2, 0.3, 0.31, 0.45):
        d = orc.point(p, 200.0, 0.0, zr * 200.0, 0.0)
        sa = 1.0 / (1.0 + math.exp(-(zr - 0.1) / 0.01))
        sb = 1.0 / (1.0 + math.exp(-(0.3 - zr) / 0.01))
        assert d["X_co"] == pytest.approx(1e-4 * sa * sb, rel=1e-12)
    hard = p.replace(edge_w=0.0)
    assert orc.point(hard, 200.0, 0.0, 0.09 * 200, 0.0)["X_co"] == 0.0
    assert orc.point(hard, 200.0, 0.0, 0.2 * 200, 0.0)["X_co"] == 1e-4
    assert orc.point(hard, 200.0, 0.0, 0.31 * 200, 0.0)["X_co"] == 0.0
