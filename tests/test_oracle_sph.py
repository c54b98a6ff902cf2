"""Pins of the oracle's 3-D spherical grid march (next row f4; no GPU).

- A uniform full sphere (constant fields, gas at rest, r linear from 0, theta over [0, pi]):
  every ray gives I = S (1 - exp(-beta L)) with L = 2 sqrt(r_out^2 - b^2) the chord of a ray at
  impact parameter b, computed here from the ray geometry, and S, beta the local values.
- A uniform wedge seen face on (theta within a of the midplane): a ray at impact parameter b
  crosses gas over |z| <= b tan a inside the sphere; optically thin, I = S beta L_w up to the
  midpoint rule's resolution of the wedge's edges (one sample at each).
- A uniform flow v = (0, w_y, w_z) written in spherical components (v_r, v_theta, v_phi) at the
  nodes shifts the line of every pixel to v_los = w_y sin i - w_z cos i: the cube is then
  symmetric in channel order about that velocity (up to the interpolation of the components
  in theta and phi, second order in the node spacing), and not about zero.
- Reversing every velocity mirrors the cube in channel order (channels symmetric about 0).
- An expanding sphere with temperature falling outward, optically thick: on the central ray
  the red (receding, far-side) peak is brighter than the blue one, since the far side is seen
  from its hot inner edge and the near side from its cool outer edge.
- The parametric disk (no jitter) written onto spherical grids of increasing resolution
  renders towards the axisymmetric render of the same disk (first order near the disk's
  edges, where its fields are discontinuous).
"""

import math

import numpy as np
import pytest

from paper_2509_03623_b300 import synth

GM_SUN = 1.3271244e26
AU_CM = 1.495978707e13
K_B = 1.380649e-16
AMU = 1.66053906660e-24


def uniform_sphere(T=35.0, n=1e5, vt=0.1, xco=1e-4, w=(0.0, 0.0, 0.0), nsph=(6, 9, 8),
                   r_out=80.0, th=(0.0, math.pi), r_in=0.0, r_log=0, incl=38.0, nch=1,
                   n_samples=41, nx=9, ny=7, Tfun=None):
    """Constant fields on a spherical grid; w = (wx, wy, wz) a uniform flow in Cartesian
    components, written at the nodes in spherical components."""
    gnr, gnth, gnph = nsph
    g = synth.GridSph(gnr, gnth, gnph, r_log, r_in, r_out, th[0], th[1], *([None] * 7))
    r, ths, phs = g.nodes()
    PH, TH, RR = np.meshgrid(phs, ths, r, indexing="ij")
    wx, wy, wz = w
    st, ct, sp, cp = np.sin(TH), np.cos(TH), np.sin(PH), np.cos(PH)
    vr = wx * st * cp + wy * st * sp + wz * ct
    vth = wx * ct * cp + wy * ct * sp - wz * st
    vph = -wx * sp + wy * cp
    Tn = np.full(RR.shape, T) if Tfun is None else Tfun(RR)
    g = synth.GridSph(gnr, gnth, gnph, r_log, r_in, r_out, th[0], th[1], Tn,
                      np.full(RR.shape, n), np.full(RR.shape, vt), np.full(RR.shape, xco),
                      vr, vth, vph)
    p = synth.sphere3d(0, nsph=(4, 4, 4), nx=nx, ny=ny, nch=nch, n_samples=n_samples,
                       incl=incl, pa=25.0)
    return p.replace(gs=g, half_fov_au=1.1 * r_out, v_kms=np.array([0.0]))


def ray(p, ix, iy):
    inc, pa = math.radians(p.incl_deg), math.radians(p.pa_deg)
    hf = p.half_fov_au
    X = (ix + 0.5 - 0.5 * p.nx) * 2 * hf / p.nx
    Y = (iy + 0.5 - 0.5 * p.ny) * 2 * hf / p.ny
    xs = X * math.cos(pa) + Y * math.sin(pa)
    ys = -X * math.sin(pa) + Y * math.cos(pa)
    P0 = np.array([xs, ys * math.cos(inc), ys * math.sin(inc)])
    om = np.array([0.0, math.sin(inc), -math.cos(inc)])
    return P0, om


def test_uniform_sphere_closed_form(orc):
    p = uniform_sphere()
    cube = orc.render(p)[0]
    local = orc.point(p, 1.0, 2.0, 3.0, 0.0)
    S, beta = local["S"], local["beta"]
    assert local["gas"]
    hits = 0
    R = p.gs.r_out
    for iy in range(p.ny):
        for ix in range(p.nx):
            P0, om = ray(p, ix, iy)
            b2 = P0 @ P0 - (P0 @ om) ** 2
            L = 2.0 * math.sqrt(R * R - b2) * AU_CM if b2 < R * R else 0.0
            want = S * -math.expm1(-beta * L) if L > 0 else 0.0
            assert cube[iy, ix] == pytest.approx(want, rel=1e-11, abs=1e-30), (ix, iy)
            hits += L > 0
    assert 0 < hits < p.nx * p.ny  # the corner rays miss the sphere


def test_uniform_wedge_face_on(orc):
    """Face on (i = 0) the rays run along -z; at impact parameter b the gas of the wedge
    |pi/2 - theta| <= a lies at |z| <= b tan a (and inside the sphere)."""
    a = 0.4
    ns = 4000
    p = uniform_sphere(n=1e-3, th=(0.5 * math.pi - a, 0.5 * math.pi + a), incl=0.0, nx=7,
                       ny=5, n_samples=ns)
    cube = orc.render(p)[0]
    local = orc.point(p, 30.0, 0.0, 0.0, 0.0)
    S, beta = local["S"], local["beta"]
    R = p.gs.r_out
    for iy in range(p.ny):
        for ix in range(p.nx):
            P0, om = ray(p, ix, iy)
            b = math.hypot(P0[0], P0[1])
            if b >= R:
                assert cube[iy, ix] == 0.0
                continue
            half = math.sqrt(R * R - b * b)
            Lw = 2.0 * min(b * math.tan(a), half)
            ds = 2.0 * half / ns
            want = S * beta * Lw * AU_CM  # optically thin (beta L ~ 1e-8)
            assert abs(cube[iy, ix] - want) <= S * beta * 2.0 * ds * AU_CM * 1.0001 + 1e-12 * want


def test_uniform_flow_shifts_the_line(orc):
    wy, wz = 1.3, -0.9
    # (even image sizes: no ray through the centre, where the direction r^ is undefined)
    p = uniform_sphere(w=(0.0, wy, wz), nsph=(6, 181, 240), n=3e6, nx=8, ny=8)
    inc = math.radians(p.incl_deg)
    vc = wy * math.sin(inc) - wz * math.cos(inc)
    q = p.replace(v_kms=vc + np.linspace(-1.2, 1.2, 13))
    cube = orc.render(q)
    peak = np.abs(cube).max()
    assert peak > 0
    # node spacing 1 deg in theta, 1.5 deg in phi: the interpolated flow is off by
    # ~w d^2 / 8 ~ 1e-4 km/s, against a line width of ~0.35 km/s
    np.testing.assert_allclose(cube, cube[::-1], rtol=0, atol=2e-3 * peak)
    c0 = orc.render(p.replace(v_kms=np.linspace(-1.2, 1.2, 13)))
    assert np.abs(c0 - c0[::-1]).max() > 0.05 * np.abs(c0).max()


def test_reversed_velocities_mirror_the_cube(orc):
    base = synth.sphere3d(3, nsph=(24, 12, 16), nx=10, ny=10, nch=15, vmax=4.0, n_samples=96)
    g = base.gs
    rev = base.replace(gs=synth.GridSph(g.nr, g.nth, g.nph, g.r_log, g.r_in, g.r_out, g.th0,
                                        g.th1, g.T, g.n_h2, g.vturb, g.x_co, -g.vr, -g.vth,
                                        -g.vph))
    a, b = orc.render(base), orc.render(rev)
    assert np.abs(a).max() > 0
    np.testing.assert_allclose(b, a[::-1], rtol=1e-8, atol=1e-13 * np.abs(a).max())


def test_expanding_sphere_red_peak(orc):
    vr = 1.0
    p = uniform_sphere(w=(0.0, 0.0, 0.0), nsph=(40, 9, 8), n=3e5, nx=1, ny=1, n_samples=800,
                       Tfun=lambda r: 100.0 * (1.0 + r / 10.0) ** -1)
    g = p.gs
    p = p.replace(gs=synth.GridSph(g.nr, g.nth, g.nph, g.r_log, g.r_in, g.r_out, g.th0, g.th1,
                                   g.T, g.n_h2, g.vturb, g.x_co, np.full_like(g.T, vr),
                                   np.zeros_like(g.T), np.zeros_like(g.T)),
                  v_kms=np.array([-vr, vr]))
    blue, red = orc.render(p)[:, 0, 0]
    assert red > 1.5 * blue > 0


def disk_on_sph(p, nsph, r_in, r_out, th_half):
    """The analytic fields of the parametric disk p (no jitter) at the nodes of a spherical
    grid."""
    gnr, gnth, gnph = nsph
    th0, th1 = 0.5 * math.pi - th_half, 0.5 * math.pi + th_half
    g = synth.GridSph(gnr, gnth, gnph, 1, r_in, r_out, th0, th1, *([None] * 7))
    rr, ths, phs = g.nodes()
    PH, TH, RR = np.meshgrid(phs, ths, rr, indexing="ij")
    R = RR * np.sin(TH)
    Z = RR * np.cos(TH)
    Rs = np.maximum(R, 1e-6)
    Tm = 20.0 * (Rs / 100.0) ** -0.5
    Ta = 60.0 * (Rs / 100.0) ** -0.5
    zq = 70.0 * (Rs / 150.0) ** 1.3
    T = Tm + (Ta - Tm) * np.where(np.abs(Z) < zq, np.sin(math.pi * np.abs(Z) / (2 * zq)) ** 2, 1.0)
    m = p.m_mol_amu * AMU
    H = np.sqrt(K_B * Tm / m) / np.sqrt(GM_SUN * p.mstar_msun / (Rs * AU_CM) ** 3)
    sig0 = synth._sigma0_from_mass(0.09, p.r_in_au, p.r_out_au)
    sig = sig0 * (Rs / 100.0) ** -1 * np.exp(-Rs / 300.0)
    n = sig / (math.sqrt(2 * math.pi) * H) * np.exp(-(Z * AU_CM) ** 2 / (2 * H ** 2)) / m
    zr = np.abs(Z) / Rs
    inside = (R >= p.r_in_au) & (R <= p.r_out_au) & (zr <= p.zr_max)
    n = np.where(inside, n, 0.0)
    c_lo, p_lo, c_hi, p_hi = p.surf
    hlo = c_lo * (Rs / 100.0) ** p_lo
    hhi = c_hi * (Rs / 100.0) ** p_hi
    sg = lambda u: 0.5 * (1.0 + np.tanh(0.5 * u))  # logistic, without overflow
    xco = p.x_co * sg((zr - hlo) / p.edge_w) * sg((hhi - zr) / p.edge_w)
    vphi = np.sqrt(GM_SUN * p.mstar_msun * (Rs * AU_CM) ** 2
                   / ((Rs * AU_CM) ** 2 + (Z * AU_CM) ** 2) ** 1.5) / 1e5
    g = synth.GridSph(gnr, gnth, gnph, 1, r_in, r_out, th0, th1, T, n,
                      np.full_like(T, p.vturb.flat[0]), xco, np.zeros_like(T), np.zeros_like(T),
                      vphi)
    return p.replace(gs=g, half_fov_au=1.1 * p.r_out_au)


def test_disk_on_refined_spheres_converges_to_axisymmetric_render(orc):
    """The disk's fields are discontinuous at r_in, r_out and z/r = zr_max (no gas outside),
    where trilinear interpolation is first order, so the pin asks for a steady fall of the
    difference with each halving of the node spacing and 3 % at the finest grid; an error in
    the spherical geometry, the interpolation or the velocity components leaves an O(1)
    difference that does not fall."""
    base = synth.disk(0, jitter=0.0, nr=512, nz=256, r_in=60.0, r_out=300.0, nx=12, ny=12,
                      nch=12, vmax=4.0, n_samples=256, incl=40.0, edge_w=0.05)
    ref = orc.render(base)
    errs = []
    for k in (1, 2, 4):
        q = disk_on_sph(base, (32 * k, 16 * k, 24 * k), 40.0, 340.0, 0.5)
        c = orc.render(q)
        errs.append(np.abs(c - ref).sum() / np.abs(ref).sum())
    assert errs[-1] < 0.03, errs
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8, errs
