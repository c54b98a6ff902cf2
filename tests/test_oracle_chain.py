"""Pins of the oracle's physics-constrained field chain (no GPU): hydrostatic density from a
temperature grid (Eq. gas_density_temp), normalisation to Sigma(r), H2 column above each
node (Eq. column_density) and the CO-layer surfaces of Eq. co_layer.

Each pin is fixed by something other than the oracle's own arithmetic:
- the surface-density profile and the mirror-symmetric normalisation, from the profile's
  formula evaluated here (the column at the midplane is half the surface density);
- zero gravity: the equation reduces to d ln(rho T)/dz = 0, so rho T is constant;
- an isothermal column: ln rho(z) - ln rho(0) = -(G M m / k T)(1/r - 1/sqrt(r^2 + z^2)) in
  closed form, approached at second order by the node integration;
- the column density of that closed-form density by adaptive quadrature (scipy);
- surfaces: a temperature linear in z/r crosses T_freeze at a closed-form height; the
  photodissociation height is the root of the quadrature column (scipy brentq).
"""

import math

import numpy as np
import pytest
from scipy import integrate, optimize

from paper_2509_03623_b300 import synth

GM_SUN = 1.3271244e26
AU_CM = 1.495978707e13
K_B = 1.380649e-16
AMU = 1.66053906660e-24


def column_problem(nr=5, nz=257, zr_max=0.5, r_in=20.0, r_out=300.0, mstar=2.0):
    p = synth.config_small(0)
    return p.replace(nr=nr, nz=nz, zr_max=zr_max, r_in_au=r_in, r_out_au=r_out, r_log=1,
                     mstar_msun=mstar, T=np.full((nz, nr), 30.0),
                     n_h2=np.zeros((nz, nr)), vturb=np.zeros((nz, nr)),
                     h_lo=np.zeros(nr), h_hi=np.zeros(nr))


def sigma_of(c, r_au):
    x = r_au / c.r_c_au
    return c.sigma0_gcm2 * x ** -c.gamma * np.exp(-x ** (2.0 - c.gamma))


def test_midplane_column_is_half_the_surface_density(orc):
    p = column_problem()
    rng = np.random.default_rng(0)
    T = 20.0 + 40.0 * rng.random((p.nz, p.nr))
    c = synth.chain_params(p)
    out = orc.field_chain(p, c, T)
    m = p.m_mol_amu * AMU
    want = sigma_of(c, p.r_nodes()) / (2.0 * m)
    np.testing.assert_allclose(out["N_h2"][0], want, rtol=1e-12)
    assert np.all(out["N_h2"][-1] == 0.0)
    assert np.all(np.diff(out["N_h2"], axis=0) <= 0.0)


def test_chain_mass_normalisation():
    """Sigma0 from the closed-form mass integral reproduces M_gas by quadrature."""
    p = column_problem(r_in=10.0, r_out=600.0)
    c = synth.chain_params(p, m_gas_msun=0.09)
    f = lambda r: 2 * math.pi * r * AU_CM ** 2 * sigma_of(c, r)
    mass, _ = integrate.quad(f, p.r_in_au, p.r_out_au, limit=200)
    assert mass / 1.98847e33 == pytest.approx(0.09, rel=1e-3)  # M_sun in g (IAU nominal / G)


def test_zero_gravity_keeps_pressure_constant(orc):
    p = column_problem(mstar=0.0)
    rng = np.random.default_rng(1)
    T = 15.0 + 60.0 * rng.random((p.nz, p.nr))
    out = orc.field_chain(p, synth.chain_params(p), T)
    P = out["n_h2"] * T
    np.testing.assert_allclose(P / P[0], 1.0, rtol=1e-12)


@pytest.mark.parametrize("T0", [12.0, 40.0])
def test_isothermal_column_closed_form_second_order(orc, T0):
    errs = []
    for nz in (129, 257, 513):
        p = column_problem(nz=nz)
        out = orc.field_chain(p, synth.chain_params(p), np.full((nz, p.nr), T0))
        r = p.r_nodes() * AU_CM
        z = p.zr_nodes()[:, None] * r[None, :]
        a = GM_SUN * p.mstar_msun * p.m_mol_amu * AMU / (K_B * T0)
        want = -a * (1.0 / r[None, :] - 1.0 / np.sqrt(r[None, :] ** 2 + z ** 2))
        got = np.log(out["n_h2"] / out["n_h2"][0])
        errs.append(np.abs(got - want).max())
    assert errs[-1] < 1e-4 * max(1.0, np.abs(want).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def test_column_density_against_quadrature(orc):
    """Quadrature column of the closed-form isothermal density; the node integration (two
    trapezoid rules: the density shape and the column) converges to it at second order."""
    T0 = 25.0
    errs = []
    for nz in (513, 1025, 2049):
        p = column_problem(nz=nz)
        c = synth.chain_params(p)
        out = orc.field_chain(p, c, np.full((p.nz, p.nr), T0))
        m = p.m_mol_amu * AMU
        a = GM_SUN * p.mstar_msun * m / (K_B * T0)
        worst = 0.0
        for i in (0, 2, 4):
            r = p.r_nodes()[i] * AU_CM
            zmax = p.zr_max * r
            shape = lambda z: math.exp(-a * (1.0 / r - 1.0 / math.sqrt(r * r + z * z)))
            norm, _ = integrate.quad(shape, 0.0, zmax, epsabs=0, epsrel=1e-12, limit=200)
            n0 = sigma_of(c, p.r_nodes()[i]) / (2.0 * norm * m)
            N0 = out["N_h2"][0, i]
            for wj in (0.0, 0.02, 0.05, 0.1, 0.15, 0.3):
                j = int(round(wj / p.zr_max * (nz - 1)))
                if out["N_h2"][j, i] < 1e-6 * N0:
                    continue  # far tail: below any CO threshold of interest
                zj = p.zr_nodes()[j] * r
                N, _ = integrate.quad(lambda z: n0 * shape(z), zj, zmax, epsabs=0, epsrel=1e-12,
                                      limit=200)
                worst = max(worst, abs(out["N_h2"][j, i] / N - 1.0))
        errs.append(worst)
    assert errs[-1] < 3e-4, errs  # 12 nodes per local decay length at w = 0.3, r = 20 au
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.1)


def test_freeze_out_surface_of_a_linear_temperature(orc):
    p = column_problem(nz=33)
    w = p.zr_nodes()
    c = synth.chain_params(p, T_freeze=19.0)
    # column 0: midplane already warm; 1..3: T = a + b w crosses 19 K; 4: always frozen
    T = np.empty((p.nz, p.nr))
    T[:, 0] = 25.0 + 10.0 * w
    for i, (a, b) in zip((1, 2, 3), ((10.0, 40.0), (15.0, 100.0), (5.0, 29.0))):
        T[:, i] = a + b * w
    T[:, 4] = 10.0 + 5.0 * w
    out = orc.field_chain(p, c, T)
    assert out["h_lo"][0] == 0.0
    for i, (a, b) in zip((1, 2, 3), ((10.0, 40.0), (15.0, 100.0), (5.0, 29.0))):
        assert out["h_lo"][i] == pytest.approx((19.0 - a) / b, abs=1e-12)
    assert out["h_lo"][4] == p.zr_max


def test_photodissociation_surface_against_quadrature_root(orc):
    T0 = 25.0
    p = column_problem(nz=2049)
    c = synth.chain_params(p, N_dissoc_cm2=1.3e21)
    out = orc.field_chain(p, c, np.full((p.nz, p.nr), T0))
    m = p.m_mol_amu * AMU
    a = GM_SUN * p.mstar_msun * m / (K_B * T0)
    for i in range(p.nr):
        r = p.r_nodes()[i] * AU_CM
        zmax = p.zr_max * r
        shape = lambda z: math.exp(-a * (1.0 / r - 1.0 / math.sqrt(r * r + z * z)))
        norm, _ = integrate.quad(shape, 0.0, zmax, epsabs=0, epsrel=1e-12, limit=200)
        n0 = sigma_of(c, p.r_nodes()[i]) / (2.0 * norm * m)
        colw = lambda w: 0.706 * integrate.quad(lambda z: n0 * shape(z), w * r, zmax,
                                                epsabs=0, epsrel=1e-12, limit=200)[0]
        if colw(0.0) <= c.N_dissoc_cm2:
            assert out["h_hi"][i] == 0.0
            continue
        root = optimize.brentq(lambda w: colw(w) - c.N_dissoc_cm2, 0.0, p.zr_max, xtol=1e-14)
        assert out["h_hi"][i] == pytest.approx(root, abs=1e-5), i


def test_no_photodissociation_layer_when_the_column_is_thin(orc):
    p = column_problem(nz=65)
    c = synth.chain_params(p, m_gas_msun=1e-12)
    out = orc.field_chain(p, c, np.full((p.nz, p.nr), 30.0))
    assert np.all(out["h_hi"] == 0.0)
