"""Pins of the oracle's pressure-corrected rotation (Eq. gas_velocity_pressure) and of the
march with a rotation field (no GPU).

- Uniform pressure: the pressure term vanishes and every node keeps the Keplerian speed.
- n_H2 T linear (and quadratic) in the grid coordinates (ln r, z/r): the second-order
  differences are exact, so v_phi^2 = G M r^2/(r^2+z^2)^{3/2} + (r / rho) dP/dr|_z with
  dP/dr|_z = k (b_u / r - w c_w / r) written out here.
- Rendering with the Keplerian speeds tabulated on a fine grid converges to the Keplerian
  render (interpolation error of v_phi only, second order in the node spacing), and a
  rotation field of zeros gives a spectrum symmetric about v_sys (no rotation).
"""

import math

import numpy as np
import pytest

from paper_2509_03623_b300 import synth

GM_SUN = 1.3271244e26
AU_CM = 1.495978707e13
K_B = 1.380649e-16
AMU = 1.66053906660e-24


def grid_problem(nr=17, nz=13, r_log=1):
    p = synth.config_small(0)
    return p.replace(nr=nr, nz=nz, r_log=r_log, T=np.full((nz, nr), 40.0),
                     n_h2=np.ones((nz, nr)), vturb=np.zeros((nz, nr)), h_lo=np.zeros(nr),
                     h_hi=np.zeros(nr))


def kepler_kms(p):
    r = p.r_nodes()[None, :] * AU_CM
    z = p.zr_nodes()[:, None] * r
    return np.sqrt(GM_SUN * p.mstar_msun * r * r / (r * r + z * z) ** 1.5) / 1e5


def test_uniform_pressure_is_keplerian(orc):
    p = grid_problem()
    v = orc.pressure_vphi(p, np.full((p.nz, p.nr), 3e8), np.full((p.nz, p.nr), 25.0))
    np.testing.assert_allclose(v, kepler_kms(p), rtol=1e-13)


@pytest.mark.parametrize("r_log,quad", [(1, False), (0, False), (1, True)])
def test_polynomial_pressure_exact(orc, r_log, quad):
    p = grid_problem(r_log=r_log)
    r_au = p.r_nodes()[None, :]
    w = p.zr_nodes()[:, None]
    u = np.log(r_au) if r_log else r_au * AU_CM
    du = u.max() - u.min()
    x = (u - u.min()) / du  # grid coordinate scaled to [0, 1]
    T = 30.0
    a, b, c, d = 5e8, -1.1e8, -3e8, 2e7
    nT = a + b * x + c * w + (d * x * x + 4e7 * w * w if quad else 0.0)
    assert nT.min() > 0
    n = nT / T
    dnT_du = (b + (2.0 * d * x if quad else 0.0)) / du
    dnT_dw = c + (8e7 * w if quad else 0.0)
    r = r_au * AU_CM
    dudr = 1.0 / r if r_log else 1.0
    dPdr = K_B * (dnT_du * dudr - (w / r) * dnT_dw)
    m = p.m_mol_amu * AMU
    v2 = (kepler_kms(p) * 1e5) ** 2 + r / (m * n) * dPdr
    want = np.sqrt(np.maximum(v2, 0.0)) / 1e5
    got = orc.pressure_vphi(p, np.broadcast_to(n, (p.nz, p.nr)).copy(), np.full((p.nz, p.nr), T))
    np.testing.assert_allclose(got, want, rtol=1e-10)


def test_pressure_support_beyond_gravity_clamps_to_zero(orc):
    p = grid_problem().replace(mstar_msun=0.0)
    r_au = p.r_nodes()[None, :]
    n = np.broadcast_to(1e9 * (r_au / r_au.min()) ** -2, (p.nz, p.nr)).copy()  # dP/dr < 0
    v = orc.pressure_vphi(p, n, np.full((p.nz, p.nr), 30.0))
    assert np.all(v == 0.0)


def test_tabulated_kepler_rotation_converges_to_kepler_render(orc):
    base = synth.config_small(2).replace(nx=16, ny=16, n_samples=96)
    ref = orc.render(base)
    errs = []
    for nr, nz in ((64, 32), (128, 64), (256, 128)):
        q = synth.disk(2, nr=nr, nz=nz).replace(nx=16, ny=16, n_samples=96)
        vk = kepler_kms(q)
        a = orc.render(q)
        b = orc.render(q.replace(vphi=vk))
        errs.append(np.abs(b - a).max() / np.abs(a).max())
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_zero_rotation_field_gives_symmetric_spectrum(orc):
    p = synth.config_small(1).replace(nx=12, ny=12, n_samples=64, v_kms=np.linspace(-3, 3, 13))
    cube = orc.render(p.replace(vphi=np.zeros((p.nz, p.nr))))
    np.testing.assert_allclose(cube, cube[::-1], rtol=1e-9, atol=1e-12 * np.abs(cube).max())


@pytest.mark.parametrize("r_log,nr,nz", [(1, 9, 7), (0, 6, 5), (1, 2, 2), (1, 12, 3)])
def test_rotation_reverse_mode_matches_central_differences(orc, r_log, nr, nz):
    """dL/dn_H2 and dL/dT of L = sum g v_phi from orc_pressure_vphi_adjoint equal central
    differences of orc_pressure_vphi on every node (log and linear radii, two-node axes with
    their first-order stencil, one-sided edges). The fields keep v_phi^2 > 0 away from 0 so no
    node sits on the clamp."""
    p = grid_problem(nr=nr, nz=nz, r_log=r_log)
    rng = np.random.default_rng(nr * 10 + nz)
    n = 1e7 * np.exp(rng.uniform(-0.3, 0.3, (nz, nr)))
    T = 30.0 * np.exp(rng.uniform(-0.3, 0.3, (nz, nr)))
    g = rng.standard_normal((nz, nr))
    v0 = orc.pressure_vphi(p, n, T)
    assert np.all(v0 > 0)
    gn, gT = orc.pressure_vphi_adjoint(p, g, n, T)
    loss = lambda nn, TT: float((g * orc.pressure_vphi(p, nn, TT)).sum())
    for arr, grad, is_n in ((n, gn, True), (T, gT, False)):
        for k in range(arr.size):
            h = 1e-6 * arr.flat[k]
            ap, am = arr.copy(), arr.copy()
            ap.flat[k] += h
            am.flat[k] -= h
            fd = ((loss(ap, T) - loss(am, T)) if is_n else (loss(n, ap) - loss(n, am))) / (2 * h)
            scale = np.abs(grad).max()
            assert grad.flat[k] == pytest.approx(fd, rel=1e-5, abs=1e-7 * scale), (is_n, k)
