"""Pins of the oracle's reverse mode through the 3-D spherical grid (no GPU).

- Central finite differences of the oracle's own spherical forward march, field by field
  (T, n_H2, v_turb, the CO abundance and the three velocity components v_r, v_theta, v_phi),
  at the nodes carrying the largest gradients and at random ones among those carrying any,
  on a grid whose azimuth wraps (the last node's cells reach back to the first).
- Uniform full sphere, one line-centre channel: the gradients summed over all nodes are the
  derivatives with respect to a uniform change of the field (the trilinear weights sum to
  one), so sum_i dI/dn_i = S e^-tau tau / n with tau = beta L and L = 2 sqrt(r_out^2 - b^2)
  the chord at impact parameter b, and sum_i X dI/dX_i = sum_i n dI/dn_i.
- Gas at rest seen face on (i = 0): the line of sight omega = (0, 0, -1) has no azimuthal
  component, so the v_phi gradient is exactly zero.
"""

import dataclasses
import math

import numpy as np

from paper_2509_03623_b300 import synth
from tests.test_oracle_sph import AU_CM, ray, uniform_sphere

FIELDS = ("T", "n_h2", "vturb", "x_co", "vr", "vth", "vph")


def small_sphere(seed=0, **kw):
    p = synth.sphere3d(seed, nsph=(7, 6, 5), nx=12, ny=10, nch=6, vmax=3.0, n_samples=40,
                       incl=40.0, pa=25.0, **kw)
    g = p.gs
    g = dataclasses.replace(g, vturb=np.full_like(g.vturb, 0.15), n_h2=g.n_h2 * 0.05)
    return p.replace(gs=g)


def loss(orc, p, w):
    return float((orc.render(p) * w).sum())


def with_node(p, field, idx, value):
    a = getattr(p.gs, field).copy()
    a.flat[idx] = value
    return p.replace(gs=dataclasses.replace(p.gs, **{field: a}))


def test_sph_adjoint_vs_central_differences(orc):
    p = small_sphere(3)
    rng = np.random.default_rng(9)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    cube, g = orc.render_adjoint3(p, w)
    np.testing.assert_allclose(cube, orc.render(p), rtol=1e-14, atol=0)
    L = float(np.abs(cube * w).sum())
    checked = 0
    for field in FIELDS:
        gf, arr = g[field], getattr(p.gs, field)
        flat = np.abs(gf).ravel()
        ok = flat >= 0.02 * flat.max()
        if field in ("n_h2", "x_co"):
            ok &= arr.ravel() > 0
        cand = np.flatnonzero(ok)
        top = cand[np.argsort(flat[cand])[-2:]]
        rest = np.setdiff1d(cand, top)
        picks = list(top) + list(rng.choice(rest, size=min(4, rest.size), replace=False))
        # nodes of the last azimuth plane, whose cells wrap to the first, among them
        last = np.flatnonzero(np.arange(arr.size) // (p.gs.nth * p.gs.nr) == p.gs.nph - 1)
        wrap = np.intersect1d(last, cand)
        if wrap.size:
            picks.append(int(wrap[np.argmax(flat[wrap])]))
        for idx in picks:
            v0 = float(arr.flat[idx])
            h = 1e-4 if field in ("vr", "vth", "vph") else 1e-3 * abs(v0)
            f = (loss(orc, with_node(p, field, idx, v0 + h), w)
                 - loss(orc, with_node(p, field, idx, v0 - h), w)) / (2 * h)
            roundoff = 1e-15 * L / h
            assert abs(f - gf.flat[idx]) <= 1e-5 * abs(gf.flat[idx]) + roundoff, (
                field, int(idx), f, gf.flat[idx])
            checked += 1
    assert checked >= 35


def test_sph_adjoint_uniform_identities(orc):
    p = uniform_sphere(n=1e4)
    cube = orc.render(p)
    iy, ix = np.unravel_index(int(np.argmax(cube[0])), cube[0].shape)
    w = np.zeros_like(cube)
    w[0, iy, ix] = 1.0
    _, g = orc.render_adjoint3(p, w)
    local = orc.point(p, 1.0, 2.0, 3.0, 0.0)
    P0, om = ray(p, ix, iy)
    b2 = P0 @ P0 - (P0 @ om) ** 2
    tau = local["beta"] * 2.0 * math.sqrt(p.gs.r_out ** 2 - b2) * AU_CM
    assert 0.1 < tau < 5.0, tau
    n, xco = float(p.gs.n_h2.flat[0]), float(p.gs.x_co.flat[0])
    dIdn = local["S"] * np.exp(-tau) * tau / n
    assert abs(g["n_h2"].sum() - dIdn) <= 1e-9 * abs(dIdn), (g["n_h2"].sum(), dIdn)
    np.testing.assert_allclose(xco * g["x_co"].sum(), n * g["n_h2"].sum(), rtol=1e-12)


def test_sph_adjoint_face_on_no_azimuthal_gradient(orc):
    p = uniform_sphere(n=1e4, incl=0.0, nch=5).replace(v_kms=np.linspace(-0.5, 0.5, 5))
    w = np.random.default_rng(2).standard_normal((p.nch, p.ny, p.nx))
    _, g = orc.render_adjoint3(p, w)
    assert np.abs(g["vr"]).max() > 0 and np.abs(g["vth"]).max() > 0
    assert np.all(g["vph"] == 0.0)
