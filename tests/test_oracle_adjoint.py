"""Pins of the oracle's hand-derived reverse mode (no GPU): central finite differences of
the oracle's own forward march, a dot-product (Jacobian transpose) test, the uniform-slab
closed form dI/dn = (S - I0) e^-tau tau / n, and the chain rule to the surface power-law
parameters."""

import math

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.test_oracle_pins import uniform_problem


def small_problem(seed=0):
    p = synth.disk(seed, nr=12, nz=6, nx=14, ny=12, nch=5, vmax=2.0, n_samples=40,
                   incl=40.0, pa=25.0)
    # broaden the line and thin the disk so every field matters to the loss
    return p.replace(vturb=np.full_like(p.vturb, 0.15), n_h2=p.n_h2 * 0.05)


def loss(orc, p, w):
    return float((orc.render(p) * w).sum())


def fd(orc, p, w, field, idx, rel=1e-3):
    arr = getattr(p, field).copy()
    h = rel * abs(arr.flat[idx]) if arr.flat[idx] != 0 else rel
    a = arr.copy()
    a.flat[idx] += h
    b = arr.copy()
    b.flat[idx] -= h
    return (loss(orc, p.replace(**{field: a}), w) - loss(orc, p.replace(**{field: b}), w)) / (2 * h)


def test_p11_adjoint_vs_central_differences(orc):
    p = small_problem(1)
    rng = np.random.default_rng(5)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    cube, g = orc.render_adjoint(p, w)
    np.testing.assert_allclose(cube, orc.render(p), rtol=1e-14, atol=0)
    checked = 0
    for field, n_cells in (("T", 10), ("n_h2", 10), ("vturb", 6), ("h_lo", 3), ("h_hi", 3)):
        gf = g[field]
        flat = np.abs(gf).ravel()
        # random cells among those that carry gradient: |g| >= 2% of the field's largest
        cand = np.flatnonzero(flat >= 0.02 * flat.max())
        picks = rng.choice(cand, size=min(n_cells, cand.size), replace=False)
        arr = getattr(p, field)
        # the surfaces enter through logistic edges of width 0.01 in z/r: a smaller relative
        # step keeps the O(h^2) truncation below the tolerance
        rel = 1e-4 if field.startswith("h_") else 1e-3
        for idx in picks:
            f = fd(orc, p, w, field, int(idx), rel)
            # FD truncation O(h^2) plus roundoff eps |L| / h of the two renders
            h = rel * abs(arr.flat[idx])
            roundoff = 1e-15 * float(np.abs(cube * w).sum()) / h
            assert abs(f - gf.flat[idx]) <= 1e-5 * abs(gf.flat[idx]) + roundoff, (
                field, int(idx), f, gf.flat[idx])
            checked += 1
    assert checked == 32


def test_p11_dot_product(orc):
    p = small_problem(2)
    rng = np.random.default_rng(9)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    _, g = orc.render_adjoint(p, w)
    # <J v, w> via a central difference along v = <v, J^T w> from the adjoint
    vT = rng.standard_normal(p.T.shape) * p.T
    vn = rng.standard_normal(p.n_h2.shape) * p.n_h2
    vl = rng.standard_normal(p.nr) * p.h_lo
    eps = 1e-4
    plus = p.replace(T=p.T + eps * vT, n_h2=p.n_h2 + eps * vn, h_lo=p.h_lo + eps * vl)
    minus = p.replace(T=p.T - eps * vT, n_h2=p.n_h2 - eps * vn, h_lo=p.h_lo - eps * vl)
    jv = (loss(orc, plus, w) - loss(orc, minus, w)) / (2 * eps)
    vjt = (g["T"] * vT).sum() + (g["n_h2"] * vn).sum() + (g["h_lo"] * vl).sum()
    assert jv == pytest.approx(vjt, rel=1e-6)


def test_p11_slab_closed_form(orc):
    # uniform slab: I = S (1 - e^-tau) + I0 e^-tau with tau proportional to n, so
    # sum over nodes of dI/dn = (S - I0) e^-tau tau / n
    n, I0 = 4e3, 1.5e-13
    p = uniform_problem(T=33.0, n=n, I0=I0)
    w = np.zeros((1, 1, 2))
    w[0, 0, 0] = 1.0
    cube, g = orc.render_adjoint(p, w)
    I = cube[0, 0, 0]
    b = orc.render(p.replace(I0=0.0))[0, 0, 0]
    trans = (I - b) / I0
    tau = -math.log(trans)
    S = b / (1 - trans)
    assert g["n_h2"].sum() == pytest.approx((S - I0) * trans * tau / n, rel=1e-10)
    # the background enters only through e^-tau: dI/dI0 = e^-tau (checked by linearity)
    assert orc.render(p.replace(I0=2 * I0))[0, 0, 0] - I == pytest.approx(trans * I0, rel=1e-9)


def test_surface_power_law_chain_rule(orc):
    """dL/dp_s = sum_i dL/dh_s[i] h_s[i] ln(r_i / 100 au) for h_s = c_s (r/100)^p_s."""
    p = small_problem(3)
    rng = np.random.default_rng(2)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    _, g = orc.render_adjoint(p, w)
    r = p.r_nodes()
    c_lo, p_lo, c_hi, p_hi = p.surf
    dp_lo = float((g["h_lo"] * p.h_lo * np.log(r / 100.0)).sum())
    dc_hi = float((g["h_hi"] * p.h_hi / c_hi).sum())
    d = 1e-4
    def with_surf(cl, pl, ch, phh):
        lo, hi = synth.surfaces(r, cl, pl, ch, phh)
        return p.replace(h_lo=lo, h_hi=hi)
    fd_p = (loss(orc, with_surf(c_lo, p_lo + d, c_hi, p_hi), w)
            - loss(orc, with_surf(c_lo, p_lo - d, c_hi, p_hi), w)) / (2 * d)
    fd_c = (loss(orc, with_surf(c_lo, p_lo, c_hi + d * c_hi, p_hi), w)
            - loss(orc, with_surf(c_lo, p_lo, c_hi - d * c_hi, p_hi), w)) / (2 * d * c_hi)
    assert dp_lo == pytest.approx(fd_p, rel=1e-5)
    assert dc_hi == pytest.approx(fd_c, rel=1e-5)


def test_adjoint_mach_mode_and_units(orc):
    p = small_problem(4).replace(vturb_mach=1, units=1, I0=1e-4)
    p = p.replace(vturb=np.full_like(p.vturb, 0.3))
    rng = np.random.default_rng(3)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    _, g = orc.render_adjoint(p, w)
    for field, idx in (("vturb", 20), ("T", 31), ("n_h2", 19)):
        idx = int(np.argsort(np.abs(g[field]).ravel())[-1 - idx % 5])
        f = fd(orc, p, w, field, idx)
        assert f == pytest.approx(g[field].flat[idx], rel=2e-5, abs=1e-9 * np.abs(g[field]).max())


def test_adjoint_through_a_rotation_field(orc):
    """With a tabulated rotation field (Keplerian speeds plus a perturbation), dL/d(field)
    from orc_render_adjoint_vphi matches central differences of the forward march at random
    nodes that carry gradient, and the other fields' gradients are those of a problem whose
    line-of-sight velocity comes from the field (spot checks)."""
    from tests.test_oracle_vphi import kepler_kms
    p = small_problem(2)
    rng = np.random.default_rng(8)
    vk = kepler_kms(p) * (1.0 + 0.05 * rng.standard_normal((p.nz, p.nr)))
    p = p.replace(vphi=vk)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    cube, g = orc.render_adjoint_vphi(p, w)
    np.testing.assert_allclose(cube, orc.render(p), rtol=1e-14, atol=0)
    for field, n_cells in (("vphi", 12), ("T", 4), ("n_h2", 4)):
        gf = g[field]
        flat = np.abs(gf).ravel()
        cand = np.flatnonzero(flat >= 0.02 * flat.max())
        assert cand.size > 0, field
        rel = 1e-4
        for idx in rng.choice(cand, size=min(n_cells, cand.size), replace=False):
            if field == "vphi":
                # rotation speeds are ~50 line widths, so the second-order stencil's truncation
                # is ~1e-5 at this step and the FP64 renders' roundoff ~1e-5 at a ten times
                # smaller one: the fourth-order stencil (truncation O(h^4))
                f = (4.0 * fd(orc, p, w, field, int(idx), rel)
                     - fd(orc, p, w, field, int(idx), 2 * rel)) / 3.0
            else:
                f = fd(orc, p, w, field, int(idx), rel)
            h = rel * abs(getattr(p, field).flat[idx])
            roundoff = 1e-15 * float(np.abs(cube * w).sum()) / h
            assert abs(f - gf.flat[idx]) <= 1e-5 * abs(gf.flat[idx]) + roundoff, (
                field, int(idx), f, gf.flat[idx])
