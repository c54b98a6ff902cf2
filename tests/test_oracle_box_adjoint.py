"""Pins of the oracle's reverse mode through the 3-D Cartesian grid (no GPU).

- Central finite differences of the oracle's own 3-D forward march, field by field (T, n_H2,
  v_turb, the CO abundance and the two velocity components the line of sight sees), at the
  nodes carrying the largest gradients and at random ones among those carrying any.
- The x velocity component does not enter v_los = omega . v + v_sys (omega has no x
  component), so its gradient is exactly zero.
- Uniform box, one line-centre channel: the gradients summed over all nodes are the
  derivatives with respect to a uniform change of the field (the trilinear weights sum to
  one). With I = S (1 - e^-tau) and tau proportional to n_H2 and to the abundance, that gives
  sum_i dI/dn_i = S e^-tau tau / n, and sum_i X dI/dX_i = sum_i n dI/dn_i.
"""

import dataclasses

import numpy as np

from paper_2509_03623_b300 import synth
from tests.test_oracle_box import AU_CM, box_chord, ray, uniform_box

FIELDS = ("T", "n_h2", "vturb", "x_co", "vx", "vy", "vz")


def small_box(seed=0):
    p = synth.box3d(seed, n3=(7, 6, 5), nx=12, ny=10, nch=6, vmax=3.0, n_samples=36,
                    incl=40.0, pa=25.0)
    g = p.g3
    # broaden the line and thin the gas so every field matters to the loss
    g = dataclasses.replace(g, vturb=np.full_like(g.vturb, 0.15), n_h2=g.n_h2 * 0.05)
    return p.replace(g3=g)


def loss(orc, p, w):
    return float((orc.render(p) * w).sum())


def with_node(p, field, idx, value):
    a = getattr(p.g3, field).copy()
    a.flat[idx] = value
    return p.replace(g3=dataclasses.replace(p.g3, **{field: a}))


def test_box_adjoint_vs_central_differences(orc):
    p = small_box(2)
    rng = np.random.default_rng(7)
    w = rng.standard_normal((p.nch, p.ny, p.nx))
    cube, g = orc.render_adjoint3(p, w)
    np.testing.assert_allclose(cube, orc.render(p), rtol=1e-14, atol=0)
    assert np.all(g["vx"] == 0.0)
    L = float(np.abs(cube * w).sum())
    checked = 0
    for field in FIELDS[:4] + FIELDS[5:]:
        gf, arr = g[field], getattr(p.g3, field)
        flat = np.abs(gf).ravel()
        # nodes with a value (a zero density or abundance is the edge of the gas, where a
        # step of either sign is not smooth) that carry at least 2 % of the largest gradient
        ok = flat >= 0.02 * flat.max()
        if field in ("n_h2", "x_co"):
            ok &= arr.ravel() > 0
        cand = np.flatnonzero(ok)
        top = cand[np.argsort(flat[cand])[-2:]]
        rest = np.setdiff1d(cand, top)
        picks = list(top) + list(rng.choice(rest, size=min(4, rest.size), replace=False))
        for idx in picks:
            v0 = float(arr.flat[idx])
            # velocities: an absolute step well below the line width; the others relative
            h = 1e-4 if field.startswith("v") and field != "vturb" else 1e-3 * abs(v0)
            f = (loss(orc, with_node(p, field, idx, v0 + h), w)
                 - loss(orc, with_node(p, field, idx, v0 - h), w)) / (2 * h)
            roundoff = 1e-15 * L / h
            assert abs(f - gf.flat[idx]) <= 1e-5 * abs(gf.flat[idx]) + roundoff, (
                field, int(idx), f, gf.flat[idx])
            checked += 1
    assert checked >= 30


def test_box_adjoint_uniform_identities(orc):
    p = uniform_box(n=1e5)
    cube = orc.render(p)
    iy, ix = np.unravel_index(int(np.argmax(cube[0])), cube[0].shape)
    w = np.zeros_like(cube)
    w[0, iy, ix] = 1.0  # L = I of the brightest pixel in the line-centre channel
    _, g = orc.render_adjoint3(p, w)
    # tau = beta L along that ray (the slab-method chord and the local opacity; the forward
    # closed form I = S (1 - e^-tau) is pinned in test_oracle_box)
    local = orc.point(p, 1.0, 2.0, 3.0, 0.0)
    tau = local["beta"] * box_chord(*ray(p, ix, iy), p.g3.extent) * AU_CM
    assert 0.1 < tau < 5.0, tau
    n, xco = float(p.g3.n_h2.flat[0]), float(p.g3.x_co.flat[0])
    dIdn = local["S"] * np.exp(-tau) * tau / n
    assert abs(g["n_h2"].sum() - dIdn) <= 1e-9 * abs(dIdn), (g["n_h2"].sum(), dIdn)
    np.testing.assert_allclose(xco * g["x_co"].sum(), n * g["n_h2"].sum(), rtol=1e-12)
    assert np.all(g["vx"] == 0.0)
