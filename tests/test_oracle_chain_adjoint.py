"""Pin of the oracle's reverse mode through the field chain (no GPU): for a scalar loss
L = sum g_n n_H2 + sum g_lo h_lo + sum g_hi h_hi of the chain's outputs, dL/dT from
orc_field_chain_adjoint equals central finite differences of the chain's forward
(orc_field_chain) on every node of a small grid, and on selected nodes of a finer one. The
temperature field crosses T_freeze and the column crosses the photodissociation threshold
inside the grid, so both surfaces carry gradient; steps stay well inside the crossing cells
(the choice of cell is piecewise constant in T)."""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth


def chain_problem(nr, nz, seed):
    rng = np.random.default_rng(seed)
    p = synth.config_small(0).replace(nr=nr, nz=nz, zr_max=0.5, r_in_au=20.0, r_out_au=300.0,
                                      r_log=1, n_h2=np.zeros((nz, nr)), vturb=np.zeros((nz, nr)),
                                      h_lo=np.zeros(nr), h_hi=np.zeros(nr))
    w = np.linspace(0.0, 0.5, nz)[:, None]
    r = p.r_nodes()[None, :]
    # warm atmosphere over a cold midplane: crosses 19 K at w ~ 0.1-0.2
    T = 12.0 + 60.0 * w / 0.5 * (100.0 / r) ** 0.2 + rng.uniform(-0.5, 0.5, (nz, nr))
    return p.replace(T=T), rng


def loss_and_weights(orc, p, c, T, gw):
    out = orc.field_chain(p, c, T)
    gn, glo, ghi = gw
    return (gn * out["n_h2"]).sum() + (glo * out["h_lo"]).sum() + (ghi * out["h_hi"]).sum()


@pytest.mark.parametrize("seed", [0, 1])
def test_chain_adjoint_matches_central_differences(orc, seed):
    p, rng = chain_problem(nr=4, nz=17, seed=seed)
    c = synth.chain_params(p)
    out = orc.field_chain(p, c, p.T)
    assert np.all((out["h_lo"] > 0) & (out["h_lo"] < p.zr_max)), out["h_lo"]
    assert np.all((out["h_hi"] > 0) & (out["h_hi"] < p.zr_max)), out["h_hi"]
    nscale = out["n_h2"].max()
    gw = (rng.standard_normal((p.nz, p.nr)) / nscale, rng.standard_normal(p.nr),
          rng.standard_normal(p.nr))
    gT = orc.field_chain_adjoint(p, c, p.T, *gw)
    fd = np.zeros_like(gT)
    for j in range(p.nz):
        for i in range(p.nr):
            h = 1e-4 * p.T[j, i]
            Tp, Tm = p.T.copy(), p.T.copy()
            Tp[j, i] += h
            Tm[j, i] -= h
            fd[j, i] = (loss_and_weights(orc, p, c, Tp, gw)
                        - loss_and_weights(orc, p, c, Tm, gw)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    np.testing.assert_allclose(gT, fd, rtol=1e-5, atol=1e-6 * scale)


def test_chain_adjoint_each_output_alone(orc):
    """Each output's gradient alone (n only, h_lo only, h_hi only) on a finer grid, at the
    nodes where it is largest: a mistake confined to one branch of the reverse mode fails
    here even where the others would mask it."""
    p, rng = chain_problem(nr=3, nz=65, seed=3)
    c = synth.chain_params(p)
    nscale = orc.field_chain(p, c, p.T)["n_h2"].max()
    zeros = (np.zeros((p.nz, p.nr)), np.zeros(p.nr), np.zeros(p.nr))
    for k in range(3):
        gw = list(zeros)
        gw[k] = (rng.standard_normal((p.nz, p.nr)) / nscale if k == 0
                 else rng.standard_normal(p.nr))
        gT = orc.field_chain_adjoint(p, c, p.T, *gw)
        picks = np.argsort(np.abs(gT).ravel())[::-1][:6]
        for flat in picks:
            j, i = divmod(int(flat), p.nr)
            h = 1e-4 * p.T[j, i]
            Tp, Tm = p.T.copy(), p.T.copy()
            Tp[j, i] += h
            Tm[j, i] -= h
            fd = (loss_and_weights(orc, p, c, Tp, gw) - loss_and_weights(orc, p, c, Tm, gw)) / (2 * h)
            assert gT[j, i] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(gT).max()), (k, j, i)


def chain_fields(orc, p, c, T):
    out = orc.field_chain(p, c, T)
    return p.replace(T=np.asarray(T, dtype=np.float64), n_h2=out["n_h2"], h_lo=out["h_lo"],
                     h_hi=out["h_hi"])


def test_render_through_the_chain_matches_central_differences(orc):
    """L(T) = sum g * render(chain(T)): dL/dT = the render adjoint's dT plus the chain adjoint
    of the render adjoint's dn, dh_lo, dh_hi, against central differences of the composition
    at the nodes where the gradient is largest."""
    p, rng = chain_problem(nr=12, nz=9, seed=5)
    p = p.replace(nx=8, ny=8, v_kms=np.linspace(-3.0, 3.0, 6), n_samples=48, half_fov_au=330.0)
    c = synth.chain_params(p)
    q = chain_fields(orc, p, c, p.T)
    cube0 = orc.render(q)
    g = rng.standard_normal(cube0.shape) / np.abs(cube0).max()
    _, gr = orc.render_adjoint(q, g)
    gT = gr["T"] + orc.field_chain_adjoint(p, c, p.T, gr["n_h2"], gr["h_lo"], gr["h_hi"])
    loss = lambda T: float((g * orc.render(chain_fields(orc, p, c, T))).sum())
    picks = np.argsort(np.abs(gT).ravel())[::-1][:8]
    for flat in picks:
        j, i = divmod(int(flat), p.nr)
        h = 1e-4 * p.T[j, i]
        Tp, Tm = p.T.copy(), p.T.copy()
        Tp[j, i] += h
        Tm[j, i] -= h
        fd = (loss(Tp) - loss(Tm)) / (2 * h)
        assert gT[j, i] == pytest.approx(fd, rel=1e-4, abs=1e-6 * np.abs(gT).max()), (j, i)
