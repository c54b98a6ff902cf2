"""Pins of the oracle's reverse mode through the neural field (no GPU).

- Central finite differences of the oracle's own FP64 neural-field render, for weights and
  biases of every layer and for grid nodes under the modulation.
- A network whose output layer is zero leaves the fields unmodulated: the node gradients
  must equal those of the grid-only adjoint, and no gradient reaches the hidden layers.
- The output biases shift every sample's outputs alike, so (bilinear weights summing to one)
  dL/db_out = (sum_a T_a dL/dT_a, sum_a n_a dL/dn_a, h_s sum_i dL/dh_lo_i, h_s sum_i dL/dh_hi_i)
  over the grid nodes a and radii i, for any network.
"""

import numpy as np
import pytest

from paper_2509_03623_b300 import synth
from tests.test_oracle_adjoint import small_problem


def small_net(seed=3):
    """A narrow network (generic dims: 8 features, 2 x 16 SiLU, 4 outputs) with non-zero
    biases and an output layer strong enough that every output matters."""
    w = synth.mlp_weights(seed, n_freq=4, width=16, hidden=2, sigma_b=1.5, out_gain=0.5)
    rng = np.random.default_rng(seed + 10)
    w.b = [rng.uniform(-0.2, 0.2, size=b.shape) for b in w.b]
    w.W = [x.astype(np.float64) for x in w.W]
    w.h_scale = 0.02
    return w


def loss(orc, p, w, G):
    return float((orc.render_mlp(p, w) * G).sum())


def perturbed(w, kind, l, idx, h):
    import copy
    v = copy.deepcopy(w)
    arr = (v.W if kind == "W" else v.b)[l]
    arr = np.array(arr, dtype=np.float64)
    arr.flat[idx] += h
    (v.W if kind == "W" else v.b)[l] = arr
    return v


def test_mlp_adjoint_vs_central_differences(orc):
    p = small_problem(2)
    w = small_net()
    rng = np.random.default_rng(9)
    G = rng.standard_normal((p.nch, p.ny, p.nx))
    _, g = orc.render_mlp_adjoint(p, w, G)
    checked = 0
    for kind in ("W", "b"):
        for l in range(len(w.W)):
            grad = (g["W"] if kind == "W" else g["b"])[l]
            flat = np.abs(grad).ravel()
            # the two largest entries of each array, and one random entry above 5% of its max
            cand = list(np.argsort(flat)[-2:])
            big = np.flatnonzero(flat >= 0.05 * flat.max())
            cand.append(int(rng.choice(big)))
            for idx in cand:
                h = 1e-4
                fd = (loss(orc, p, perturbed(w, kind, l, idx, h), G)
                      - loss(orc, p, perturbed(w, kind, l, idx, -h), G)) / (2 * h)
                assert fd == pytest.approx(grad.flat[idx], rel=2e-5, abs=1e-9 * flat.max()), \
                    (kind, l, int(idx))
                checked += 1
    # node gradients under the modulation (T and n_H2 enter through exp(o) factors)
    for field in ("T", "n_h2", "vturb"):
        flat = np.abs(g[field]).ravel()
        idx = int(np.argmax(flat))
        arr = getattr(p, field)
        h = 1e-4 * abs(arr.flat[idx])
        a, b = arr.copy(), arr.copy()
        a.flat[idx] += h
        b.flat[idx] -= h
        fd = (loss(orc, p.replace(**{field: a}), w, G)
              - loss(orc, p.replace(**{field: b}), w, G)) / (2 * h)
        assert fd == pytest.approx(g[field].flat[idx], rel=2e-5), field
        checked += 1
    assert checked == 2 * 3 * len(w.W) + 3


def test_zero_output_layer_reduces_to_grid_adjoint(orc):
    p = small_problem(3)
    w = small_net(4)
    w.W[-1] = np.zeros_like(w.W[-1])
    w.b[-1] = np.zeros_like(w.b[-1])
    rng = np.random.default_rng(2)
    G = rng.standard_normal((p.nch, p.ny, p.nx))
    cube_m, gm = orc.render_mlp_adjoint(p, w, G)
    cube_g, gg = orc.render_adjoint(p, G)
    np.testing.assert_allclose(cube_m, cube_g, rtol=1e-13, atol=1e-13 * np.abs(cube_g).max())
    for k in ("T", "n_h2", "vturb", "h_lo", "h_hi"):
        np.testing.assert_allclose(gm[k], gg[k], rtol=1e-10, atol=1e-12 * np.abs(gg[k]).max(),
                                   err_msg=k)
    # with o = 0 everywhere only the output-layer parameters see dL/d(outputs); the hidden
    # layers' gradients vanish because the zero output weights block the backward pass
    for l in range(len(w.W) - 1):
        assert np.abs(gm["W"][l]).max() == 0.0 and np.abs(gm["b"][l]).max() == 0.0
    assert np.abs(gm["b"][-1]).max() > 0.0


def test_output_bias_gradient_identities(orc):
    p = small_problem(4)
    w = small_net(5)
    rng = np.random.default_rng(6)
    G = rng.standard_normal((p.nch, p.ny, p.nx))
    _, g = orc.render_mlp_adjoint(p, w, G)
    want = np.array([(g["T"] * p.T).sum(), (g["n_h2"] * p.n_h2).sum(),
                     w.h_scale * g["h_lo"].sum(), w.h_scale * g["h_hi"].sum()])
    np.testing.assert_allclose(g["b"][-1], want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
