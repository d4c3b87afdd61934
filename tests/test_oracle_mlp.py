"""Pins for the oracle's warm-start network.

* gradients equal central finite differences of the loss (FP64, relative error <= 1e-6);
* the first Adam step from zero moments moves every parameter by lr * g / (|g| + eps)
  (closed form: the bias-corrected moments equal g and g^2);
* BF16 rounding: exact for values already representable, ties to even, error <= 2^-9 relative;
* feature / target / inject maps reproduce a profile that is linear in z exactly where the
  interpolation is exact, and the features of a uniform density are uniform.
"""
import numpy as np

import synth
from oracle import mlp, poisson

SIZES = (7, 11, 9, 5)


def test_gradients_match_finite_differences():
    g = np.random.default_rng(0)
    p = synth.mlp_init(3, SIZES).astype(float) + g.normal(scale=0.05, size=synth.mlp_init(3, SIZES).size)
    X = g.normal(size=(6, SIZES[0]))
    T = g.normal(size=(6, SIZES[3]))
    _, grad = mlp.loss_and_grads(p, SIZES, X, T)
    h = 1e-6
    idx = g.choice(p.size, 40, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        num = (mlp.loss_and_grads(p + e, SIZES, X, T)[0] - mlp.loss_and_grads(p - e, SIZES, X, T)[0]) / (2 * h)
        assert abs(num - grad[i]) <= 1e-6 * max(1e-3, abs(num)), (i, num, grad[i])


def test_first_adam_step_closed_form():
    g = np.random.default_rng(1)
    w = g.normal(size=50)
    grad = g.normal(size=50)
    w1, m, v = mlp.adam_step(w, np.zeros(50), np.zeros(50), grad, 1, 1e-3)
    np.testing.assert_allclose(w1, w - 1e-3 * grad / (np.abs(grad) + 1e-8), rtol=1e-12, atol=1e-15)


def test_bf16_rounding():
    x = np.array([1.0, 1.5, -2.25, 3.0e-3, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 123.456], np.float32)
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.5 and r[2] == -2.25
    assert r[4] == 1.0                       # tie -> even mantissa
    assert r[5] == np.float32(1 + 4 * 2 ** -8)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)


def test_profile_maps():
    grid = poisson.Grid(3, 2, 40, 1.0, 1.0, 8.0)
    rho = np.full(grid.shape, 5e6)
    f = mlp.features(grid, rho, n=32)
    assert np.allclose(f[2:-2], f[2])        # uniform away from the grounded ends
    z = np.arange(1, grid.nz) / grid.nz
    phi = np.broadcast_to((0.3 * z)[:, None, None], grid.shape)
    t = mlp.targets(grid, phi, n=16, scale=0.1)
    zj = (np.arange(16) + 0.5) / 16
    np.testing.assert_allclose(t[:-1], 3.0 * zj[:-1], rtol=1e-12)
    back = mlp.inject(grid, t, scale=0.1)[:, 0, 0]
    inner = (z > zj[0]) & (z < zj[-2])
    np.testing.assert_allclose(back[inner], 0.3 * z[inner], rtol=1e-12)


def test_profile_maps_hand_computed():
    """Three interior planes of two lateral points each, values worked out by hand: the lateral
    means are (1, 3, 5) x scale; the grounded planes add 0 at t = 0 and t = 4 (units of hz).
    Four samples sit at t = 0.5, 1.5, 2.5, 3.5, i.e. halfway between neighbouring planes."""
    grid = poisson.Grid(2, 1, 4, 1.0, 1.0, 4.0)
    phi = np.array([0.5, 1.5, 2.0, 4.0, 6.0, 4.0]).reshape(grid.shape) * 0.1   # means 0.1, 0.3, 0.5 V
    t = mlp.targets(grid, phi, n=4, scale=0.1)
    np.testing.assert_allclose(t, [0.5, 2.0, 4.0, 2.5], rtol=1e-14)
    t2 = mlp.targets(grid, phi, n=2, scale=0.1)                      # samples at t = 1 and t = 3
    np.testing.assert_allclose(t2, [1.0, 5.0], rtol=1e-14)
    # features: log10 of the donor density (m^-3), floored at 1e15, minus 21, over 6
    nd = np.array([1e20, 1e20, 1e22, 1e22, 1e12, 1e12]).reshape(grid.shape)
    f = mlp.features(grid, nd * mlp.Q_E, n=2)
    np.testing.assert_allclose(f, [(20 - 21) / 6, (15 - 21) / 6], rtol=1e-12)
    f4 = mlp.features(grid, nd * mlp.Q_E, n=4)
    expect = [np.log10(0.5e20), np.log10(0.5 * (1e20 + 1e22)), np.log10(0.5 * (1e22 + 1e12)), 15.0]
    np.testing.assert_allclose(f4, (np.array(expect) - 21) / 6, rtol=1e-12)
    # inject: samples at z/Lz = 1/4 and 3/4 land on planes 1 and 3; plane 2 is their mean
    back = mlp.inject(grid, np.array([2.0, -1.0]), scale=0.1)
    np.testing.assert_allclose(back[:, 0, 0], [0.2, 0.05, -0.1], rtol=1e-14)
    assert np.all(back == back[:, :1, :1])
