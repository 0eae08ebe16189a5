"""Pins of the surrogate oracle (oracle/mlp.py): backpropagation against central
finite differences, the forward pass against its small-weight linearisation and
its symmetries, Adam against its constant-gradient closed form, the
initialisation against the Glorot bound."""
import math

import numpy as np
import pytest

from oracle import mcmc, mlp


def _random_params(seed):
    return np.random.default_rng(seed).uniform(-0.3, 0.3, mlp.NPAR)


def test_layout_counts():
    assert mlp.NPAR == 4 * 128 + 128 + 128 * 128 + 128 + 128 + 1 == 17281
    W1, b1, W2, b2, W3, b3 = mlp.unpack(np.arange(mlp.NPAR, dtype=float))
    assert W1[1, 0] == 128 and b1[0] == 512 and W2[0, 1] == 641 and W2[1, 0] == 640 + 128
    assert b2[0] == 17024 and W3[0] == 17152 and b3 == 17280
    assert np.array_equal(mlp.pack(W1, b1, W2, b2, W3, b3), np.arange(mlp.NPAR))


def test_backprop_matches_central_finite_differences():
    gen = np.random.default_rng(2)
    p = _random_params(1)
    xn = gen.normal(size=(16, 4))
    tn = gen.normal(size=16)
    loss, g = mlp.loss_grad(p, xn, tn)
    idx = np.concatenate([gen.choice(mlp.NPAR, 300, replace=False),
                          [0, 511, 512, 639, 640, 17023, 17024, 17151, 17152, 17280]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, xn, tn)[0] - mlp.loss_grad(pm, xn, tn)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(abs(g[i]), 1e-2 * np.max(np.abs(g))), i


def test_forward_linearises_to_matrix_product():
    # Zero biases and weights of scale s: f(x) = s^3 x W1 W2 W3 + O(s^5).
    gen = np.random.default_rng(8)
    W1, W2, W3 = gen.normal(size=(4, 128)), gen.normal(size=(128, 128)), gen.normal(size=128)
    s = 1e-3
    p = mlp.pack(s * W1, np.zeros(128), s * W2, np.zeros(128), s * W3, 0.0)
    x = gen.normal(size=(5, 4))
    f, _ = mlp.forward(p, x)
    lin = x @ W1 @ W2 @ W3
    assert np.max(np.abs(f / s**3 - lin)) < 1e-4 * np.max(np.abs(lin))


def test_hidden_unit_permutations_and_odd_symmetry():
    gen = np.random.default_rng(4)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(_random_params(3))
    x = gen.normal(size=(7, 4))
    f0, _ = mlp.forward(mlp.pack(W1, b1, W2, b2, W3, b3), x)
    P, Q = gen.permutation(128), gen.permutation(128)
    f1, _ = mlp.forward(mlp.pack(W1[:, P], b1[P], W2[P][:, Q], b2[Q], W3[Q], b3), x)
    assert np.max(np.abs(f1 - f0)) < 1e-13
    fT, _ = mlp.forward(mlp.pack(W1, b1, W2.T, b2, W3, b3), x)
    assert np.max(np.abs(fT - f0)) > 1e-3       # a transposed W2 is caught
    z = np.zeros(128)
    podd = mlp.pack(W1, z, W2, z, W3, 0.0)
    assert np.max(np.abs(mlp.forward(podd, -x)[0] + mlp.forward(podd, x)[0])) < 1e-14


def test_adam_constant_gradient_closed_form():
    # With a constant gradient the bias-corrected moments are g and g^2 at every
    # step, so each step moves p by -lr g / (|g| + eps).
    gen = np.random.default_rng(6)
    g = gen.normal(size=50) * 10.0 ** gen.uniform(-6, 2, 50)
    p0 = gen.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    lr = 1e-3
    for t in range(1, 6):
        p, m, v = mlp.adam_step(p, g, m, v, t, lr)
        want = p0 - t * lr * g / (np.abs(g) + mlp.ADAM_EPS)
        assert np.max(np.abs(p - want)) < 1e-15 * t + 1e-15


def test_init_is_glorot_uniform_from_philox():
    p = mlp.init_params(42)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    for W, a in ((W1, math.sqrt(6 / 132)), (W2, math.sqrt(6 / 256)), (W3, math.sqrt(6 / 129))):
        assert np.max(np.abs(W)) <= a
        assert abs(W.var() - a * a / 3) < 6 * a * a * math.sqrt(4 / 45 / W.size)
    assert not b1.any() and not b2.any() and b3 == 0.0
    w = mcmc.philox((700, 0, mlp.INIT_STREAM, 0), mcmc.seed_key(42))
    assert p[700] == (2 * mcmc.u52(w[0], w[1]) - 1) * math.sqrt(6 / 256)
    assert np.array_equal(p, mlp.init_params(42)) and not np.array_equal(p, mlp.init_params(43))


def test_batch_rows():
    assert np.array_equal(mlp.batch_rows(1, 0, 10, 10), np.arange(10))
    r = mlp.batch_rows(1, 3, 4000, 10000)
    assert len(r) == 4000 and r.min() >= 0 and r.max() <= 9999
    assert np.all(np.abs(np.bincount(r // 1000, minlength=10) / 400 - 1) < 0.25)
    assert not np.array_equal(r, mlp.batch_rows(1, 4, 4000, 10000))


def test_training_fits_a_smooth_function():
    gen = np.random.default_rng(12)
    psi = gen.normal(size=(512, 4))
    y = -np.sum(psi**2, axis=1) + psi[:, 0] * psi[:, 1] + 1000.0
    p0 = mlp.init_params(5)
    p, norm, losses = mlp.train(p0, psi, y, steps=300, batch=512, lr=3e-3, seed=5)
    assert losses[-1] < 0.02 * losses[0]
    pred = mlp.predict(p, norm, psi)
    assert np.sqrt(np.mean((pred - y) ** 2)) < 0.2 * y.std()
