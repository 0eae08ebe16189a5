"""CPU oracle for the log-likelihood surrogate -- TEST INFRASTRUCTURE ONLY.

A 4 -> 128 -> 128 -> 1 perceptron with tanh hidden layers, trained by mean
squared error with Adam (Kingma & Ba, ICLR 2015), written as plain FP64 NumPy
matrix products and hand-written backpropagation.  The network maps the
log-rates Psi = log(theta) (SI A.1) to the snapshot log-likelihood; inputs and
targets are standardised with the training set's means and standard
deviations.  Only ``tests/`` and the CPU legs of ``bench.py`` may import it.

Parameter layout (one flat vector of 17,281 values, row-major, y = x W + b):
W1[4][128] at 0, b1[128] at 512, W2[128][128] at 640, b2[128] at 17,024,
W3[128] at 17,152, b3 at 17,280.

Parity status: pinned by ``tests/test_oracle_mlp.py`` -- backpropagation
against central finite differences, the forward pass against its small-weight
linearisation (the plain product x W1 W2 W3) and a hidden-unit permutation
symmetry, Adam against its constant-gradient closed form, the initialisation
against the Glorot bound and the Philox stream.
"""
from __future__ import annotations

import math

import numpy as np

from . import mcmc

D, H = 4, 128
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 0, 512, 640, 17024, 17152, 17280
NPAR = 17281
ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8
INIT_STREAM = 0x4D4C5000  # Philox counter word 2 of the weight initialisation


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(D, H), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H, H),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3], p[OFF_B3])


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2), np.ravel(W3),
                           np.atleast_1d(b3)]).astype(np.float64)


def init_params(seed: int):
    """Glorot-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)), zero
    biases.  The uniform for flat index i is the first 52-bit uniform of Philox
    block (i, 0, INIT_STREAM, 0) under the seed's key, mapped to (2u - 1) a."""
    key = mcmc.seed_key(seed)
    p = np.zeros(NPAR)
    for lo, hi, fi, fo in ((OFF_W1, OFF_B1, D, H), (OFF_W2, OFF_B2, H, H), (OFF_W3, OFF_B3, H, 1)):
        a = math.sqrt(6.0 / (fi + fo))
        for i in range(lo, hi):
            w = mcmc.philox((i, 0, INIT_STREAM, 0), key)
            p[i] = (2.0 * mcmc.u52(w[0], w[1]) - 1.0) * a
    return p


def fit_norm(psi, y):
    """Means and population standard deviations of inputs and targets (a zero
    deviation is replaced by 1)."""
    psi = np.asarray(psi, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    mx, sx = psi.mean(axis=0), psi.std(axis=0)
    my, sy = float(y.mean()), float(y.std())
    sx = np.where(sx > 0, sx, 1.0)
    return {"mu_x": mx, "sd_x": sx, "mu_y": my, "sd_y": sy if sy > 0 else 1.0}


def forward(p, xn):
    """Network output f(xn) and the hidden activations (standardised units)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    xn = np.atleast_2d(np.asarray(xn, dtype=np.float64))
    h1 = np.tanh(xn @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    return h2 @ W3 + b3, (xn, h1, h2)


def predict(p, norm, psi):
    """Surrogate log-likelihood at Psi in the data's units."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.float64))
    f, _ = forward(p, (psi - norm["mu_x"]) / norm["sd_x"])
    return norm["mu_y"] + norm["sd_y"] * f


def loss_grad(p, xn, tn):
    """Mean squared error L = (1/n) sum (f - t)^2 and dL/dp by backpropagation."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    tn = np.asarray(tn, dtype=np.float64)
    f, (x, h1, h2) = forward(p, xn)
    n = len(tn)
    r = f - tn
    loss = float(np.dot(r, r) / n)
    dy = 2.0 * r / n                       # dL/df
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * (1.0 - h2 * h2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (1.0 - h1 * h1)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(p, g, m, v, t: int, lr: float, beta1=ADAM_BETA1, beta2=ADAM_BETA2, eps=ADAM_EPS):
    """One Adam update (step t >= 1): moment averages, bias correction by
    1 - beta^t, step lr * mhat / (sqrt(vhat) + eps).  Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def batch_rows(seed: int, step: int, batch: int, n: int):
    """Rows of minibatch ``step``: all rows in order when batch >= n, else draws
    with replacement, row r taking floor(w * n / 2^32) of word 0 of Philox block
    (r, step, INIT_STREAM + 1, 0)."""
    if batch >= n:
        return np.arange(n)
    key = mcmc.seed_key(seed)
    return np.array([(mcmc.philox((r, step, INIT_STREAM + 1, 0), key)[0] * n) >> 32 for r in range(batch)])


def train(p, psi, y, steps: int, batch: int, lr: float, seed: int, norm=None, eps=ADAM_EPS):
    """Adam on the standardised data; returns (p, norm, losses)."""
    norm = norm or fit_norm(psi, y)
    xn = (np.asarray(psi, dtype=np.float64) - norm["mu_x"]) / norm["sd_x"]
    tn = (np.asarray(y, dtype=np.float64) - norm["mu_y"]) / norm["sd_y"]
    m = np.zeros(NPAR)
    v = np.zeros(NPAR)
    losses = []
    for s in range(steps):
        rows = batch_rows(seed, s, batch, len(tn))
        loss, g = loss_grad(p, xn[rows], tn[rows])
        p, m, v = adam_step(p, g, m, v, s + 1, lr, eps=eps)
        losses.append(loss)
    return p, norm, np.array(losses)
