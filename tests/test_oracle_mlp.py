"""Pins of the FP64 learned-start network reference (oracle/mlp.py), no GPU."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def small_net(seed=0, sizes=(7, 6, 5, 4)):
    rng = np.random.default_rng(seed)
    W = [rng.normal(0, 0.6, (sizes[i + 1], sizes[i])) for i in range(len(sizes) - 1)]
    b = [rng.normal(0, 0.3, sizes[i + 1]) for i in range(len(sizes) - 1)]
    return M.MLP(W, b), rng


def test_gelu_matches_erf_table():
    # gelu(z) = z/2 (1 + erf(z/sqrt2)); erf values from the standard table.
    for z, erf_val in ((1.0, 0.6826894921370859), (2.0, 0.9544997361036416), (-0.5, -0.3829249225480262)):
        assert M.gelu(z) == pytest.approx(0.5 * z * (1 + erf_val), rel=1e-14)
        assert math.erf(z / math.sqrt(2)) == pytest.approx(erf_val, rel=1e-14)
    z = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.abs(fd - M.gelu_grad(z)).max() < 1e-8


def test_gradients_match_central_differences():
    net, rng = small_net()
    X = rng.normal(0, 1, (9, 7))
    Y = rng.normal(0, 1, (9, 4))
    loss, gW, gb = net.gradients(X, Y)
    assert loss == pytest.approx(net.loss(X, Y), rel=1e-15)
    h = 1e-6
    for l in range(len(net.W)):
        for idx in [(0, 0), (1, 2), (net.W[l].shape[0] - 1, net.W[l].shape[1] - 1)]:
            w0 = net.W[l][idx]
            net.W[l][idx] = w0 + h
            lp = net.loss(X, Y)
            net.W[l][idx] = w0 - h
            lm = net.loss(X, Y)
            net.W[l][idx] = w0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gW[l][idx]) <= 1e-6 * max(1e-3, abs(fd))
        for j in range(net.b[l].shape[0]):
            b0 = net.b[l][j]
            net.b[l][j] = b0 + h
            lp = net.loss(X, Y)
            net.b[l][j] = b0 - h
            lm = net.loss(X, Y)
            net.b[l][j] = b0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gb[l][j]) <= 1e-6 * max(1e-3, abs(fd))


def test_adam_first_step_is_lr_times_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -1e-3, 40.0])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    p0 = p[0].copy()
    M.adam_step(p, g, m, v, step=1, lr=1e-3)
    # With bias correction, m_hat = g and v_hat = g^2 on the first step.
    assert np.allclose(p[0] - p0, -1e-3 * np.sign(g[0]), rtol=1e-4)


def test_adam_descends_a_quadratic():
    rng = np.random.default_rng(3)
    target = rng.normal(0, 1, 5)
    p = [np.zeros(5)]
    m = [np.zeros(5)]
    v = [np.zeros(5)]
    for k in range(1, 4001):
        M.adam_step(p, [2 * (p[0] - target)], m, v, step=k, lr=1e-2)
    assert np.abs(p[0] - target).max() < 1e-3
