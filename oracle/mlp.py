"""FP64 reference of the learned-start network -- TEST INFRASTRUCTURE ONLY.

The learned start is not in the paper: a small multilayer perceptron maps a column's loads to a
starting voltage for the fixed-point iteration.  This module is the plain double-precision
definition of that network, used to check the library's BF16 tensor-core forward and backward
kernels; only the tests and the benchmark's CPU leg use it.

Network (layer sizes n_0, ..., n_L):   a_0 = x,
    z_l = W_l a_{l-1} + b_l,   a_l = gelu(z_l)  for l < L,   y = z_L,
with gelu(z) = z/2 (1 + erf(z / sqrt 2)).  Loss: mean squared error over all outputs of the batch.
Optimiser: Adam (Kingma & Ba, 2015) with bias correction.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss against the analytic
gradients; gelu against tabulated erf values and its derivative against a finite difference;
Adam's first step moves every parameter by lr * sign(g) (up to eps).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)
INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


class MLP:
    """Weights W[l] (n_{l+1} x n_l) and biases b[l] (n_{l+1}) in float64."""

    def __init__(self, W, b):
        self.W = [np.array(w, dtype=np.float64) for w in W]
        self.b = [np.array(v, dtype=np.float64) for v in b]

    def forward(self, X):
        """X [B][n_0] -> (y [B][n_L], cache of (a_{l-1}, z_l) per layer)."""
        a = np.asarray(X, dtype=np.float64)
        cache = []
        L = len(self.W)
        for l in range(L):
            z = a @ self.W[l].T + self.b[l]
            cache.append((a, z))
            a = gelu(z) if l < L - 1 else z
        return a, cache

    def loss(self, X, Y):
        y, _ = self.forward(X)
        return float(np.mean((y - Y) ** 2))

    def gradients(self, X, Y):
        """Loss and its gradients with respect to every W[l] and b[l]."""
        y, cache = self.forward(X)
        n = y.size
        loss = float(np.mean((y - Y) ** 2))
        dz = 2.0 * (y - Y) / n
        gW = [None] * len(self.W)
        gb = [None] * len(self.W)
        for l in range(len(self.W) - 1, -1, -1):
            a_prev, z = cache[l]
            gW[l] = dz.T @ a_prev
            gb[l] = dz.sum(axis=0)
            if l > 0:
                da = dz @ self.W[l]
                dz = da * gelu_grad(cache[l - 1][1])
        return loss, gW, gb


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; `step` counts from 1."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= beta1
        mm += (1.0 - beta1) * g
        vv *= beta2
        vv += (1.0 - beta2) * g * g
        mhat = mm / (1.0 - beta1 ** step)
        vhat = vv / (1.0 - beta2 ** step)
        p -= lr * mhat / (np.sqrt(vhat) + eps)
