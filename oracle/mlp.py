"""FP64 oracle of the dense MLPs (dynamics surrogate and policy).

TEST INFRASTRUCTURE ONLY: used by tests/ and never by the product path.

An MLP of L layers computes z_l = W_l x_l + b_l, x_{l+1} = act_l(z_l); hidden
layers share one activation, the last layer has its own.  ELU is the paper's
network activation (App. E); SiLU is the surrogate's; tanh bounds the policy's
actions.  The loss of training is the mean squared error over batch and
outputs.  Everything is float64 numpy; a matrix product is the library's.
"""
from __future__ import annotations

import numpy as np

NONE, ELU, SILU, TANH = 0, 1, 2, 3


def act(z, kind):
    if kind == ELU:
        return np.where(z > 0, z, np.expm1(np.minimum(z, 0)))
    if kind == SILU:
        return z / (1.0 + np.exp(-z))
    if kind == TANH:
        return np.tanh(z)
    return z


def act_grad(z, kind):
    if kind == ELU:
        return np.where(z > 0, 1.0, np.exp(np.minimum(z, 0)))
    if kind == SILU:
        s = 1.0 / (1.0 + np.exp(-z))
        return s * (1.0 + z * (1.0 - s))
    if kind == TANH:
        return 1.0 - np.tanh(z) ** 2
    return np.ones_like(z)


def forward(params, x, hidden, out, keep=False):
    """params: list of (W [out, in], b [out]).  Returns y (and the per-layer
    inputs and pre-activations when keep)."""
    xs, zs = [np.asarray(x, np.float64)], []
    for l, (W, b) in enumerate(params):
        z = xs[-1] @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        zs.append(z)
        xs.append(act(z, out if l == len(params) - 1 else hidden))
    return (xs[-1], xs, zs) if keep else xs[-1]


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def backward(params, x, t, hidden, out):
    """Gradients of the mean squared error: list of (dW, db) per layer."""
    y, xs, zs = forward(params, x, hidden, out, keep=True)
    B, n = y.shape
    dA = 2.0 * (y - np.asarray(t, np.float64)) / (B * n)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        dZ = dA * act_grad(zs[l], out if l == len(params) - 1 else hidden)
        grads[l] = (dZ.T @ xs[l], dZ.sum(0))
        dA = dZ @ np.asarray(params[l][0], np.float64)
    return grads
