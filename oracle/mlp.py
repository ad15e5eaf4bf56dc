"""FP64 reference of the learned support proposer (test infrastructure only).

The proposer is a small MLP y (p) -> 512 -> 512 -> n with GELU activations and
sigmoid outputs, trained with binary cross-entropy on the multi-hot OMP support
of each signal; at inference the 2s atoms with the largest logits are the
candidate set of a restricted OMP.  This module states the network, its loss
and gradients, and the Adam update in plain numpy (float64), so the GPU
kernels can be checked against it; its own gradients are pinned by finite
differences in tests/test_oracle_mlp.py.

Conventions: activations are row-major (batch, features); weights W_l are
(out, in) and biases (out,):  a1 = Y W1^T + b1, h1 = gelu(a1),
a2 = h1 W2^T + b2, h2 = gelu(a2), z = h2 W3^T + b3.
GELU is the exact form 0.5 x (1 + erf(x / sqrt(2))).
Loss: mean over the batch of sum over atoms of softplus(z) - t z
(binary cross-entropy with logits, t in {0, 1}).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x * SQRT1_2))


def gelu_grad(x):
    """d gelu / dx = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x * SQRT1_2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def softplus(z):
    return np.logaddexp(0.0, z)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def forward(params, Y):
    """Returns (z, cache)."""
    W1, b1, W2, b2, W3, b3 = params
    a1 = Y @ W1.T + b1
    h1 = gelu(a1)
    a2 = h1 @ W2.T + b2
    h2 = gelu(a2)
    z = h2 @ W3.T + b3
    return z, (Y, a1, h1, a2, h2)


def loss(z, T):
    return float(np.mean(np.sum(softplus(z) - T * z, axis=1)))


def backward(params, cache, z, T):
    """Gradients of loss() with respect to (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    Y, a1, h1, a2, h2 = cache
    B = z.shape[0]
    dz = (sigmoid(z) - T) / B
    dW3 = dz.T @ h2
    db3 = dz.sum(axis=0)
    dh2 = dz @ W3
    da2 = dh2 * gelu_grad(a2)
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * gelu_grad(a1)
    dW1 = da1.T @ Y
    db1 = da1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) in place; t is the 1-based step count."""
    for k in range(len(params)):
        m[k] = b1 * m[k] + (1 - b1) * grads[k]
        v[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v


def multi_hot(idx, cnt, n):
    """(m, s) supports with counts -> (m, n) 0/1 targets."""
    m = idx.shape[0]
    T = np.zeros((m, n))
    for i in range(m):
        T[i, idx[i, :cnt[i]]] = 1.0
    return T
