"""Pins of the FP64 proposer reference: its gradients against central finite
differences of its own loss, GELU against the erf definition at known points,
and Adam against its closed-form first step."""
import math

import numpy as np

from oracle import mlp


def _tiny(seed=0):
    g = np.random.default_rng(seed)
    p, n, h, B = 5, 7, 6, 4
    params = [g.standard_normal((h, p)) * 0.5, g.standard_normal(h) * 0.1,
              g.standard_normal((h, h)) * 0.5, g.standard_normal(h) * 0.1,
              g.standard_normal((n, h)) * 0.5, g.standard_normal(n) * 0.1]
    Y = g.standard_normal((B, p))
    T = (g.random((B, n)) < 0.3).astype(float)
    return params, Y, T


def test_gradients_match_finite_differences():
    params, Y, T = _tiny()
    z, cache = mlp.forward(params, Y)
    grads = mlp.backward(params, cache, z, T)
    h = 1e-6
    for k, P in enumerate(params):
        num = np.zeros_like(P)
        it = np.nditer(P, flags=["multi_index"])
        for _ in it:
            ix = it.multi_index
            old = P[ix]
            P[ix] = old + h
            lp = mlp.loss(mlp.forward(params, Y)[0], T)
            P[ix] = old - h
            lm = mlp.loss(mlp.forward(params, Y)[0], T)
            P[ix] = old
            num[ix] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(grads[k], num, rtol=1e-6, atol=1e-9)


def test_gelu_and_its_derivative():
    assert mlp.gelu(np.array(0.0)) == 0.0
    x = np.array([1.0, -1.0, 2.5])
    phi = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in x]))
    np.testing.assert_allclose(mlp.gelu(x), x * phi, rtol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h),
                               rtol=1e-8)


def test_loss_is_bce_with_logits():
    z = np.array([[0.0, 2.0, -3.0]])
    t = np.array([[1.0, 0.0, 1.0]])
    s = 1 / (1 + np.exp(-z))
    bce = -(t * np.log(s) + (1 - t) * np.log(1 - s)).sum()
    assert abs(mlp.loss(z, t) - bce) < 1e-12


def test_adam_first_step_moves_each_weight_by_lr_times_sign():
    params = [np.array([1.0, -2.0, 3.0])]
    grads = [np.array([0.5, -4.0, 1e-3])]
    p, _, _ = mlp.adam_step([params[0].copy()], grads, [np.zeros(3)], [np.zeros(3)], 1, lr=0.01)
    np.testing.assert_allclose(p[0], params[0] - 0.01 * np.sign(grads[0]), rtol=0, atol=1e-7)
