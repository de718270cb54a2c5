"""Pins for oracle.mlp: central finite differences of the loss against the
backpropagated gradient for every parameter block, the softmax cross-entropy
gradient identity, and Adam's first step size."""
import numpy as np

from oracle import mlp


def _data(seed, B=7):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, mlp.N_IN)), rng.integers(0, mlp.N_OUT, size=B)


def test_gradient_matches_central_differences():
    theta = mlp.init_params(1)
    theta[mlp.N_PARAMS - mlp.N_OUT:] = np.random.default_rng(3).normal(size=mlp.N_OUT)  # nonzero b3
    x, y = _data(2)
    L, g = mlp.grad(theta, x, y)
    assert abs(L - mlp.loss(theta, x, y)) < 1e-14
    rng = np.random.default_rng(4)
    idx = rng.choice(mlp.N_PARAMS, size=200, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, x, y) - mlp.loss(tm, x, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_last_layer_gradient_is_softmax_minus_onehot():
    theta = mlp.init_params(5)
    x, y = _data(6, B=3)
    z, (_, _, _, h2) = mlp.forward(theta, x)
    sm = np.exp(z - z.max(1, keepdims=True))
    sm /= sm.sum(1, keepdims=True)
    _, g = mlp.grad(theta, x, y)
    gb3 = g[-mlp.N_OUT:]
    expect = (sm - np.eye(mlp.N_OUT)[y]).sum(0) / len(y)
    assert np.max(np.abs(gb3 - expect)) < 1e-14


def test_adam_first_step_has_learning_rate_size():
    theta = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    t2, m, v = mlp.adam_step(theta, np.zeros(5), np.zeros(5), g, 1, 0.01)
    nz = g != 0
    assert np.allclose(np.abs(t2[nz]), 0.01, rtol=1e-6) and t2[3] == 0
