"""Pins of the warm-start network's FP64 oracle (oracle/mlp.py) against
things other than itself: the normal distribution's tabulated values, the
bfloat16 format's definition, central finite differences, and closed forms of
Adam's update."""
import math

import numpy as np

from oracle import mlp


def test_bf16_rounding_follows_the_format():
    # 8 significand bits: 1 + 2^-7 is the successor of 1; 1 + 2^-8 is the
    # midpoint and ties to the even neighbour 1; 1 + 3 * 2^-8 ties to 1 + 2^-6
    vals = np.array([1.0, 1 + 2 ** -7, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 0.0])
    want = np.array([1.0, 1 + 2 ** -7, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 0.0])
    np.testing.assert_array_equal(mlp.bf16_round(vals), want)


def test_gelu_against_normal_table_and_symmetry():
    # Phi(1) = 0.8413447460685429 (standard normal table)
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(-1.0) - (-1.0 + 0.8413447460685429)) < 1e-15
    assert mlp.gelu(0.0) == 0.0
    z = np.linspace(-6, 6, 101)
    # Phi(-z) = 1 - Phi(z)  =>  GELU(z) - GELU(-z) = z
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14)
    assert abs(mlp.gelu_grad(0.0) - 0.5) < 1e-16


def test_gelu_grad_against_finite_differences():
    z = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, atol=1e-9)


def test_scalar_network_by_hand():
    # y = w2 GELU(w1 x + b1) + b2 with scalars: the matrix code must agree
    w1, b1, w2, b2, x = 0.7, -0.2, -1.3, 0.4, 1.5
    z = w1 * x + b1
    want = w2 * 0.5 * z * (1 + math.erf(z / math.sqrt(2))) + b2
    params = [(np.array([[w1]]), np.array([b1])), (np.array([[w2]]), np.array([b2]))]
    y, _ = mlp.forward(params, np.array([[x]]))
    assert abs(y[0, 0] - want) < 1e-15


def _net(rng, dims):
    return [(rng.standard_normal((dims[i + 1], dims[i])) / math.sqrt(dims[i]), 0.1 * rng.standard_normal(dims[i + 1]))
            for i in range(len(dims) - 1)]


def test_backward_against_central_differences():
    rng = np.random.default_rng(7)
    dims = [5, 4, 3, 4, 6]  # three hidden layers, non-square everywhere
    params = _net(rng, dims)
    A0 = rng.standard_normal((7, dims[0]))
    T = rng.standard_normal((7, dims[-1]))

    def loss(ps):
        y, _ = mlp.forward(ps, A0)
        return mlp.mse(y, T)[0]

    Y, cache = mlp.forward(params, A0)
    _, dY = mlp.mse(Y, T)
    grads = mlp.backward(params, cache, dY)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            fd = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = loss(params)
                arr[idx] = old - h
                lm = loss(params)
                arr[idx] = old
                fd[idx] = (lp - lm) / (2 * h)
            np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_mse_gradient_against_finite_differences():
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((3, 4))
    T = rng.standard_normal((3, 4))
    _, g = mlp.mse(Y, T)
    h = 1e-6
    for idx in np.ndindex(Y.shape):
        Yp = Y.copy(); Yp[idx] += h
        Ym = Y.copy(); Ym[idx] -= h
        fd = (mlp.mse(Yp, T)[0] - mlp.mse(Ym, T)[0]) / (2 * h)
        assert abs(g[idx] - fd) < 1e-8


def test_adam_closed_forms():
    # first step with bias correction: -lr g / (|g| + eps); a constant
    # gradient keeps m_hat = g and v_hat = g^2, so every step is the same
    g = np.array([3.0, -0.5, 1e-3])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        p, m, v = mlp.adam_step(p, g, m, v, t, lr, eps=eps)
    np.testing.assert_allclose(p, -5 * lr * g / (np.abs(g) + eps), rtol=1e-12)


def test_standardiser_constant_column():
    X = np.array([[1.0, 5.0], [3.0, 5.0]])
    mu, sd = mlp.standardiser(X)
    np.testing.assert_allclose(mu, [2.0, 5.0])
    np.testing.assert_allclose(sd, [1.0, 1.0])
