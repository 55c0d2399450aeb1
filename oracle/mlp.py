"""FP64 CPU oracle of the learned warm-start network.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  It shares no code with
the GPU package and imports nothing from it.

The network is a multilayer perceptron: hidden layer l computes
Z_l = A_{l-1} W_l^T + b_l and A_l = GELU(Z_l) with the exact GELU
x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 (Hendrycks and Gimpel, "Gaussian Error
Linear Units", 2016); the output layer is affine.  The loss is the mean
squared error over all outputs of the batch, and parameters follow Adam with
bias correction (Kingma and Ba, "Adam: a method for stochastic
optimization", ICLR 2015, Algorithm 1).  Inputs and targets are standardised
column by column with statistics of the training set.

Precision: every product and sum here is FP64.  The GPU network keeps its
weights, the layer inputs and the back-propagated pre-activation gradients in
bfloat16; passing ``q=bf16_round`` makes the oracle round the same values at
the same points (round to nearest, ties to even), so that both compute the
same function.  With ``q=None`` nothing is rounded (used by the
finite-difference pins, which need the exact gradient of a smooth function).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (8 significand bits), ties to even: the
    value is first rounded to float32, then its low 16 bits are rounded
    away.  Returns FP64."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    """Exact GELU: z Phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def standardiser(X, floor=1e-12):
    """Column means and population standard deviations of X; a column whose
    deviation is at most floor * (1 + |mean|) gets deviation 1."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = np.sqrt(((X - mu) ** 2).mean(axis=0))
    sd = np.where(sd <= floor * (1.0 + np.abs(mu)), 1.0, sd)
    return mu, sd


def _q(q, a):
    return a if q is None else q(a)


def forward(params, A0, q=None):
    """params: list of (W [out x in], b [out]).  A0: layer-0 input [M x in]
    (already standardised).  Returns the output Y [M x out] and the cache for
    backward (pre-activations Z_l and layer inputs A_l)."""
    A = _q(q, A0)
    acts, zs = [A], []
    n = len(params)
    Y = None
    for l, (W, b) in enumerate(params):
        Z = A @ _q(q, W).T + b
        if l < n - 1:
            zs.append(Z)
            A = _q(q, gelu(Z))
            acts.append(A)
        else:
            Y = Z
    return Y, (zs, acts)


def mse(Y, T):
    """Mean squared error over all entries and its gradient dL/dY."""
    D = Y - T
    n = D.size
    return float((D * D).sum() / n), 2.0 * D / n


def backward(params, cache, dY, q=None):
    """Gradients (dW_l, db_l) of the loss for every layer, given dL/dY."""
    zs, acts = cache
    n = len(params)
    grads = [None] * n
    D = _q(q, dY)
    for l in range(n - 1, -1, -1):
        W = _q(q, params[l][0])
        grads[l] = (D.T @ acts[l], D.sum(axis=0))
        if l > 0:
            D = _q(q, (D @ W) * gelu_grad(zs[l - 1]))
    return grads


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of parameter p with gradient g at step t >= 1 (returns
    new p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train_step(params, moments, t, A0, T, lr, q=None):
    """Forward, loss, backward and Adam on every parameter.  moments: list of
    ((mW, vW), (mb, vb)) per layer.  Returns (loss, new params, new moments,
    grads)."""
    Y, cache = forward(params, A0, q)
    loss, dY = mse(Y, T)
    grads = backward(params, cache, dY, q)
    new_p, new_m = [], []
    for (W, b), (gW, gb), ((mW, vW), (mb, vb)) in zip(params, grads, moments):
        W2, mW2, vW2 = adam_step(W, gW, mW, vW, t, lr)
        b2_, mb2, vb2 = adam_step(b, gb, mb, vb, t, lr)
        new_p.append((W2, b2_))
        new_m.append(((mW2, vW2), (mb2, vb2)))
    return loss, new_p, new_m, grads
