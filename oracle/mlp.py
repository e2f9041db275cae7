"""FP64 reference of the tuner's cost model -- TEST INFRASTRUCTURE ONLY.

A 16-64-64-1 multilayer perceptron with ReLU hidden layers, trained with the
mean-squared error L = (1/m) sum_r (y_r - t_r)^2 and Adam (Kingma & Ba, 2015,
Algorithm 1, with bias-corrected moments).  The parameter vector is laid out
as W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3 (W[out][in]).

Plain numpy in float64: forward pass, backward pass written out layer by layer
(the chain rule, no autograd), one Adam step.  Pinned in
tests/test_mlp_oracle.py by central finite differences, a linear-regime closed
form and the closed form of Adam's first step.
"""
from __future__ import annotations

import numpy as np

IN, H = 16, 64
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", ())]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, X):
    P = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"] + P["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(p, X, T):
    P = unpack(p)
    T = np.asarray(T, dtype=np.float64)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    m = y.shape[0]
    e = y - T
    L = float(np.sum(e * e) / m)
    dy = 2.0 * e / m                      # dL/dy
    g = {}
    g["W3"] = h2.T @ dy                   # dL/dW3
    g["b3"] = np.sum(dy)
    dh2 = np.outer(dy, P["W3"])           # dL/dh2
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def adam_step(p, grad, m1, m2, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    p = np.asarray(p, np.float64)
    m1 = b1 * np.asarray(m1, np.float64) + (1 - b1) * grad
    m2 = b2 * np.asarray(m2, np.float64) + (1 - b2) * grad * grad
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2


def he_uniform(seed: int):
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            fan_in = shape[-1]
            lim = np.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-lim, lim, size=shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)
