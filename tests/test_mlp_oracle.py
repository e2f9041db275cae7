"""Pins of the FP64 cost-model oracle (CPU): central finite differences of the
loss, the linear regime of the network as a plain matrix product, the dead
hidden layer, and the closed form of Adam's first step."""
import numpy as np
import pytest

from oracle import mlp


def rand_problem(seed, m=24):
    rng = np.random.default_rng(seed)
    p = mlp.he_uniform(seed)
    p[mlp.NPARAM - 1] = 0.3
    X = rng.random((m, mlp.IN))
    T = rng.standard_normal(m)
    return p, X, T


def test_param_count():
    assert mlp.NPARAM == 5313


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    p, X, T = rand_problem(seed)
    L, g = mlp.loss_and_grad(p, X, T)
    rng = np.random.default_rng(seed + 100)
    idx = rng.choice(mlp.NPARAM, 300, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 1087, 1088, 5247, 5248]])
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        Lp, _ = mlp.loss_and_grad(q, X, T)
        q[i] -= 2 * h
        Lm, _ = mlp.loss_and_grad(q, X, T)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_linear_regime_is_a_matrix_product():
    rng = np.random.default_rng(5)
    d = {"W1": rng.random((64, 16)), "b1": rng.random(64), "W2": rng.random((64, 64)),
         "b2": rng.random(64), "W3": rng.standard_normal(64), "b3": np.array(0.7)}
    p = mlp.pack(d)
    X = rng.random((9, 16))
    y, _ = mlp.forward(p, X)
    ref = ((X @ d["W1"].T + d["b1"]) @ d["W2"].T + d["b2"]) @ d["W3"] + 0.7
    assert np.allclose(y, ref, rtol=1e-13)


def test_dead_second_layer():
    p, X, T = rand_problem(7)
    d = mlp.unpack(p.copy())
    d = {k: np.array(v) for k, v in d.items()}
    d["W2"][:] = 0
    d["b2"][:] = -1.0
    p = mlp.pack(d)
    y, _ = mlp.forward(p, X)
    assert np.all(y == d["b3"])
    L, g = mlp.loss_and_grad(p, X, T)
    G = mlp.unpack(g)
    assert np.all(G["W1"] == 0) and np.all(G["b1"] == 0) and np.all(G["W3"] == 0)
    assert G["b3"] == pytest.approx(2 * np.mean(y - T), rel=1e-12)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(9)
    p = rng.standard_normal(mlp.NPARAM)
    g = rng.standard_normal(mlp.NPARAM)
    z = np.zeros(mlp.NPARAM)
    lr, eps = 1e-2, 1e-8
    p1, m1, m2 = mlp.adam_step(p, g, z, z, 1, lr=lr, eps=eps)
    # bias correction makes m_hat = g and v_hat = g^2 at t = 1
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)
