"""GPU parity of the cost-model kernels (forward, backward, Adam) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_1910_08498_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def problem(seed, m):
    rng = np.random.default_rng(seed)
    p = mlp.he_uniform(seed)
    p[-1] = 0.25
    X = rng.random((m, 16))
    T = rng.standard_normal(m)
    return p, X, T


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m", [1, 31, 32, 33, 1000])
def test_forward(m):
    p, X, _ = problem(m, m)
    y = torch.empty(m, device="cuda")
    L.fr_mlp_forward(dev(p), dev(X), y)
    ref, _ = mlp.forward(p.astype(np.float32), X.astype(np.float32))
    got = y.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 2e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("m", [1, 33, 500])
def test_backward(m):
    p, X, T = problem(10 + m, m)
    p32, X32, T32 = (a.astype(np.float32) for a in (p, X, T))
    g = torch.empty(mlp.NPARAM, device="cuda")
    loss = torch.empty(1, device="cuda")
    L.fr_mlp_backward(dev(p32), dev(X32), dev(T32), g, loss)
    Lr, gr = mlp.loss_and_grad(p32, X32, T32)
    assert loss.item() == pytest.approx(Lr, rel=2e-5)
    got = g.cpu().numpy()
    assert np.max(np.abs(got - gr)) <= 2e-5 * max(1.0, np.max(np.abs(gr)))


def test_backward_deterministic():
    p, X, T = problem(3, 300)
    outs = []
    for _ in range(2):
        g = torch.empty(mlp.NPARAM, device="cuda")
        loss = torch.empty(1, device="cuda")
        L.fr_mlp_backward(dev(p), dev(X), dev(T), g, loss)
        outs.append(g.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_adam_steps():
    rng = np.random.default_rng(4)
    p = rng.standard_normal(mlp.NPARAM).astype(np.float32)
    pd, m1, m2 = dev(p), torch.zeros(mlp.NPARAM, device="cuda"), torch.zeros(mlp.NPARAM, device="cuda")
    pr, m1r, m2r = p.astype(np.float64), np.zeros(mlp.NPARAM), np.zeros(mlp.NPARAM)
    for t in range(1, 6):
        g = rng.standard_normal(mlp.NPARAM).astype(np.float32)
        L.fr_mlp_adam(pd, dev(g), m1, m2, t, lr=1e-2)
        pr, m1r, m2r = mlp.adam_step(pr, g.astype(np.float64), m1r, m2r, t, lr=1e-2)
    assert np.max(np.abs(pd.cpu().numpy() - pr)) <= 1e-5


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(6)
    X = rng.random((400, 16)).astype(np.float32)
    T = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 9]).astype(np.float32)
    ctx = L.fr_create(32)
    try:
        l0 = float(np.mean((T - T.mean()) ** 2))
        loss = L.fr_mlp_train(ctx, X, T, epochs=1500, lr=3e-3, seed=1)
        assert loss < 0.05 * l0
        p = L.fr_mlp_get(ctx)
        y, _ = mlp.forward(p, X)
        assert float(np.mean((y - T) ** 2)) == pytest.approx(loss, rel=1e-3)
    finally:
        L.fr_destroy(ctx)
