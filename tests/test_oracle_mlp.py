"""Pins of the oracle network (oracle/mlp.py): the hand-written backward pass against
central finite differences and against an independent autograd implementation; Adam's
first step against its closed form."""
import numpy as np
import pytest

import oracle.mlp as om


def _problem(F=7, H=128, B=33, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = om.init_params(F, H, seed=seed) + 0.05 * rng.normal(size=om.n_params(F, H))
    X = rng.normal(size=(B, F))
    y = rng.normal(size=B)
    return p, X, y


def test_gradient_matches_central_differences():
    F, H = 7, 128
    p, X, y = _problem(F, H)
    loss, g = om.loss_and_grad(p, X, y, F, H)
    rng = np.random.Generator(np.random.PCG64(11))
    idx = rng.choice(p.size, size=150, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (om.loss_and_grad(pp, X, y, F, H)[0] - om.loss_and_grad(pm, X, y, F, H)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_gradient_matches_autograd():
    torch = pytest.importorskip("torch")
    F, H = 5, 128
    p, X, y = _problem(F, H, B=17, seed=5)
    loss, g = om.loss_and_grad(p, X, y, F, H)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    shapes = [(H, F), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)]
    parts, o = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        parts.append(pt[o:o + n].reshape(sh))
        o += n
    W1, b1, W2, b2, W3, b3, w4, b4 = parts
    Xt, yt = torch.tensor(X), torch.tensor(y)
    out = torch.tanh(torch.tanh(torch.tanh(Xt @ W1.T + b1) @ W2.T + b2) @ W3.T + b3) @ w4 + b4[0]
    lt = torch.mean((out - yt) ** 2)
    lt.backward()
    assert float(lt) == pytest.approx(loss, rel=1e-13)
    np.testing.assert_allclose(pt.grad.numpy(), g, rtol=1e-10, atol=1e-14)


def test_adam_first_step_closed_form():
    g = np.array([1e-3, -2.0, 5.0, 0.0])
    p = np.zeros(4)
    p1, m, v = om.adam_step(p, g, np.zeros(4), np.zeros(4), step=1, lr=0.01, eps=1e-8)
    # bias-corrected moments equal g and g^2 after one step: update = lr g / (|g| + eps)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_training_reduces_loss():
    F, H = 4, 128
    rng = np.random.Generator(np.random.PCG64(2))
    X = rng.normal(size=(64, F))
    y = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2
    p = om.init_params(F, H, seed=1)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = om.loss_and_grad(p, X, y, F, H)[0]
    for step in range(1, 201):
        loss, g = om.loss_and_grad(p, X, y, F, H)
        p, m, v = om.adam_step(p, g, m, v, step, lr=3e-3)
    assert om.loss_and_grad(p, X, y, F, H)[0] < 0.05 * l0
