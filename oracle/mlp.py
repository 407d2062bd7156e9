"""Oracle of the surrogate network: FP64 forward, backward and Adam (test infrastructure only).

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may import this
module.  The network maps per-mode harmonic features to log(rate):

  h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3), y = w4 . h3 + b4
  loss = mean over the batch of (y - target)^2

Parameters are packed in one flat vector in the order W1 (H x F, row-major), b1 (H), W2 (H x H),
b2, W3 (H x H), b3, w4 (H), b4 (1) -- the layout the CUDA kernels use.  The backward pass is
the chain rule written out by hand (no autograd); the tests pin it against central finite
differences and against an independent autograd implementation.
"""
from __future__ import annotations

import numpy as np


def n_params(F: int, H: int = 128) -> int:
    return H * F + H + 2 * (H * H + H) + H + 1


def unpack(p, F, H=128):
    p = np.asarray(p, dtype=np.float64)
    o = 0

    def take(n, shape):
        nonlocal o
        v = p[o:o + n].reshape(shape)
        o += n
        return v
    W1 = take(H * F, (H, F))
    b1 = take(H, (H,))
    W2 = take(H * H, (H, H))
    b2 = take(H, (H,))
    W3 = take(H * H, (H, H))
    b3 = take(H, (H,))
    w4 = take(H, (H,))
    b4 = take(1, (1,))
    assert o == p.size
    return W1, b1, W2, b2, W3, b3, w4, b4


def init_params(F, H=128, seed=0):
    """Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_in, fan_out in ((F, H), (H, H), (H, H)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    lim = np.sqrt(6.0 / (H + 1))
    parts.append(rng.uniform(-lim, lim, size=H))
    parts.append(np.zeros(1))
    return np.concatenate(parts)


def forward(p, X, F, H=128):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p, F, H)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    h3 = np.tanh(h2 @ W3.T + b3)
    y = h3 @ w4 + b4[0]
    return y, (X, h1, h2, h3)


def loss_and_grad(p, X, target, F, H=128):
    """Mean-squared loss and its gradient with respect to the packed parameters."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p, F, H)
    y, (X, h1, h2, h3) = forward(p, X, F, H)
    B = X.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B                       # d loss / d y
    g_w4 = h3.T @ dy
    g_b4 = np.array([dy.sum()])
    d3 = np.outer(dy, w4) * (1.0 - h3 * h3)
    g_W3 = d3.T @ h2
    g_b3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * (1.0 - h2 * h2)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    g_W1 = d1.T @ X
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_W3.ravel(), g_b3, g_w4, g_b4])
    return loss, g


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
