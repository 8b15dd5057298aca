"""CPU reference of the pivot-proposer network (TEST INFRASTRUCTURE ONLY, like the rest of
``oracle``: imported by tests/ only, never by the library or the benchmark).

Not in the paper: a small multilayer perceptron that scores candidate rows and columns of a Pi
block (the learned proposer of the pivot search). Layout of the flat FP32 parameter vector, for
F inputs and H = 128 hidden units per layer (two hidden layers, ReLU, one logit):
    W1 (H x F), b1 (H), W2 (H x H), b2 (H), W3 (H), b3 (1)
Forward:  h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  z = W3 . h2 + b3.
Loss: mean over samples of w_s * BCE(sigmoid(z_s), y_s), with w_s = pos_weight for positives
and 1 otherwise; BCE with logits = max(z, 0) - z y + log(1 + exp(-|z|)).
Adam (Kingma and Ba, 2015) with bias correction.

Pins (tests/test_oracle_mlp.py): gradients against central finite differences of the loss,
a one-hidden-unit case worked by hand, and the Adam step against its closed form.
"""

from __future__ import annotations

import numpy as np

H = 128


def n_params(F: int, h: int = H) -> int:
    return h * F + h + h * h + h + h + 1


def unpack(p, F: int, h: int = H):
    p = np.asarray(p)
    o = 0
    W1 = p[o:o + h * F].reshape(h, F); o += h * F
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    W3 = p[o:o + h]; o += h
    b3 = p[o:o + 1]; o += 1
    return W1, b1, W2, b2, W3, b3


def init(seed: int, F: int, h: int = H):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from numpy's PCG64 generator."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, (h, F)) * np.sqrt(6.0 / F), np.zeros(h),
             rng.uniform(-1, 1, (h, h)) * np.sqrt(6.0 / h), np.zeros(h),
             rng.uniform(-1, 1, h) * np.sqrt(6.0 / h), np.zeros(1)]
    return np.concatenate([x.ravel() for x in parts]).astype(np.float32)


def forward(p, X, F: int, h: int = H):
    """Logits z (n,) and the cache for backward, in float64 for a reference free of FP32 rounding."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(t, dtype=np.float64) for t in unpack(p, F, h)]
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0)
    z = h2 @ W3 + b3[0]
    return z, (X, a1, h1, a2, h2)


def loss_grad(p, X, y, F: int, pos_weight: float = 1.0, h: int = H):
    """Mean weighted BCE-with-logits loss and its gradient (same layout as p)."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(t, dtype=np.float64) for t in unpack(p, F, h)]
    z, (Xd, a1, h1, a2, h2) = forward(p, X, F, h)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    w = np.where(y > 0.5, pos_weight, 1.0)
    loss = float(np.sum(w * (np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))) / n)
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = w * (sig - y) / n
    dW3 = h2.T @ dz
    db3 = np.array([dz.sum()])
    dh2 = np.outer(dz, W3) * (a2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    dW1 = dh1.T @ Xd
    db1 = dh1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3, db3])
    return loss, g


def adam(p, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step (t >= 1); returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
