"""Pins for the CPU reference of the pivot-proposer network (oracle/mlp.py): its gradient against
central finite differences of its loss, a one-hidden-unit network worked out by hand, and Adam
against the closed form of its first step (|update| = lr for every parameter with g != 0)."""

import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("pos_weight", [1.0, 4.0])
def test_gradient_matches_finite_differences(pos_weight):
    rng = np.random.default_rng(0)
    F, h, n = 5, 6, 11
    p = mlp.init(3, F, h).astype(np.float64)
    X = rng.standard_normal((n, F))
    y = (rng.uniform(size=n) < 0.4).astype(float)
    loss, g = mlp.loss_grad(p, X, y, F, pos_weight, h)
    num = np.zeros_like(p)
    step = 1e-6
    for i in range(len(p)):
        e = np.zeros_like(p)
        e[i] = step
        lp, _ = mlp.loss_grad(p + e, X, y, F, pos_weight, h)
        lm, _ = mlp.loss_grad(p - e, X, y, F, pos_weight, h)
        num[i] = (lp - lm) / (2 * step)
    assert np.abs(num - g).max() <= 1e-7 * max(1.0, np.abs(g).max())


def test_one_hidden_unit_by_hand():
    # F = 1, h = 1: z = w3 relu(w2 relu(w1 x + b1) + b2) + b3
    F, h = 1, 1
    w1, b1, w2, b2, w3, b3 = 2.0, -1.0, 3.0, 0.5, -1.5, 0.25
    p = np.array([w1, b1, w2, b2, w3, b3])
    x, y = 1.5, 1.0
    a1 = w1 * x + b1          # 2.0
    a2 = w2 * a1 + b2         # 6.5
    z = w3 * a2 + b3          # -9.5
    z_ref, _ = mlp.forward(p, np.array([[x]]), F, h)
    assert z_ref[0] == pytest.approx(z)
    s = 1 / (1 + np.exp(-z))
    dz = s - y
    expect = np.array([dz * w3 * w2 * x, dz * w3 * w2, dz * w3 * a1, dz * w3, dz * a2, dz])
    loss, g = mlp.loss_grad(p, np.array([[x]]), np.array([y]), F, 1.0, h)
    assert loss == pytest.approx(np.log1p(np.exp(-z)))
    assert np.allclose(g, expect, rtol=1e-12)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(7)
    g = rng.standard_normal(7)
    g[2] = 0.0
    with np.errstate(invalid="ignore"):  # eps = 0 leaves 0/0 where g = 0
        q, m, v = mlp.adam(p, g, np.zeros(7), np.zeros(7), 1, lr=0.01, eps=0.0)
    step = p - q
    assert np.allclose(np.abs(step[g != 0]), 0.01) and np.all(np.sign(step[g != 0]) == np.sign(g[g != 0]))
    assert np.isnan(step[2]) or step[2] == 0.0


def test_layout_and_sizes():
    F = 7
    p = mlp.init(0, F)
    assert p.dtype == np.float32 and len(p) == mlp.n_params(F) == 128 * 7 + 128 + 128 * 128 + 128 + 128 + 1
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, F)
    assert W1.shape == (128, 7) and W2.shape == (128, 128) and W3.shape == (128,) and b3.shape == (1,)
