"""Pins of the MLP oracle: central finite differences of the loss, closed forms for
degenerate parameters, and the Adam recurrence written out for one coordinate."""
import math

import numpy as np
import pytest

from oracle import mlp as M

F, H = 12, 32


def _rand(seed, n=40):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, M.n_params(F, H))
    X = rng.normal(0, 1, (n, F))
    t = rng.normal(0, 1, n)
    return theta, X, t


@pytest.mark.parametrize("seed", range(3))
def test_gradient_vs_central_differences(seed):
    theta, X, t = _rand(seed)
    L, g = M.loss_and_grad(theta, X, t, F, H)
    rng = np.random.default_rng(100 + seed)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (M.loss_and_grad(tp, X, t, F, H)[0] - M.loss_and_grad(tm, X, t, F, H)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))


def test_constant_model_closed_form():
    """All weights zero: y = b3 for every sample, L = mean((b3 - t)^2), dL/db3 = 2 mean(b3 - t),
    and every other gradient entry vanishes except dL/dw3 (h2 = 0 makes it zero too)."""
    _, X, t = _rand(7)
    theta = np.zeros(M.n_params(F, H))
    theta[-1] = 0.37
    L, g = M.loss_and_grad(theta, X, t, F, H)
    assert math.isclose(L, float(np.mean((0.37 - t) ** 2)), rel_tol=1e-14)
    assert math.isclose(g[-1], 2 * float(np.mean(0.37 - t)), rel_tol=1e-12)
    assert np.all(g[:-1] == 0.0)


def test_forward_matches_loss_path():
    theta, X, t = _rand(3)
    y = M.forward(theta, X, F, H)
    L, _ = M.loss_and_grad(theta, X, t, F, H)
    assert math.isclose(L, float(np.mean((y - t) ** 2)), rel_tol=1e-14)


def test_adam_first_step_is_signed_lr():
    """With zero moments, the first bias-corrected Adam step moves each coordinate by
    lr * g / (|g| + eps), i.e. almost exactly lr against the gradient's sign."""
    theta = np.zeros(5)
    g = np.array([0.5, -2.0, 1e-3, 3.0, -1e-4])
    new, m, v = M.adam_step(theta, np.zeros(5), np.zeros(5), g, 1, 0.01)
    want = -0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(new, want, rtol=1e-12, atol=0)


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(0)
    X = rng.normal(0, 1, (256, F))
    t = np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.1 * X[:, 5]
    theta = rng.normal(0, 0.1, M.n_params(F, H))
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0, _ = M.loss_and_grad(theta, X, t, F, H)
    for k in range(1, 301):
        _, g = M.loss_and_grad(theta, X, t, F, H)
        theta, m, v = M.adam_step(theta, m, v, g, k, 0.01)
    L1, _ = M.loss_and_grad(theta, X, t, F, H)
    assert L1 < 0.1 * L0
