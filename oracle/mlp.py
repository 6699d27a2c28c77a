"""Oracle of the task-cost MLP: FP64 forward pass, loss, gradient and Adam step.

TEST INFRASTRUCTURE ONLY: the library never imports this module.

The model predicts the (standardised) log running time of a work unit from its
features. Parameters, in this order in one flat vector:
    W1 [H x F], b1 [H], W2 [H x H], b2 [H], w3 [H], b3 [1]
Forward, per sample x (already standardised):
    h1 = tanh(W1 x + b1);  h2 = tanh(W2 h1 + b2);  y = w3 . h2 + b3
Loss over n samples with targets t (standardised):  L = (1/n) sum (y - t)^2.
Adam (Kingma & Ba, 2015) with bias correction:
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
    theta <- theta - lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)
"""
from __future__ import annotations

import numpy as np


def n_params(F: int, H: int) -> int:
    return H * F + H + H * H + H + H + 1


def unpack(theta, F: int, H: int):
    theta = np.asarray(theta, np.float64)
    o = 0
    W1 = theta[o:o + H * F].reshape(H, F); o += H * F
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def forward(theta, X, F: int, H: int):
    W1, b1, W2, b2, w3, b3 = unpack(theta, F, H)
    X = np.asarray(X, np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss_and_grad(theta, X, t, F: int, H: int):
    W1, b1, W2, b2, w3, b3 = unpack(theta, F, H)
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    n = X.shape[0]
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ w3 + b3
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / n
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, w3) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return L, g


def adam_step(theta, m, v, g, k: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def standardise(X):
    """Per-feature mean and standard deviation (population); a constant feature gets sd 1."""
    X = np.asarray(X, np.float64)
    mu = X.mean(0)
    sd = X.std(0)
    sd = np.where(sd > 0, sd, 1.0)
    return mu, sd
