"""FP64 oracle of the learned predictor's MLP (test infrastructure only).

Network: x -> relu(W1 x + b1) -> relu(W2 . + b2) -> W3 . + b3 = y (2 outputs).
Loss over n rows: mean_i [ (y_i0 - t_reg_i)^2 + softplus(y_i1) - t_cls_i y_i1 ]
(squared error on the budget head, binary cross-entropy with logits on the
route head).  Parameters are one flat vector W1[h1][din] b1 W2[h2][h1] b2
W3[2][h2] b3, the layout of the library's predictor.  Plain numpy in float64;
the backward pass is the chain rule written out layer by layer.  Training is
Adam on standardised inputs; `standardise` and `adam_step` state both steps.
"""
from __future__ import annotations

import numpy as np


def unpack(flat, din, h1, h2):
    flat = np.asarray(flat, np.float64)
    o = 0
    W1 = flat[o:o + h1 * din].reshape(h1, din); o += h1 * din
    b1 = flat[o:o + h1]; o += h1
    W2 = flat[o:o + h2 * h1].reshape(h2, h1); o += h2 * h1
    b2 = flat[o:o + h2]; o += h2
    W3 = flat[o:o + 2 * h2].reshape(2, h2); o += 2 * h2
    b3 = flat[o:o + 2]; o += 2
    assert o == len(flat)
    return W1, b1, W2, b2, W3, b3


def forward(flat, x, din, h1, h2):
    W1, b1, W2, b2, W3, b3 = unpack(flat, din, h1, h2)
    x = np.asarray(x, np.float64)
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3.T + b3
    return y, (x, z1, a1, z2, a2)


def loss(flat, x, t_reg, t_cls, din, h1, h2):
    y, _ = forward(flat, x, din, h1, h2)
    n = len(y)
    e = y[:, 0] - np.asarray(t_reg, np.float64)
    z = y[:, 1]
    t = np.asarray(t_cls, np.float64)
    sp = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))
    return float((e * e + sp - t * z).sum() / n)


def loss_grad(flat, x, t_reg, t_cls, din, h1, h2):
    W1, b1, W2, b2, W3, b3 = unpack(flat, din, h1, h2)
    y, (x, z1, a1, z2, a2) = forward(flat, x, din, h1, h2)
    n = len(y)
    t_reg = np.asarray(t_reg, np.float64)
    t_cls = np.asarray(t_cls, np.float64)
    dy = np.zeros_like(y)
    dy[:, 0] = 2.0 * (y[:, 0] - t_reg) / n
    dy[:, 1] = (1.0 / (1.0 + np.exp(-y[:, 1])) - t_cls) / n
    dW3 = dy.T @ a2
    db3 = dy.sum(0)
    dz2 = (dy @ W3) * (z2 > 0)
    dW2 = dz2.T @ a1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ x
    db1 = dz1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss(flat, x, t_reg, t_cls, din, h1, h2), g


def num_params(din, h1, h2):
    return h1 * din + h1 + h2 * h1 + h2 + 2 * h2 + 2


def standardise(x):
    """Per-feature mean and population standard deviation of the training rows
    (floored at 1e-6), and the rows standardised with them, in float64."""
    x = np.asarray(x, np.float64)
    mu = x.mean(0)
    sd = np.maximum(np.sqrt(np.maximum((x * x).mean(0) - mu * mu, 0.0)), 1e-6)
    return mu, sd, (x - mu) / sd


def adam_step(flat, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, "Adam: A Method for Stochastic
    Optimization", Algorithm 1) at step t >= 1, float64: first and second
    moment estimates, their bias corrections, then the parameter step.
    Returns (new parameters, new m, new v)."""
    flat, m, v, g = (np.asarray(a, np.float64) for a in (flat, m, v, g))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return flat - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
