"""Pins of the FP64 MLP oracle: central finite differences of its own loss
(an independent check of the hand-written chain rule), and closed forms for a
network whose hidden layers are switched off."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    din, h1, h2, n = 5, 7, 6, 9
    flat = rng.standard_normal(mlp.num_params(din, h1, h2)) * 0.5
    x = rng.standard_normal((n, din))
    tr = rng.standard_normal(n)
    tc = (rng.random(n) < 0.5).astype(float)
    _, g = mlp.loss_grad(flat, x, tr, tc, din, h1, h2)
    h = 1e-6
    for k in range(len(flat)):
        e = np.zeros_like(flat)
        e[k] = h
        fd = (mlp.loss(flat + e, x, tr, tc, din, h1, h2) - mlp.loss(flat - e, x, tr, tc, din, h1, h2)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_zero_weights_closed_form():
    """With all weights and hidden biases zero the outputs equal b3: the loss
    is mean (b30 - t)^2 + log(1 + e^b31) - t_cls b31 and only b3 has gradient."""
    din, h1, h2 = 3, 4, 4
    flat = np.zeros(mlp.num_params(din, h1, h2))
    flat[-2:] = [0.5, 0.0]
    x = np.ones((2, din))
    tr = np.array([1.0, 2.0])
    tc = np.array([1.0, 0.0])
    l, g = mlp.loss_grad(flat, x, tr, tc, din, h1, h2)
    exp = ((0.5 - 1.0) ** 2 + (0.5 - 2.0) ** 2) / 2 + np.log(2.0)
    assert abs(l - exp) < 1e-12
    assert np.all(g[:-2] == 0.0)
    assert abs(g[-2] - (2 * (0.5 - 1.0) + 2 * (0.5 - 2.0)) / 2) < 1e-12
    assert abs(g[-1] - ((0.5 - 1.0) + (0.5 - 0.0)) / 2) < 1e-12
