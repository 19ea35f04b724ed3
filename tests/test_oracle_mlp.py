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


def _hand():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mlp_hand.json")))
    flat = np.concatenate([np.ravel(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float64)
    return g, flat


def test_forward_matches_hand_worked_network():
    """The 2-3-3-2 network of tests/golden/mlp_hand.json, worked by hand: both
    hidden layers have negative pre-activations (and a zero one), so the
    outputs pin where the ReLUs sit and which way each matrix is applied."""
    g, flat = _hand()
    y, (x, z1, a1, z2, a2) = mlp.forward(flat, g["x"], g["din"], g["h1"], g["h2"])
    np.testing.assert_array_equal(z1, np.array(g["z1"], np.float64))
    np.testing.assert_array_equal(z2, np.array(g["z2"], np.float64))
    np.testing.assert_array_equal(y, np.array(g["y"], np.float64))
    l = mlp.loss(flat, g["x"], g["t_reg"], g["t_cls"], g["din"], g["h1"], g["h2"])
    exp = (0.0625 + np.log1p(np.exp(-3.25)) + 0.0625 + np.log1p(np.exp(-2.25))) / 2
    assert abs(l - exp) < 1e-15


def test_adam_first_steps_closed_form():
    """From zero moments, the bias-corrected moments of step 1 are exactly g
    and g^2, so the step is lr * g / (|g| + eps); with the same gradient again,
    step 2's corrected moments are g and g^2 once more."""
    g = np.array([0.5, -2.0, 1e-3, 0.0, -7.0])
    th0 = np.array([0.1, -0.2, 0.3, 0.4, -0.5])
    lr = 0.01
    th1, m1, v1 = mlp.adam_step(th0, np.zeros(5), np.zeros(5), g, 1, lr)
    np.testing.assert_allclose(th1, th0 - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)
    th2, m2, v2 = mlp.adam_step(th1, m1, v1, g, 2, lr)
    np.testing.assert_allclose(th2, th1 - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m2, 0.19 * g, rtol=1e-14)
    np.testing.assert_allclose(v2, 0.001999 * g * g, rtol=1e-12)


def test_standardise_definition():
    x = np.array([[1.0, 10.0, 3.0], [3.0, 10.0, -3.0], [5.0, 10.0, 0.0]])
    mu, sd, xs = mlp.standardise(x)
    np.testing.assert_allclose(mu, [3.0, 10.0, 0.0])
    np.testing.assert_allclose(sd, [np.sqrt(8.0 / 3.0), 1e-6, np.sqrt(6.0)])
    np.testing.assert_allclose(xs[:, 0], [-2 / np.sqrt(8 / 3), 0, 2 / np.sqrt(8 / 3)])
