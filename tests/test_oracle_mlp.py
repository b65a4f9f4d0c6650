"""Pins of the learned-classifier oracle (oracle/mlp.py), no GPU.

* gradients against central finite differences of the loss (float64);
* the network with hand-set weights equals the piecewise-linear function it
  encodes (a closed form);
* the spline start passes through its knots and is linear between them (the
  closed form of a piecewise-linear interpolant), and gradient steps on the
  output layer lower the loss at every step (a convex quadratic with a step
  below 2/L); the trained predictions beat a constant guess;
* predictions are clamped to [0, P-1] (NaN -> 0).
"""
import numpy as np

from oracle import mlp


def _theta(seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.N_PARAMS)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.random(64)
    y = np.sort(rng.random(64))
    theta = _theta(2)
    loss, grad = mlp.loss_and_grad(theta, x, y)
    h = 1e-6
    idx = list(range(0, mlp.N_PARAMS, 7)) + [mlp.N_PARAMS - 1]
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num = (mlp.loss_and_grad(tp, x, y)[0] - mlp.loss_and_grad(tm, x, y)[0]) / (2 * h)
        assert abs(num - grad[i]) <= 1e-6 + 1e-5 * abs(num), i


def test_hand_set_network_is_its_piecewise_linear_function():
    # unit j of layer 1 is relu(x - j/32); layer 2 copies unit 0 and unit 16;
    # output = h2[0] - h2[1]  ==>  f(x) = relu(x) - relu(x - 1/2)
    W1 = np.ones(32)
    b1 = -np.arange(32) / 32.0
    W2 = np.zeros((32, 32))
    W2[0, 0] = 1.0
    W2[1, 16] = 1.0
    b2 = np.zeros(32)
    w3 = np.zeros(32)
    w3[0], w3[1] = 1.0, -1.0
    theta = np.concatenate([W1, b1, W2.ravel(), b2, w3, [0.0]])
    x = np.linspace(-1, 2, 301)
    y, _ = mlp.forward(theta, x)
    assert np.allclose(y, np.maximum(x, 0) - np.maximum(x - 0.5, 0))


def test_spline_start_interpolates_its_knots():
    rng = np.random.default_rng(3)
    keys = np.sort(np.concatenate([rng.normal(0, 1, 3000), rng.normal(8, 0.3, 1000)]))
    x = (keys - keys[0]) / (keys[-1] - keys[0])
    y = (np.arange(x.size) + 0.5) / x.size
    theta, kx, ky = mlp.spline_start(x, y)
    assert len(kx) == mlp.KNOTS
    f, _ = mlp.forward(theta, kx)
    assert np.allclose(f, ky, atol=1e-12)
    mid = (kx[:-1] + kx[1:]) / 2
    fm, _ = mlp.forward(theta, mid)
    assert np.allclose(fm, (ky[:-1] + ky[1:]) / 2, atol=1e-12)


def test_spline_start_merges_equal_x():
    x = np.array([0.0, 0.0, 0.0, 0.5, 0.5, 1.0])
    y = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.9])
    theta, kx, ky = mlp.spline_start(x, y)
    assert kx.tolist() == [0.0, 0.5, 1.0]
    f, _ = mlp.forward(theta, kx)
    assert np.allclose(f, ky)


def test_head_steps_lower_the_loss_and_beat_a_constant():
    rng = np.random.default_rng(5)
    keys = np.sort(np.concatenate([rng.normal(0, 1, 3000), rng.normal(8, 0.3, 1000)]))
    x = (keys - keys[0]) / (keys[-1] - keys[0])
    y = (np.arange(x.size) + 0.5) / x.size
    theta, _, _ = mlp.spline_start(x, y)
    losses = []
    for _ in range(32):
        loss, g = mlp.loss_and_grad(theta, x, y)
        losses.append(loss)
        theta = mlp.head_step(theta, g, 0.02)
    assert all(b < a for a, b in zip(losses, losses[1:]))
    P = 64
    true_b = np.minimum((y * P).astype(int), P - 1)
    pred = mlp.predict_bucket(theta, x, P)
    assert np.mean(np.abs(pred - true_b)) < np.mean(np.abs(P // 2 - true_b)) / 4


def test_head_step_moves_only_the_output_layer():
    theta = _theta(6)
    g = np.ones(mlp.N_PARAMS)
    t2 = mlp.head_step(theta, g, 0.5)
    assert np.array_equal(t2[:mlp.HEAD.start], theta[:mlp.HEAD.start])
    assert np.allclose(t2[mlp.HEAD], theta[mlp.HEAD] - 0.5)


def test_prediction_is_clamped():
    theta = np.zeros(mlp.N_PARAMS)
    theta[-1] = 5.0
    assert mlp.predict_bucket(theta, np.array([0.1]), 16).tolist() == [15]
    theta[-1] = -3.0
    assert mlp.predict_bucket(theta, np.array([0.1]), 16).tolist() == [0]
    theta[-1] = np.nan
    assert mlp.predict_bucket(theta, np.array([0.1]), 16).tolist() == [0]
