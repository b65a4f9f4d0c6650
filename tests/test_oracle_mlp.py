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


def test_spline_start_is_balanced():
    """Each unit's three weights carry its output weight equally (|w1_j| =
    |W2_jj| = |w3_j|, the cube root of the plain interpolant's slope change);
    the function is the plain interpolant's (checked above at knots and
    midpoints), and the knots are -b1/w1."""
    rng = np.random.default_rng(4)
    x = np.sort(rng.random(500))
    y = (np.arange(500) + 0.5) / 500
    theta, kx, ky = mlp.spline_start(x, y)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(theta)
    on = w3 != 0
    assert on.sum() >= 8
    assert np.allclose(np.abs(W1[on]), np.abs(np.diag(W2))[on])
    assert np.allclose(np.abs(W1[on]), np.abs(w3[on]))
    slopes = np.diff(ky) / np.diff(kx)
    change = np.concatenate([[slopes[0]], np.diff(slopes)])
    assert np.allclose(W1[on] * np.diag(W2)[on] * w3[on], change[on[:len(change)]])
    assert np.allclose(-b1[on] / W1[on], kx[:on.sum()])


def test_descent_lowers_the_loss_moves_every_layer_and_beats_a_constant():
    rng = np.random.default_rng(5)
    keys = np.sort(np.concatenate([rng.normal(0, 1, 3000), rng.normal(8, 0.3, 1000)]))
    x = (keys - keys[0]) / (keys[-1] - keys[0])
    y = (np.arange(x.size) + 0.5) / x.size
    theta, _, _ = mlp.spline_start(x, y)
    best, losses = mlp.descent(theta, x, y, 16)
    assert all(b <= a for a, b in zip(losses, losses[1:]))
    assert losses[-1] < losses[0]
    moved = best - theta
    for part in (slice(0, 32), slice(32, 64), slice(64, 64 + 1024), slice(1088, 1120), slice(1120, 1152)):
        assert np.abs(moved[part]).max() > 0
    P = 64
    true_b = np.minimum((y * P).astype(int), P - 1)
    pred = mlp.predict_bucket(best, x, P)
    assert np.mean(np.abs(pred - true_b)) < np.mean(np.abs(P // 2 - true_b)) / 4


def test_descent_keeps_the_start_when_no_step_helps():
    """At a minimum (a network that already fits exactly) every step is
    rejected and the start comes back unchanged."""
    x = np.linspace(0, 1, 64)
    y = 0.25 + 0.5 * x
    theta = np.zeros(mlp.N_PARAMS)
    theta[0] = 1.0          # W1[0]
    theta[64] = 1.0         # W2[0][0]
    theta[1088 + 32] = 0.5  # w3[0]
    theta[-1] = 0.25        # b3
    best, losses = mlp.descent(theta, x, y, 8)
    assert losses[-1] <= 1e-30 and np.array_equal(best, theta)


def test_prediction_is_clamped():
    theta = np.zeros(mlp.N_PARAMS)
    theta[-1] = 5.0
    assert mlp.predict_bucket(theta, np.array([0.1]), 16).tolist() == [15]
    theta[-1] = -3.0
    assert mlp.predict_bucket(theta, np.array([0.1]), 16).tolist() == [0]
    theta[-1] = np.nan
    assert mlp.predict_bucket(theta, np.array([0.1]), 16).tolist() == [0]
