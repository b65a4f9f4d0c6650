"""CPU oracle of the learned bucket classifier (float64, numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the product path never
imports it.

The classifier is not in the paper.  It predicts the bucket of a key from an
estimate of the cumulative distribution of the keys, learned from the sample
the method draws anyway (Fig. 1 step 4 / Fig. 3 step 4), and a bounded search
against the true splitters corrects every prediction, so buckets are exactly
#{i : S_i <= key} (Fig. 2 step 9) whatever the network predicts.

Network: x -> h1 = relu(W1 x + b1) (32) -> h2 = relu(W2 h1 + b2) (32)
-> y = w3 . h2 + b3.  Loss: mean squared error against the empirical CDF of
the sorted sample, y_i = (i + 1/2) / S.  Training starts from the
piecewise-linear interpolant of the training points (spline_start), its
units rescaled so that each carries its weight equally over its three
weights (the same function, better conditioned), and takes full-batch
gradient-descent steps on all parameters with backtracking (descent).
Parameters are packed in one vector
in the order W1 (32), b1 (32), W2 (32x32, row-major, W2[i, j] multiplies
h1[j] into unit i), b2 (32), w3 (32), b3 (1): 1153 values.
"""
from __future__ import annotations

import numpy as np

H = 32
N_PARAMS = H + H + H * H + H + H + 1


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + H]; o += H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def forward(theta, x):
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    z1 = np.outer(x, W1) + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(theta, x, target):
    """Mean squared error and its gradient (backpropagation written out)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    y, (x, z1, h1, z2, h2) = forward(theta, x)
    m = x.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / m                       # d loss / d y
    g_b3 = dy.sum()
    g_w3 = h2.T @ dy
    dz2 = np.outer(dy, w3) * (z2 > 0)      # through relu
    g_b2 = dz2.sum(axis=0)
    g_W2 = dz2.T @ h1
    dz1 = (dz2 @ W2) * (z1 > 0)
    g_b1 = dz1.sum(axis=0)
    g_W1 = dz1.T @ x
    grad = np.concatenate([g_W1, g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, grad


KNOTS = H + 1      # knots of the spline start


def spline_start(x, y):
    """Parameters of the piecewise-linear interpolant of the points (x, y)
    (x ascending) at KNOTS knots of evenly spaced index j*(M-1)//H, equal x
    merged (the later y kept): unit j of layer 1 is relu(x - knot_j), unit j of
    layer 2 passes it on, the output weights are the slope changes.  Each
    unit j is then rescaled: with a = |w3_j|^(1/3), its layer-1 weights and
    its layer-2 weight are multiplied by a and its output weight divided by
    a^2 -- relu(a z) = a relu(z) for a > 0, so the function is unchanged and
    the three weights carry |w3_j| equally."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    M = x.shape[0]
    kx, ky = [], []
    for j in range(KNOTS if M else 0):
        i = j * (M - 1) // H if M > 1 else 0
        if not kx or x[i] > kx[-1]:
            kx.append(x[i])
            ky.append(y[i])
        else:
            ky[-1] = y[i]
    segs = max(len(kx) - 1, 0)
    slope = [(ky[j + 1] - ky[j]) / (kx[j + 1] - kx[j]) for j in range(segs)]
    W1 = np.array([1.0 if j < segs else 0.0 for j in range(H)])
    b1 = np.array([-kx[j] if j < segs else -1.0 for j in range(H)])
    W2 = np.eye(H)
    b2 = np.zeros(H)
    w3 = np.array([(slope[0] if j == 0 else slope[j] - slope[j - 1]) if j < segs else 0.0 for j in range(H)])
    b3 = ky[0] if kx else 0.0
    for j in range(segs):
        if w3[j] != 0.0:
            a = abs(w3[j]) ** (1.0 / 3.0)
            W1[j] *= a
            b1[j] *= a
            W2[j, j] *= a
            w3[j] /= a * a
    return np.concatenate([W1, b1, W2.ravel(), b2, w3, [b3]]), np.array(kx), np.array(ky)


def descent(theta, x, y, steps, first=0.1, grow=1.5, shrink=0.25):
    """Full-batch gradient descent on all parameters with backtracking: from
    the best parameters so far, a step of size eta along the negative
    gradient (first eta = first * loss / |grad|^2, so that the linear model
    predicts a drop of that fraction of the loss); a step that lowers the
    loss is kept and eta grows, else it is dropped and eta shrinks.  Returns
    the best parameters and the loss after each step (never increasing)."""
    best = np.array(theta, dtype=np.float64)
    lb, gb = loss_and_grad(best, x, y)
    eta = first * lb / max(float(np.dot(gb, gb)), 1e-300)
    losses = [lb]
    for _ in range(steps):
        cand = best - eta * gb
        l, g = loss_and_grad(cand, x, y)
        if l < lb:
            best, lb, gb = cand, l, g
            eta *= grow
        else:
            eta *= shrink
        losses.append(lb)
    return best, losses


def predict_bucket(theta, x, P):
    """Predicted sub-bucket: floor(P * y) clamped to [0, P-1]."""
    y, _ = forward(theta, x)
    b = np.floor(np.nan_to_num(y, nan=0.0) * P)
    return np.clip(b, 0, P - 1).astype(np.int64)
