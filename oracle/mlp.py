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
piecewise-linear interpolant of the training points (spline_start) and takes
full-batch gradient steps on the output layer (head_step).  Parameters are packed in one vector
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
HEAD = slice(2 * H + H * H + H, N_PARAMS)   # w3 and b3: the trained parameters


def spline_start(x, y):
    """Parameters of the piecewise-linear interpolant of the points (x, y)
    (x ascending) at KNOTS knots of evenly spaced index j*(M-1)//H, equal x
    merged (the later y kept): unit j of layer 1 is relu(x - knot_j), layer 2
    is the identity, the output weights are the slope changes."""
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
    return np.concatenate([W1, b1, W2.ravel(), b2, w3, [b3]]), np.array(kx), np.array(ky)


def head_step(theta, grad, lr):
    """One gradient-descent step on the output layer (w3, b3) only."""
    theta = np.array(theta, dtype=np.float64)
    theta[HEAD] -= lr * np.asarray(grad, dtype=np.float64)[HEAD]
    return theta


def predict_bucket(theta, x, P):
    """Predicted sub-bucket: floor(P * y) clamped to [0, P-1]."""
    y, _ = forward(theta, x)
    b = np.floor(np.nan_to_num(y, nan=0.0) * P)
    return np.clip(b, 0, P - 1).astype(np.int64)
