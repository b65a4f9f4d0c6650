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
the sorted sample, y_i = (i + 1/2) / S.  Parameters are packed in one vector
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


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015); t counts from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def predict_bucket(theta, x, P):
    """Predicted sub-bucket: floor(P * y) clamped to [0, P-1]."""
    y, _ = forward(theta, x)
    b = np.floor(np.nan_to_num(y, nan=0.0) * P)
    return np.clip(b, 0, P - 1).astype(np.int64)
