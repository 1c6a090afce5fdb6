"""CPU oracle of the learned skip proposal's network (test infrastructure).

A two-layer perceptron on 8 per-vertex features: h = relu(W1 x + b1) with 32
hidden units, z = w2 . h + b2, p = sigmoid(z) = the predicted probability
that the vertex moves in the coming sweep.  Trained with the mean binary
cross-entropy L = mean(-y log p - (1 - y) log(1 - p)).  Everything here is
float64 numpy on the same float16-rounded inputs and weights the GPU kernels
take; parity with the GPU is within float32 accumulation error.

The skip proposal itself is an addition to the paper's method (the paper has
no learned component); the features are statistics the local-moving phase
already keeps (Section 3 notation).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 8, 32


def features(deg, K, size_d, sigma_d, two_m, moved_last, since_move, attach):
    """The 8 input features of every vertex (float64, before float16 rounding):
    0 log2(1 + deg) / 16; 1 moved in the previous sweep; 2 min(sweeps since
    its last move, 8) / 8; 3 log2(1 + |community|) / 24; 4 sqrt(Sigma_d / 2m);
    5 K_i / Sigma_d; 6 K_{i->C_i} / K_i at the vertex's last decision; 7 1."""
    deg = np.asarray(deg, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    sd = np.asarray(sigma_d, dtype=np.float64)
    x = np.empty((len(deg), N_IN), dtype=np.float64)
    x[:, 0] = np.log2(1.0 + deg) / 16.0
    x[:, 1] = np.asarray(moved_last, dtype=np.float64)
    x[:, 2] = np.minimum(np.asarray(since_move, dtype=np.float64), 8.0) / 8.0
    x[:, 3] = np.log2(1.0 + np.asarray(size_d, dtype=np.float64)) / 24.0
    x[:, 4] = np.sqrt(sd / float(two_m)) if two_m > 0 else 0.0
    x[:, 5] = np.where(sd > 0, K / np.where(sd > 0, sd, 1.0), 0.0)
    x[:, 6] = np.asarray(attach, dtype=np.float64)
    x[:, 7] = 1.0
    return x


def forward(x, W1, b1, w2, b2):
    """Returns (p, z, h)."""
    x = np.asarray(x, dtype=np.float64)
    h = np.maximum(x @ np.asarray(W1, dtype=np.float64).T + np.asarray(b1, dtype=np.float64), 0.0)
    z = h @ np.asarray(w2, dtype=np.float64) + float(b2)
    p = 1.0 / (1.0 + np.exp(-z))
    return p, z, h


def loss(x, y, W1, b1, w2, b2):
    p, z, _ = forward(x, W1, b1, w2, b2)
    y = np.asarray(y, dtype=np.float64)
    # stable form of the binary cross-entropy from the logit
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def gradients(x, y, W1, b1, w2, b2):
    """Gradients of the mean binary cross-entropy (dW1, db1, dw2, db2)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p, z, h = forward(x, W1, b1, w2, b2)
    n = len(x)
    dz = (p - y) / n
    dw2 = h.T @ dz
    db2 = float(dz.sum())
    dh = np.outer(dz, np.asarray(w2, dtype=np.float64)) * (h > 0)
    dW1 = dh.T @ x
    db1 = dh.sum(axis=0)
    return dW1, db1, dw2, db2


def to_half(a):
    """Round to float16 and back (what the GPU kernels read)."""
    return np.asarray(a, dtype=np.float16).astype(np.float64)


def adam_step(params, grads, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, "Adam: A Method for Stochastic
    Optimization", ICLR 2015, Algorithm 1), elementwise over flat float64
    arrays: the biased first and second moment estimates
    m1 <- beta1 m1 + (1 - beta1) g and m2 <- beta2 m2 + (1 - beta2) g^2, their
    bias-corrected forms m1 / (1 - beta1^t) and m2 / (1 - beta2^t) for step
    t >= 1, and the parameter step -lr * m1_hat / (sqrt(m2_hat) + eps).
    Returns new (params, m1, m2); the inputs are not modified."""
    g = np.asarray(grads, dtype=np.float64)
    m1 = beta1 * np.asarray(m1, dtype=np.float64) + (1.0 - beta1) * g
    m2 = beta2 * np.asarray(m2, dtype=np.float64) + (1.0 - beta2) * g * g
    m1_hat = m1 / (1.0 - beta1 ** step)
    m2_hat = m2 / (1.0 - beta2 ** step)
    params = np.asarray(params, dtype=np.float64) - lr * m1_hat / (np.sqrt(m2_hat) + eps)
    return params, m1, m2


def flatten(W1, b1, w2, b2):
    """The parameters in the library's layout: W1 row by row, b1, w2, b2."""
    return np.concatenate([np.asarray(W1, dtype=np.float64).reshape(-1), np.asarray(b1, dtype=np.float64),
                           np.asarray(w2, dtype=np.float64), [float(b2)]])
