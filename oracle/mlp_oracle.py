"""FP64 reference of the learned-threshold network (test infrastructure: only the
tests use it; the engine never imports it).

Network: standardised features (F = 257) -> H = 128 ReLU units -> 1 output, mean
squared error loss; written with numpy matrix products in FP64, in the parameter
layout of the engine: W1[H][F] | b1[H] | W2[H] | b2 | mu[F] | sigma[F] | margin.
Features of a query row: log |q|^2 and the sorted log squared distances (FP64 direct
difference) to the 256 corpus samples, with the same floor for zero distances.
"""
from __future__ import annotations

import numpy as np

F, H = 257, 128
N_TRAIN = H * F + 2 * H + 1
N_PARAMS = N_TRAIN + 2 * F + 1
LOG_FLOOR = -69.0


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H]; o += H
    b2 = p[o]; o += 1
    mu = p[o:o + F]; o += F
    sigma = p[o:o + F]; o += F
    margin = p[o]
    return W1, b1, W2, b2, mu, sigma, margin


def forward(params, X):
    """Predictions y (FP64) for raw features X (n x F)."""
    W1, b1, W2, b2, mu, sigma, _ = unpack(params)
    Xn = (np.asarray(X, dtype=np.float64) - mu) / sigma
    A = Xn @ W1.T + b1
    return np.maximum(A, 0.0) @ W2 + b2


def loss_grad(params, X, T):
    """Mean squared error and its gradient w.r.t. the trained parameters (FP64)."""
    W1, b1, W2, b2, mu, sigma, _ = unpack(params)
    Xn = (np.asarray(X, dtype=np.float64) - mu) / sigma
    T = np.asarray(T, dtype=np.float64)
    n = Xn.shape[0]
    A = Xn @ W1.T + b1
    Hh = np.maximum(A, 0.0)
    y = Hh @ W2 + b2
    e = y - T
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    dW2 = Hh.T @ dy
    db2 = dy.sum()
    dA = np.outer(dy, W2) * (A > 0)
    dW1 = dA.T @ Xn
    db1 = dA.sum(axis=0)
    return loss, np.concatenate([dW1.ravel(), db1, dW2, [db2]])


def features(Q, S):
    """Features of the rows of Q against the samples S (FP64 direct differences)."""
    Q = np.asarray(Q, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    d2 = ((Q[:, None, :] - S[None, :, :]) ** 2).sum(axis=2)
    out = np.empty((Q.shape[0], F))
    with np.errstate(divide="ignore"):
        out[:, 0] = np.maximum(np.log((Q * Q).sum(axis=1)), LOG_FLOOR)
        out[:, 1:] = np.maximum(np.log(np.sort(d2, axis=1)), LOG_FLOOR)
    return out
