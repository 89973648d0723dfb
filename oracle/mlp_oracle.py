"""FP64 CPU re-statement of the proposal encoder and its pair loss.

TEST INFRASTRUCTURE ONLY (imported by the tests).  The encoder is not part of
the paper; its definition is the library's:
    x_i = log1p(v_i),  h_i = relu(W1 x_i + b1),  e_i = W2 h_i + b2,
    z_ij = e_i . e_j + beta,
    loss = mean over pairs of  log(1 + exp(z)) - y z.
Parameters are a flat vector [W1 (256 x d_in), b1, W2 (64 x 256), b2, beta].
Gradients are written out by hand (chain rule) and pinned by central finite
differences in the CPU tests.
"""
from __future__ import annotations

import numpy as np

HIDDEN, OUT = 256, 64


def unpack(theta: np.ndarray, d_in: int):
    theta = np.asarray(theta, dtype=np.float64)
    n1 = HIDDEN * d_in
    W1 = theta[:n1].reshape(HIDDEN, d_in)
    b1 = theta[n1:n1 + HIDDEN]
    o = n1 + HIDDEN
    W2 = theta[o:o + OUT * HIDDEN].reshape(OUT, HIDDEN)
    b2 = theta[o + OUT * HIDDEN:o + OUT * HIDDEN + OUT]
    beta = theta[-1]
    return W1, b1, W2, b2, beta


def forward(theta, V_fm: np.ndarray):
    """V_fm: (nf, nv) field-major values; returns (E, cache)."""
    d_in = V_fm.shape[0]
    W1, b1, W2, b2, beta = unpack(theta, d_in)
    X = np.log1p(np.asarray(V_fm, dtype=np.float64).T)      # (nv, d_in)
    Hpre = X @ W1.T + b1
    H = np.maximum(Hpre, 0.0)
    E = H @ W2.T + b2
    return E, (X, Hpre, H, W1, W2, beta)


def pair_loss_and_grad(theta, V_fm, pairs, y):
    E, (X, Hpre, H, W1, W2, beta) = forward(theta, V_fm)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    y = np.asarray(y, dtype=np.float64)
    i, j = pairs[:, 0], pairs[:, 1]
    z = np.einsum("pd,pd->p", E[i], E[j]) + beta
    loss = np.mean(np.logaddexp(0.0, z) - y * z)
    g = (1.0 / (1.0 + np.exp(-z)) - y) / len(y)               # dloss/dz
    dE = np.zeros_like(E)
    np.add.at(dE, i, g[:, None] * E[j])
    np.add.at(dE, j, g[:, None] * E[i])
    dW2 = dE.T @ H
    db2 = dE.sum(axis=0)
    dH = (dE @ W2) * (Hpre > 0)
    dW1 = dH.T @ X
    db1 = dH.sum(axis=0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, [g.sum()]])
    return loss, grad, E


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even)."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)
