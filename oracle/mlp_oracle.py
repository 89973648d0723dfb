"""FP64 CPU re-statement of the proposal encoder and its pair loss.

TEST INFRASTRUCTURE ONLY (imported by the tests).  The encoder is not part of
the paper; its definition is the library's:
    x_iq = log1p(v_iq * n_f / S_i)  (0 for an all-zero vector),
    h_i = relu(W1 x_i + b1),  e_i = W2 h_i + b2,
    p_i = softmax(e_i),  P_ij = p_i . p_j  (clamped to [1e-6, 1 - 1e-6]),
    loss = mean over pairs of  -(y log P + (1 - y) log(1 - P)).
Parameters are a flat vector [W1 (256 x d_in), b1, W2 (64 x 256), b2].
Gradients are written out by hand (chain rule) and pinned by central finite
differences in the CPU tests.
"""
from __future__ import annotations

import numpy as np

HIDDEN, OUT = 256, 64
CLAMP = 1e-6


def n_params(d_in: int) -> int:
    return HIDDEN * d_in + HIDDEN + OUT * HIDDEN + OUT


def unpack(theta: np.ndarray, d_in: int):
    theta = np.asarray(theta, dtype=np.float64)
    n1 = HIDDEN * d_in
    W1 = theta[:n1].reshape(HIDDEN, d_in)
    b1 = theta[n1:n1 + HIDDEN]
    o = n1 + HIDDEN
    W2 = theta[o:o + OUT * HIDDEN].reshape(OUT, HIDDEN)
    b2 = theta[o + OUT * HIDDEN:o + OUT * HIDDEN + OUT]
    return W1, b1, W2, b2


def softmax(E):
    Z = E - E.max(axis=1, keepdims=True)
    X = np.exp(Z)
    return X / X.sum(axis=1, keepdims=True)


def forward(theta, V_fm: np.ndarray):
    """V_fm: (nf, nv) field-major values; returns (E, cache)."""
    d_in = V_fm.shape[0]
    W1, b1, W2, b2 = unpack(theta, d_in)
    Vv = np.asarray(V_fm, dtype=np.float64).T                # (nv, d_in)
    S = Vv.sum(axis=1, keepdims=True)
    r = np.where(S > 0, d_in / np.where(S > 0, S, 1.0), 0.0)
    X = np.log1p(Vv * r)
    Hpre = X @ W1.T + b1
    H = np.maximum(Hpre, 0.0)
    E = H @ W2.T + b2
    return E, (X, Hpre, H, W1, W2)


def pair_loss_and_grad(theta, V_fm, pairs, y):
    E, (X, Hpre, H, W1, W2) = forward(theta, V_fm)
    Pm = softmax(E)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    y = np.asarray(y, dtype=np.float64)
    i, j = pairs[:, 0], pairs[:, 1]
    P = np.einsum("pd,pd->p", Pm[i], Pm[j])
    Pc = np.clip(P, CLAMP, 1 - CLAMP)
    loss = np.mean(-(y * np.log(Pc) + (1 - y) * np.log1p(-Pc)))
    inside = (P > CLAMP) & (P < 1 - CLAMP)
    g = np.where(inside, -y / Pc + (1 - y) / (1 - Pc), 0.0) / len(y)   # dloss/dP
    dP = np.zeros_like(Pm)
    np.add.at(dP, i, g[:, None] * Pm[j])
    np.add.at(dP, j, g[:, None] * Pm[i])
    dE = Pm * (dP - np.sum(Pm * dP, axis=1, keepdims=True))          # softmax Jacobian
    dW2 = dE.T @ H
    db2 = dE.sum(axis=0)
    dH = (dE @ W2) * (Hpre > 0)
    dW1 = dH.T @ X
    db1 = dH.sum(axis=0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2])
    return loss, grad, E


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even)."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)
