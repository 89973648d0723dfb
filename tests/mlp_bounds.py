"""A-priori rounding-error bounds of the library's encoder arithmetic, used as
the tolerances of its GPU parity tests (test infrastructure).

The GPU computes the encoder of oracle/mlp_oracle.py with the same BF16
weights: inputs x = log1pf(v * r) with r = fl32(n_f / S); the five products
(W1 x, W2 h, dW2 = dE^T h, dh = dE W2, dW1 = dh^T x) on the tensor cores with
BF16 operands (x, h = relu(Hpre), dE and dh each rounded to BF16 before the
product that reads them: relative error <= 2^-9) and FP32 accumulation; FP32
softmax and pair scores; atomically accumulated (any-order) FP32 sums for
the backward pass and FP32 column sums for the bias gradients.  The
standard bound for an n-term dot product accumulated in FP32,
|fl(a.b) - a.b| <= gamma_n |a|.|b| with gamma_n = n u / (1 - n u),
u = 2^-24, is applied to every product (whatever the order the tensor cores
add in), the BF16 rounding of each operand adds 2^-9 times its magnitude,
and errors of the inputs of each stage are carried forward to first order
with the stage's absolute sensitivity (relu and the clamp are 1-Lipschitz;
the softmax satisfies |dp_k| <= p_k (|dE_k| + max_m |dE_m|)).  The returned
bounds are twice the first-order sums, which covers the neglected
second-order terms (of relative size 2^-9) by a wide margin.  Where a
rounding-level change could flip a ReLU mask (|Hpre| within its own bound),
the bound of the affected hidden unit's gradient takes the whole unmasked
value.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp_oracle as mo

U = 2.0 ** -24
UB = 2.0 ** -9  # BF16 round-to-nearest, relative


def gamma(n: int) -> float:
    return n * U / (1.0 - n * U)


def encoder_bounds(theta: np.ndarray, V_fm: np.ndarray, pairs: np.ndarray, y: np.ndarray):
    """Bounds for E (nv x 64), the mean loss, and each gradient block
    (dW1, db1, dW2, db2), for the weights theta as used on the GPU (the
    caller passes theta with W1, W2 already BF16-rounded)."""
    d_in = V_fm.shape[0]
    W1, b1, W2, b2 = mo.unpack(theta, d_in)
    E, (X, Hpre, H, _, _) = mo.forward(theta, V_fm)
    aW1, aW2 = np.abs(W1), np.abs(W2)
    n = X.shape[0]
    # inputs: r rounded once, v*r once, log1pf within 2 ulp, then BF16
    BX = (2.0 ** -22 + UB) * np.abs(X) + 2.0 ** -23
    BHpre = gamma(d_in + 1) * (np.abs(X) @ aW1.T + np.abs(b1)) + BX @ aW1.T
    BH = BHpre + UB * np.abs(H)  # the BF16 operand h
    BE = gamma(mo.HIDDEN + 1) * (np.abs(H) @ aW2.T + np.abs(b2)) + BH @ aW2.T
    Pm = mo.softmax(E)
    # softmax: first-order sensitivity plus its own FP32 arithmetic (exp,
    # a 64-term sum, one division)
    BPm = Pm * (2.0 * BE.max(axis=1, keepdims=True) + 80 * U)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    y = np.asarray(y, dtype=np.float64)
    i, j = pairs[:, 0], pairs[:, 1]
    P = np.einsum("pd,pd->p", Pm[i], Pm[j])
    BP = np.einsum("pd,pd->p", BPm[i], Pm[j]) + np.einsum("pd,pd->p", Pm[i], BPm[j]) + gamma(64) * P
    Pc = np.clip(P, mo.CLAMP, 1 - mo.CLAMP)
    N = len(y)
    g = np.where((P > mo.CLAMP) & (P < 1 - mo.CLAMP), -y / Pc + (1 - y) / (1 - Pc), 0.0)
    ell = -(y * np.log(Pc) + (1 - y) * np.log1p(-Pc))
    Bloss = float(np.mean(np.abs(g) * BP + 4 * U * np.abs(ell)) + gamma(N) * np.mean(np.abs(ell)))
    # d loss / dP and its sensitivity |g'(P)| = y / P^2 + (1 - y) / (1 - P)^2
    gp = np.where((P > mo.CLAMP) & (P < 1 - mo.CLAMP), y / Pc ** 2 + (1 - y) / (1 - Pc) ** 2, 0.0)
    Bg = gp * BP + 4 * U * np.abs(g)
    deg = np.bincount(np.concatenate([i, j]), minlength=n).max()
    dP = np.zeros_like(Pm)
    adP = np.zeros_like(Pm)
    BdP = np.zeros_like(Pm)
    for a, b in ((i, j), (j, i)):
        np.add.at(dP, a, (g / N)[:, None] * Pm[b])
        np.add.at(adP, a, (np.abs(g) / N)[:, None] * Pm[b])
        np.add.at(BdP, a, (Bg / N)[:, None] * Pm[b] + (np.abs(g) / N)[:, None] * BPm[b])
    BdP += gamma(deg + 1) * adP
    s = np.sum(Pm * dP, axis=1, keepdims=True)
    Bs = np.sum(BPm * np.abs(dP) + Pm * BdP, axis=1, keepdims=True) + gamma(64) * np.sum(Pm * adP, axis=1,
                                                                                       keepdims=True)
    dE = Pm * (dP - s)
    BdE = BPm * (np.abs(dP) + np.abs(s)) + Pm * (BdP + Bs) + 4 * U * np.abs(dE)
    adE = np.abs(dE)
    BdEo = BdE + UB * adE                          # the BF16 operand dE
    BdW2 = gamma(n) * (adE.T @ np.abs(H)) + BdEo.T @ np.abs(H) + adE.T @ BH
    Bdb2 = gamma(n) * adE.sum(axis=0) + BdE.sum(axis=0)
    mask = Hpre > 0
    dHu = dE @ W2                                  # before the ReLU mask
    BdHu = gamma(64) * (adE @ aW2) + BdEo @ aW2
    dH = dHu * mask
    BdH = np.where(mask, BdHu, 0.0)
    unsure = np.abs(Hpre) <= BHpre                 # a rounding-level change may flip the mask
    BdH = np.where(unsure, np.abs(dHu) + BdHu, BdH)
    adH = np.abs(dH)
    BdHo = BdH + UB * adH                          # the BF16 operand dh
    BdW1 = gamma(n) * (adH.T @ np.abs(X)) + BdHo.T @ np.abs(X) + adH.T @ BX
    Bdb1 = gamma(n) * adH.sum(axis=0) + BdH.sum(axis=0)
    return {"E": 2 * BE, "loss": 2 * Bloss, "W1": 2 * BdW1.ravel(), "b1": 2 * Bdb1, "W2": 2 * BdW2.ravel(),
            "b2": 2 * Bdb2}
