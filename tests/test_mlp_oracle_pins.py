"""Pins of the FP64 encoder re-statement (oracle/mlp_oracle.py): its
hand-written gradient against central finite differences of its own loss,
and the BF16 rounding helper against exact cases."""
import numpy as np

from oracle import mlp_oracle as mo


def test_pair_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    d_in, nv = 6, 9
    V = rng.exponential(1.0, size=(d_in, nv))
    V[rng.random((d_in, nv)) < 0.5] = 0.0
    n = mo.n_params(d_in)
    theta = rng.normal(0, 0.2, size=n)
    pairs = np.array([[0, 1], [2, 5], [3, 4], [1, 8], [0, 7], [6, 8]])
    y = np.array([1, 0, 1, 0, 1, 0], dtype=np.float64)
    loss, grad, _ = mo.pair_loss_and_grad(theta, V, pairs, y)
    idx = np.concatenate([rng.choice(mo.HIDDEN * d_in, 25, replace=False),
                          mo.HIDDEN * d_in + rng.choice(mo.HIDDEN, 10, replace=False),
                          mo.HIDDEN * d_in + mo.HIDDEN + rng.choice(mo.OUT * mo.HIDDEN, 25, replace=False),
                          [n - 2, n - 1]])
    eps = 1e-6
    for k in idx:
        tp = theta.copy(); tp[k] += eps
        tm = theta.copy(); tm[k] -= eps
        num = (mo.pair_loss_and_grad(tp, V, pairs, y)[0] - mo.pair_loss_and_grad(tm, V, pairs, y)[0]) / (2 * eps)
        assert abs(num - grad[k]) <= 1e-6 * max(1.0, abs(num)), (k, num, grad[k])


def test_softmax_pair_score_is_a_probability():
    rng = np.random.default_rng(1)
    E = rng.normal(0, 3, size=(10, mo.OUT))
    P = mo.softmax(E)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, rtol=1e-14)
    S = P @ P.T
    assert np.all(S >= 0) and np.all(S <= 1 + 1e-12)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -9, -2.5, 0.0], dtype=np.float32)
    r = mo.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                # tie -> even
    assert r[2] == 1.0 + 2 ** -7      # representable
    assert r[3] == 1.0 + 2 ** -7      # rounds up
    assert r[4] == -2.5 and r[5] == 0.0
