"""Pins of the FP64 encoder re-statement (oracle/mlp_oracle.py).

* A hand-worked network (two inputs, two live hidden units, three live
  outputs) on three vectors: embeddings, softmax partition sums, pair scores,
  the loss and the output-bias gradient are written out in closed form and
  compared with the oracle; a copy of the oracle with a plausible mistake
  planted in it (log for log1p, a dropped n_f / S scale or bias, a wrong
  sign, softmax axis or Jacobian term) fails those checks.
* Its hand-written gradient against central finite differences of its loss.
* The BF16 rounding helper against exact cases."""
import numpy as np
import pytest

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


def _hand_network(d_in=2):
    """A network whose outputs are worked out by hand below: hidden unit 0 =
    relu(x0 - x1), hidden unit 1 = relu(x0 + x1 - 1), e0 = 2 h0, e1 = h1,
    e2 = ln 2 (bias); every other weight and bias is 0."""
    W1 = np.zeros((mo.HIDDEN, d_in))
    W1[0] = [1.0, -1.0]
    W1[1] = [1.0, 1.0]
    b1 = np.zeros(mo.HIDDEN)
    b1[1] = -1.0
    W2 = np.zeros((mo.OUT, mo.HIDDEN))
    W2[0, 0] = 2.0
    W2[1, 1] = 1.0
    b2 = np.zeros(mo.OUT)
    b2[2] = np.log(2.0)
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2])


def test_forward_and_loss_hand_worked():
    _hand_worked_checks(mo)


def _hand_worked_checks(mo):
    # vectors u = (1, 3), v = (2, 0), w = (0, 0) (field-major columns).
    # Encoder input x_q = log1p(v_q * n_f / S): u has S = 4, n_f / S = 1/2,
    # x = (ln 1.5, ln 2.5); v has S = 2, x = (ln 3, 0); w is all zero, x = 0.
    #   u: h0 = relu(ln 0.6) = 0,        h1 = ln 3.75 - 1  -> e = (0, ln 3.75 - 1, ln 2, 0, ...)
    #   v: h0 = ln 3,  h1 = ln 3 - 1                       -> e = (2 ln 3, ln 3 - 1, ln 2, 0, ...)
    #   w: h0 = 0,     h1 = relu(-1) = 0                   -> e = (0, 0, ln 2, 0, ...)
    # softmax numerators exp(e_k): u (1, 3.75/e, 2, 1 x 61), v (9, 3/e, 2, 1 x 61),
    # w (1, 1, 2, 1 x 61); partition sums Zu = 64 + 3.75/e, Zv = 72 + 3/e, Zw = 65.
    E_ = np.e
    V = np.array([[1.0, 2.0, 0.0], [3.0, 0.0, 0.0]])
    theta = _hand_network()
    E, _ = mo.forward(theta, V)
    want = np.zeros((3, mo.OUT))
    want[0, 1], want[0, 2] = np.log(3.75) - 1.0, np.log(2.0)
    want[1, 0], want[1, 1], want[1, 2] = 2.0 * np.log(3.0), np.log(3.0) - 1.0, np.log(2.0)
    want[2, 2] = np.log(2.0)
    np.testing.assert_allclose(E, want, rtol=0, atol=1e-15)
    # scale-free input: a vector and its multiples encode the same way
    E2, _ = mo.forward(theta, V * np.array([[7.5, 0.01, 3.0]]))
    np.testing.assert_allclose(E2, E, rtol=0, atol=1e-14)
    Zu, Zv, Zw = 64.0 + 3.75 / E_, 72.0 + 3.0 / E_, 65.0
    P_uv = (9.0 + 11.25 / E_ ** 2 + 4.0 + 61.0) / (Zu * Zv)
    P_uw = (1.0 + 3.75 / E_ + 4.0 + 61.0) / (Zu * Zw)
    P_vw = (9.0 + 3.0 / E_ + 4.0 + 61.0) / (Zv * Zw)
    pairs = np.array([[0, 1], [0, 2], [1, 2]])
    y = np.array([1.0, 0.0, 1.0])
    loss, grad, _ = mo.pair_loss_and_grad(theta, V, pairs, y)
    want_loss = (-np.log(P_uv) - np.log(1.0 - P_uw) - np.log(P_vw)) / 3.0
    assert abs(loss - want_loss) <= 1e-14 * want_loss, (loss, want_loss)
    # the output-bias gradient in closed form: for a pair (i, j) with score P
    # and dloss/dP = g, the softmax Jacobian gives
    #   dloss/db2_k = g (2 p_ik p_jk - P (p_ik + p_jk)),  averaged over pairs
    num = {0: np.r_[1.0, 3.75 / E_, 2.0, np.ones(61)], 1: np.r_[9.0, 3.0 / E_, 2.0, np.ones(61)],
           2: np.r_[1.0, 1.0, 2.0, np.ones(61)]}
    Z = {0: Zu, 1: Zv, 2: Zw}
    p = {k: num[k] / Z[k] for k in num}
    Pp = {(0, 1): P_uv, (0, 2): P_uw, (1, 2): P_vw}
    db2 = np.zeros(mo.OUT)
    for (i, j), t in zip(pairs.tolist(), y):
        P = Pp[(i, j)]
        g = -t / P + (1.0 - t) / (1.0 - P)
        db2 += g * (2.0 * p[i] * p[j] - P * (p[i] + p[j]))
    db2 /= 3.0
    np.testing.assert_allclose(grad[-mo.OUT:], db2, rtol=0, atol=1e-15)
    # the hidden bias b1_0 receives gradient only from v (u and w have h0 = 0)
    # and b1_1 only from u and v (w has h1 = 0): dW1 rows carry x, so the
    # zero input of w contributes nothing anywhere in W1
    n1 = mo.HIDDEN * 2
    gW1 = grad[:n1].reshape(mo.HIDDEN, 2)
    gb1 = grad[n1:n1 + mo.HIDDEN]
    assert np.all(gW1[2:] == 0.0) and np.all(gb1[2:] == 0.0)
    # dW1[0] = dh0(v) * x(v) with x(v) = (ln 3, 0)
    assert gW1[0, 1] == 0.0 and abs(gW1[0, 0] - gb1[0] * np.log(3.0)) <= 1e-15


def test_loss_clamps_to_the_stated_range():
    # P is clamped to [1e-6, 1 - 1e-6] before the logarithms and the gradient
    # is zero where the clamp is active: a pair of identical one-hot-like
    # embeddings (P ~ 1) labelled 0 has loss -log(1e-6) and no gradient
    theta = np.zeros(mo.n_params(2))
    o = mo.HIDDEN * 2 + mo.HIDDEN + mo.OUT * mo.HIDDEN
    theta[o + 5] = 60.0  # b2_5: softmax puts all mass on output 5 for every vector
    V = np.array([[1.0, 2.0], [1.0, 0.5]])
    loss, grad, _ = mo.pair_loss_and_grad(theta, V, np.array([[0, 1]]), np.array([0.0]))
    assert abs(loss - (-np.log(1e-6))) <= 1e-9
    assert np.all(grad == 0.0)


@pytest.mark.parametrize("old,new", [
    ("np.log1p(Vv * r)", "np.log(Vv * r + 1e-30)"),          # log instead of log1p
    ("d_in / np.where(S > 0, S, 1.0)", "1.0 / np.where(S > 0, S, 1.0)"),  # n_f / S scale dropped
    ("Hpre = X @ W1.T + b1", "Hpre = X @ W1.T"),              # b1 dropped
    ("E = H @ W2.T + b2", "E = H @ W2.T - b2"),               # sign of b2
    ("H = np.maximum(Hpre, 0.0)", "H = np.abs(Hpre)"),         # wrong activation
    ("X / X.sum(axis=1, keepdims=True)", "X / X.sum(axis=0, keepdims=True)"),  # softmax axis
    ("(1 - y) * np.log1p(-Pc)", "(1 - y) * np.log1p(Pc)"),     # loss sign
    ("dE = Pm * (dP - np.sum(Pm * dP, axis=1, keepdims=True))", "dE = Pm * dP"),  # Jacobian term
])
def test_hand_worked_pins_catch_planted_mistakes(old, new):
    # each plausible mistake, planted in a copy of the oracle's source, makes
    # the hand-worked checks fail
    import inspect
    import types
    src = inspect.getsource(mo)
    assert old in src, old
    bad = types.ModuleType("mlp_oracle_mutant")
    exec(compile(src.replace(old, new), "mlp_oracle_mutant", "exec"), bad.__dict__)
    with pytest.raises(AssertionError):
        _hand_worked_checks(bad)
