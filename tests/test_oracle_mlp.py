"""Pins of the pivot-proposal perceptron oracle (oracle/mlp.py) against
finite differences, closed forms and invariants -- never against itself."""
import numpy as np
import pytest

from oracle import mlp as M


def small_params(seed=0):
    P = M.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    P["b1"] = (0.1 * rng.standard_normal(M.HIDDEN)).astype(np.float32)
    P["b2"] = (0.1 * rng.standard_normal(M.HIDDEN)).astype(np.float32)
    P["b3"] = np.array([0.05], np.float32)
    return P


def test_loss_closed_forms():
    # softplus(0) = log 2 whatever the label; large margins give ~0 loss
    assert M.loss(np.zeros(5), np.array([0, 1, 0, 1, 1.0])) == pytest.approx(np.log(2.0), rel=1e-15)
    assert M.loss(np.array([40.0, -40.0]), np.array([1.0, 0.0])) < 1e-15
    assert M.loss(np.array([-3.0]), np.array([1.0])) == pytest.approx(np.log1p(np.exp(3.0)), rel=1e-14)


def test_backward_matches_central_differences():
    # the unrounded network is smooth: its analytic gradient must match
    # central differences of the loss
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, M.F_IN))
    y = (rng.random(40) < 0.3).astype(np.float64)
    Pd = {k: np.asarray(v, np.float64) for k, v in small_params(2).items()}
    s, cache = M.forward(Pd, X, bf16_ops=False)
    g = M.backward(s, y, cache)
    h = 1e-6
    for k in Pd:
        flat = Pd[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(M.forward(Pd, X, bf16_ops=False)[0], y)
            flat[idx] = old - h
            lm = M.loss(M.forward(Pd, X, bf16_ops=False)[0], y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)), (k, idx, fd, an)


def test_bf16_products_round_both_operands():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((8, M.F_IN))
    P = small_params(5)
    s_r, c_r = M.forward(P, X, bf16_ops=True)
    # by hand: layer by layer with explicitly rounded operands
    Z1 = M.bf16(X) @ M.bf16(P["W1"]) + P["b1"]
    Z2 = M.bf16(np.maximum(Z1, 0)) @ M.bf16(P["W2"]) + P["b2"]
    s = M.bf16(np.maximum(Z2, 0)) @ M.bf16(P["w3"]) + P["b3"][0]
    assert np.allclose(s_r, s, rtol=1e-13, atol=1e-13)
    # six operand roundings of relative size <= 2^-8 on the way to a score,
    # through 1-Lipschitz ReLUs: |s_bf16 - s| <= ~6 2^-8 times the same
    # network run on absolute values (first order; asserted with slack 8)
    s_e, _ = M.forward(P, X, bf16_ops=False)
    H1a = np.abs(X) @ np.abs(P["W1"]) + np.abs(P["b1"])
    H2a = H1a @ np.abs(P["W2"]) + np.abs(P["b2"])
    sa = H2a @ np.abs(P["w3"]) + abs(P["b3"][0])
    assert np.all(np.abs(s_r - s_e) <= 8 * 2.0 ** -8 * sa)


def test_forward_closed_form():
    # one active path: x0 = 2 -> 1.5 x0 = 3 -> 0.5 * 3 = 1.5 -> 2 * 1.5 + 0.25
    # (every value exact in BF16); a negative input is cut by the first ReLU
    P = {k: np.zeros_like(v) for k, v in M.init_params(0).items()}
    P["W1"][0, 0], P["W2"][0, 0], P["w3"][0], P["b3"][0] = 1.5, 0.5, 2.0, 0.25
    X = np.zeros((2, M.F_IN))
    X[0, 0], X[1, 0] = 2.0, -2.0
    for ops in (True, False):
        s, _ = M.forward(P, X, bf16_ops=ops)
        assert list(s) == [3.25, 0.25]


def test_bf16_rounding_closed_forms():
    # 8 significant bits: ties to even at 1 + 2^-8, up at 1 + 3 * 2^-9
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -8], np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, -2.5, 1.0 + 2.0 ** -6])
    assert np.array_equal(M.bf16(x), want)


def test_adam_first_step_is_signed_lr():
    P = {"a": np.array([1.0, -2.0, 3.0], np.float32)}
    g = {"a": np.array([0.5, -4.0, 1e-3])}
    out = M.adam(P, g, {}, lr=1e-2, t=1)
    # t = 1: m_hat = g, v_hat = g^2, step = lr g / (|g| + eps)
    want = P["a"] - 1e-2 * g["a"] / (np.abs(g["a"]) + 1e-8)
    assert np.allclose(out["a"], want.astype(np.float32), rtol=0, atol=1e-7)


def test_features_invariants():
    rng = np.random.default_rng(6)
    n1, n2, r = 30, 50, 4
    A = rng.standard_normal((n1, r))
    B = rng.standard_normal((n2, r))
    X = M.features(A, B)
    assert X.shape == (n2, M.F_IN)
    # leverages of an orthonormal basis sum to r, so their normalised mean is 1
    assert X[:, 0].mean() == pytest.approx(1.0, rel=1e-13)
    # basis independence: B R with A R^{-T} is the same matrix, same features
    R = rng.standard_normal((r, r)) + 3 * np.eye(r)
    X2 = M.features(A @ np.linalg.inv(R).T, B @ R)
    assert np.allclose(X, X2, rtol=1e-9, atol=1e-10)
    # neighbour columns are the leverage at j -+ 1, 2 (periodic)
    assert np.array_equal(X[:, 2], np.roll(X[:, 0], 1))
    assert X[0, 3] == X[1, 0] and X[0, 4] == X[2, 0] and X[0, 1] == X[n2 - 2, 0]
    # a rank-1 matrix constant along j: uniform leverage, flat profile
    X1 = M.features(rng.standard_normal((n1, 1)), np.ones((n2, 1)))
    assert np.allclose(X1[:, 0], 1.0) and np.allclose(X1[:, 5:9], 0.0) and np.allclose(X1[:, 9], 1.0)
    # no previous pivots: indicator 0, distance feature saturated at 1
    assert np.all(X[:, 12] == 0.0) and np.all(X[:, 13] == 1.0)


def test_previous_pivot_features_closed_form():
    rng = np.random.default_rng(7)
    A, B = rng.standard_normal((10, 3)), rng.standard_normal((16, 3))
    X = M.features(A, B, prev=[3, 10])
    assert list(np.nonzero(X[:, 12])[0]) == [3, 10]
    # distances to {3, 10} on a 16-cycle, capped at 8, divided by 8
    want = [3, 2, 1, 0, 1, 2, 3, 3, 2, 1, 0, 1, 2, 3, 4, 4]
    assert np.array_equal(X[:, 13], np.array(want) / 8.0)
    # the other features do not depend on prev
    assert np.array_equal(X[:, :12], M.features(A, B)[:, :12])


def test_top_indices_ties_to_smaller_index():
    s = np.array([0.5, 2.0, 2.0, -1.0, 2.0, 0.5])
    assert list(M.top_indices(s, 2)) == [1, 2]
    assert list(M.top_indices(s, 4)) == [0, 1, 2, 4]
