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


@pytest.mark.parametrize("round_weights", [False, True])
def test_backward_matches_central_differences(round_weights):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, M.F_IN))
    y = (rng.random(40) < 0.3).astype(np.float64)
    P = small_params(2)
    # differentiate the network at exactly the weights the forward pass uses
    Pd = {k: np.asarray(v, np.float64) for k, v in P.items()}
    if round_weights:
        for k in ("W1", "W2", "w3"):
            Pd[k] = M.bf16(P[k])
    s, cache = M.forward(Pd, X, round_weights=False)
    g = M.backward(s, y, cache)
    h = 1e-6
    for k in Pd:
        flat = Pd[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(M.forward(Pd, X, round_weights=False)[0], y)
            flat[idx] = old - h
            lm = M.loss(M.forward(Pd, X, round_weights=False)[0], y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)), (k, idx, fd, an)


def test_forward_uses_bf16_weights():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((8, M.F_IN))
    P = small_params(5)
    s_r, _ = M.forward(P, X, round_weights=True)
    Pr = dict(P, W1=M.bf16(P["W1"]), W2=M.bf16(P["W2"]), w3=M.bf16(P["w3"]))
    s_e, _ = M.forward(Pr, X, round_weights=False)
    assert np.array_equal(s_r, s_e)


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


def test_top_indices_ties_to_smaller_index():
    s = np.array([0.5, 2.0, 2.0, -1.0, 2.0, 0.5])
    assert list(M.top_indices(s, 2)) == [1, 2]
    assert list(M.top_indices(s, 4)) == [0, 1, 2, 4]
