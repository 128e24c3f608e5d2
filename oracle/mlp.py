"""Pivot-proposal perceptron of the learned-pivot form -- FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline; the CUDA path never calls it.

The paper's cross interpolation (Sec. 3.3) starts from some pivot set and
refines it by maxvol sweeps; it prescribes no learned component.  The learned
form adds a network that scores every column index j of a cross from
features of the cross's initial TT (its second core) and local smoothness
indicators; the top-scoring indices seed the sweeps, which keep judging the
interpolation error, so plain maxvol remains the fallback.  Everything here
is this project's own construction, written out plainly:

features(A, B, prev)  -> X (n2 x F), F = 14 columns per index j:
  0  leverage l_j = (n2 / r) ||Q[j, :]||^2 with Q an orthonormal basis of B
  1-4 leverages of j-2, j-1, j+1, j+2 (periodic in j)
  5  column mean c_j = mean_i (A B^T)[i, j], standardised over j
  6  centred first difference (c_{j+1} - c_{j-1}) / 2, scaled by std(c)
  7  second difference c_{j+1} - 2 c_j + c_{j-1}, scaled by std(c)
  8  log(1 + |second difference| / (mean |second difference| + 1e-300))
  9  column energy ||(A B^T)[:, j]||^2 / mean over j
  10, 11  sin, cos of 2 pi j / n2
  12  1 if j is in `prev`, the converged column pivots of the same cross
      site at the previous stage, else 0
  13  min(periodic distance from j to `prev`, 8) / 8 (1 when prev is empty)
(std(c) and the means are over j; a spread below 1e-12 mean|c| -- a flat
profile up to round-off -- is replaced by 1.)

network: H1 = relu(X W1 + b1) (F -> 256), H2 = relu(H1 W2 + b2) (256 -> 256),
s = H2 w3 + b3 (256 -> 1), one score per index.
loss: mean over rows of the logistic loss softplus(s) - y s, y = 1 for an
index in the converged pivot set of a plain cross, else 0.
optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights.
precision: every matrix product of the forward and backward passes reads its
two operands rounded to BF16 (round to nearest, ties to even) and
accumulates exactly here (in FP32 on the tensor cores); biases, activations,
masks, the loss and the optimiser stay in higher precision.  The backward
pass treats the roundings as the identity (the products' own operands are
differentiated), so it is the exact gradient of the unrounded network when
bf16=False.
"""
import numpy as np

F_IN = 14
HIDDEN = 256


def features(A, B, prev=()):
    """Index features of the column mode of X = A B^T (A n1 x r, B n2 x r);
    prev: the previous converged pivot indices of the same cross site."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n1, r = A.shape
    n2 = B.shape[0]
    Q, _ = np.linalg.qr(B)
    lev = (n2 / r) * np.sum(Q * Q, axis=1)
    X = np.zeros((n2, F_IN))
    X[:, 0] = lev
    for col, sh in zip((1, 2, 3, 4), (2, 1, -1, -2)):
        X[:, col] = np.roll(lev, sh)  # value at j - sh
    c = B @ A.mean(axis=0)
    sd = c.std()
    sd = sd if sd > 1e-12 * np.abs(c).mean() else 1.0
    X[:, 5] = (c - c.mean()) / sd
    cp, cm = np.roll(c, -1), np.roll(c, 1)
    X[:, 6] = 0.5 * (cp - cm) / sd
    d2 = cp - 2.0 * c + cm
    X[:, 7] = d2 / sd
    X[:, 8] = np.log1p(np.abs(d2) / (np.abs(d2).mean() + 1e-300))
    G = A.T @ A
    e = np.einsum("jk,kl,jl->j", B, G, B)
    me = e.mean()
    X[:, 9] = e / (me if me > 0 else 1.0)
    ang = 2.0 * np.pi * np.arange(n2) / n2
    X[:, 10] = np.sin(ang)
    X[:, 11] = np.cos(ang)
    prev = np.asarray(list(prev), dtype=np.int64)
    if prev.size:
        X[prev, 12] = 1.0
        j = np.arange(n2)[:, None]
        d = np.abs(j - prev[None, :])
        d = np.minimum(d, n2 - d).min(axis=1)
        X[:, 13] = np.minimum(d, 8) / 8.0
    else:
        X[:, 13] = 1.0
    return X


def bf16(x):
    """Round FP32-representable values to BF16 (nearest, ties to even)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def init_params(seed):
    """He-uniform initial weights from default_rng(seed), zero biases (FP32)."""
    rng = np.random.default_rng(seed)

    def u(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=shape).astype(np.float32)

    return dict(W1=u(F_IN, (F_IN, HIDDEN)), b1=np.zeros(HIDDEN, np.float32),
                W2=u(HIDDEN, (HIDDEN, HIDDEN)), b2=np.zeros(HIDDEN, np.float32),
                w3=u(HIDDEN, (HIDDEN,)), b3=np.zeros(1, np.float32))


def mm(A, B, bf16_ops=True):
    """A @ B with both operands rounded to BF16 first (when bf16_ops)."""
    if bf16_ops:
        return bf16(A) @ bf16(B)
    return np.asarray(A, np.float64) @ np.asarray(B, np.float64)


def forward(P, X, bf16_ops=True):
    """Scores (m,) and the cached activations of rows X (m x F)."""
    W1 = np.asarray(P["W1"], np.float64)
    W2 = np.asarray(P["W2"], np.float64)
    w3 = np.asarray(P["w3"], np.float64)
    Z1 = mm(X, W1, bf16_ops) + np.asarray(P["b1"], np.float64)
    H1 = np.maximum(Z1, 0.0)
    Z2 = mm(H1, W2, bf16_ops) + np.asarray(P["b2"], np.float64)
    H2 = np.maximum(Z2, 0.0)
    s = mm(H2, w3[:, None], bf16_ops)[:, 0] + float(P["b3"][0])
    return s, dict(X=np.asarray(X, np.float64), Z1=Z1, H1=H1, Z2=Z2, H2=H2, W1=W1, W2=W2, w3=w3,
                   bf16_ops=bf16_ops)


def loss(s, y):
    """Mean logistic loss softplus(s) - y s (stable form)."""
    return float(np.mean(np.maximum(s, 0.0) + np.log1p(np.exp(-np.abs(s))) - y * s))


def backward(s, y, cache):
    """Gradients of the mean logistic loss w.r.t. W1, b1, W2, b2, w3, b3."""
    o = cache["bf16_ops"]
    m = s.shape[0]
    ds = (1.0 / (1.0 + np.exp(-s)) - y) / m
    g = {}
    g["w3"] = mm(cache["H2"].T, ds[:, None], o)[:, 0]
    g["b3"] = np.array([ds.sum()])
    dH2 = mm(ds[:, None], cache["w3"][None, :], o)
    dZ2 = dH2 * (cache["Z2"] > 0)
    g["W2"] = mm(cache["H1"].T, dZ2, o)
    g["b2"] = dZ2.sum(axis=0)
    dH1 = mm(dZ2, cache["W2"].T, o)
    dZ1 = dH1 * (cache["Z1"] > 0)
    g["W1"] = mm(cache["X"].T, dZ1, o)
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam(P, g, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the FP32 master parameters (step t >= 1)."""
    out = {}
    for k in P:
        m = b1 * state.get("m" + k, 0.0) + (1 - b1) * g[k]
        v = b2 * state.get("v" + k, 0.0) + (1 - b2) * g[k] * g[k]
        state["m" + k], state["v" + k] = m, v
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        out[k] = (np.asarray(P[k], np.float64) - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)
    return out


def top_indices(s, k):
    """The k highest scores' indices, ties to the smaller index, ascending."""
    order = np.lexsort((np.arange(s.shape[0]), -s))
    return np.sort(order[:k])
