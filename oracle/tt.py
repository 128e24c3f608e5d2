"""Oracle B, TT algebra for 2-D tensors (Sec. 3.1-3.2).

Oracle code (test infrastructure only).

A TT is a pair (A, B): A of shape (n1, r) and B of shape (n2, r), with
X[i, j] = sum_k A[i, k] B[j, k].  In the paper's notation (Eq. TT_def_2D)
X(i1, i2) = G1(i1) G2(i2), so G1 = A and G2 = B^T.
"""
import numpy as np


def full(X):
    A, B = X
    return A @ B.T


def rank(X):
    return X[0].shape[1]


def truncation_rank(s, tol, cap):
    """Smallest k with (sum_{i>k} s_i^2)^{1/2} <= tol * ||s||_2, then min(k, cap);
    at least 1 (a zero tensor keeps one zero column).  This is the "SVD
    truncate at tolerance eps_TT" of Sec. 3.2 read as a relative Frobenius
    bound."""
    s = np.asarray(s, dtype=float)
    tot = float(np.sum(s * s))
    if tot == 0.0:
        return 1
    # tail[k] = sum_{i>=k} s_i^2 (i zero-based): keeping k values leaves tail[k]
    tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
    bound = (tol * tol) * tot
    k = int(np.argmax(tail <= bound))
    return max(1, min(k, cap))


def round_tt(X, tol, cap):
    """TT rounding (Sec. 3.2): orthogonalise G2 by an RQ decomposition, then a
    truncated SVD of G1 R.

    With G2 = B^T, the RQ of G2 is the QR of B: B = Q_B R_B, G2 = R_B^T Q_B^T.
    Then G1 R_B^T = U S V^T and X = (U S)(Q_B V)^T; keep k columns.
    Returns (Y, info) with info = dict(rank_in, rank, sigma, err) where err is
    the discarded Frobenius norm."""
    A, B = X
    Qb, Rb = np.linalg.qr(B, mode="reduced")
    M = A @ Rb.T
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    k = truncation_rank(s, tol, cap)
    k = min(k, len(s)) if len(s) > 0 else 1
    A2 = U[:, :k] * s[:k][None, :]
    B2 = Qb @ Vt[:k, :].T
    err = float(np.sqrt(np.sum(s[k:] ** 2)))
    return (A2, B2), dict(rank_in=A.shape[1], rank=k, sigma=s, err=err)


def rnd(X, tol, cap):
    return round_tt(X, tol, cap)[0]


def tt_svd(F, tol, cap):
    """TT decomposition of a full matrix by truncated SVD (the 2-D TT-SVD)."""
    U, s, Vt = np.linalg.svd(F, full_matrices=False)
    k = truncation_rank(s, tol, cap)
    return (U[:, :k] * s[:k][None, :], Vt[:k, :].T)


def add(terms):
    """Linear combination sum_t c_t X_t by concatenating cores (Sec. 4.2: TT
    sums are exact with rank sum_t r_t).  terms: list of (coef, X)."""
    A = np.hstack([c * X[0] for c, X in terms])
    B = np.hstack([X[1] for _, X in terms])
    return (A, B)


def scale(c, X):
    return (c * X[0], X[1].copy())


def hadamard(X, Y):
    """Entrywise product in TT format: cores are row-wise Kronecker
    (Khatri-Rao) products, rank r_X r_Y."""
    A = (X[0][:, :, None] * Y[0][:, None, :]).reshape(X[0].shape[0], -1)
    B = (X[1][:, :, None] * Y[1][:, None, :]).reshape(X[1].shape[0], -1)
    return (A, B)


def const(c, n1, n2):
    return (np.full((n1, 1), float(c)), np.ones((n2, 1)))


def tsum(X):
    """sum_{i,j} X[i,j] = (1^T A)(B^T 1)."""
    return float(np.sum(X[0].sum(axis=0) * X[1].sum(axis=0)))


def fro(X):
    """||X||_F from the core Gram matrices: ||X||_F^2 = sum (A^T A) o (B^T B)."""
    GA = X[0].T @ X[0]
    GB = X[1].T @ X[1]
    return float(np.sqrt(max(np.sum(GA * GB), 0.0)))


def numel(X):
    return X[0].shape[0] * X[1].shape[0]


# ---------------------------------------------------------------------------
# Core operators: shifts T^{x,y} and linear stencils act on one core only.
# ---------------------------------------------------------------------------

def shift(X, s, mode):
    """(T^s X)[i, j] = X[i+s, j] (mode 0) or X[i, j+s] (mode 1), periodic."""
    A, B = X
    if mode == 0:
        return (np.roll(A, -s, axis=0), B.copy())
    return (A.copy(), np.roll(B, -s, axis=0))


def core_stencil(C, stencil):
    """sum_s c_s C[i+s, :] (periodic along rows); stencil: dict offset->coef."""
    out = np.zeros_like(C)
    for s, c in stencil.items():
        out += float(c) * np.roll(C, -s, axis=0)
    return out
