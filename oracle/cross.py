"""Oracle B, maxvol-based cross interpolation of a 2-D tensor (Sec. 3.3).

Oracle code (test infrastructure only).

The paper calls AMEn cross from the MATLAB TT-Toolbox, whose internals it does
not give.  This is a plain alternating row/column maximum-volume cross
(skeleton / CUR decomposition with the maximum-volume principle of Goreinov
et al.) with rank adaptation by "kick" fibres, written from that principle:

  1. column pivots J from the maxvol rows of an orthonormal basis of the
     initial guess's second core;
  2. sweep: evaluate the column fibres F(:, J u kick), take their leading
     left singular vectors (truncated at tol / 2 and the rank cap), choose
     rows I by maxvol; evaluate the row fibres F(I u kick, :), take their
     leading right singular vectors (same truncation), choose new columns J
     by maxvol.  The fibre truncation sits below the convergence test's tol:
     a skeleton truncated at tol itself predicts fresh fibres to about tol,
     and the test of step 3 would pass or fail on their noise;
  3. stop when the current skeleton predicts the next sweep's column fibres to
     relative Frobenius error <= tol, when the rank cap is reached with
     stationary column pivots, when a sweep no longer halves that
     prediction error while the skeleton is at the rank cap (a cap-limited
     skeleton cannot reach tol; further sweeps only reshuffle its pivots) or
     the error is already within 10 tol (a plateau just above tol), or after
     max_sweeps sweeps;
  4. return the skeleton X = U_c U_c[I]^{-1} F(I, :), then TT-round it.

Kick indices come from SplitMix64 (Steele, Lea & Flood, 2014) driven by a
counter, so both implementations draw the same indices without sharing code.
Pivot sets are not unique: only the approximation error is pinned.
"""
import numpy as np

from . import tt as T

MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output for state increment x (published constants)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def kick_indices(n, count, seed, sweep, exclude):
    """`count` distinct indices in [0, n) not in `exclude`, drawn in order from
    splitmix64(seed * 2^32 + sweep * 2^16 + t), t = 0, 1, ..."""
    out = []
    ex = set(int(e) for e in exclude)
    t = 0
    limit = 64 * (count + 1) + n
    while len(out) < count and t < limit:
        v = splitmix64(((seed & 0xFFFFFFFF) << 32) + ((sweep & 0xFFFF) << 16) + t) % n
        t += 1
        if v in ex:
            continue
        ex.add(v)
        out.append(v)
    return out


def lu_pivot_rows(U):
    """Row pivots of Gaussian elimination with partial pivoting on U (n x r),
    rows left in place: at step k the not-yet-chosen row with the largest
    |W[i, k]| (ties: the smallest row index) becomes pivot k, and every other
    unchosen row is eliminated against it."""
    W = np.array(U, dtype=float, copy=True)
    n, r = W.shape
    free = np.ones(n, dtype=bool)
    piv = []
    for k in range(r):
        col = np.where(free, np.abs(W[:, k]), -1.0)
        p = int(np.argmax(col))
        piv.append(p)
        free[p] = False
        if W[p, k] != 0.0:
            f = np.where(free, W[:, k] / W[p, k], 0.0)
            W[:, k:] -= np.outer(f, W[p, k:])
    return piv


def maxvol(U, delta=1e-2, max_iter=200):
    """Rows I (len r) of U (n x r, n >= r) of locally maximal volume: swap rows
    until every |B_ij| <= 1 + delta with B = U U[I]^{-1} (Goreinov et al.).
    argmax ties go to the smallest row-major linear index."""
    n, r = U.shape
    I = lu_pivot_rows(U)
    B = np.linalg.solve(U[I, :].T, U.T).T
    for _ in range(max_iter):
        flat = int(np.argmax(np.abs(B)))
        i, j = divmod(flat, r)
        piv = B[i, j]
        if abs(piv) <= 1.0 + delta:
            break
        bj = B[:, j].copy()
        bi = B[i, :].copy()
        bi[j] -= 1.0
        B -= np.outer(bj, bi) / piv
        I[j] = i
    return list(I)


def _orth_left(C, tol, cap):
    """Leading left singular vectors of C truncated at (tol, cap)."""
    U, s, _ = np.linalg.svd(C, full_matrices=False)
    k = T.truncation_rank(s, tol, cap)
    return U[:, :k]


def cross2d(evalF, n1, n2, x0, tol, cap, kick=4, max_sweeps=10, seed=0,
            return_info=False):
    """Cross-approximate the n1 x n2 matrix F, available entrywise through
    evalF(I, J) -> F[np.ix_(I, J)], starting from the TT guess x0."""
    Qb, _ = np.linalg.qr(x0[1], mode="reduced")
    r0 = max(1, min(Qb.shape[1], cap, n1, n2))
    J = maxvol(Qb[:, :r0]) if Qb.shape[0] > r0 else list(range(Qb.shape[0]))
    rows = np.arange(n1)
    cols = np.arange(n2)
    prev = None
    sweeps = 0
    err = np.inf
    for s in range(max_sweeps):
        sweeps = s + 1
        Jx = list(J) + kick_indices(n2, min(kick, n2 - len(J)), seed, 2 * s, J)
        C = evalF(rows, np.array(Jx))
        if prev is not None:
            Uc, I, RI = prev
            pred = Uc @ np.linalg.solve(Uc[I, :], RI[:, Jx])
            nc = np.linalg.norm(C)
            err_prev = err
            err = np.linalg.norm(C - pred) / nc if nc > 0 else 0.0
            if err <= tol:
                break
            if np.isfinite(err_prev) and err > 0.5 * err_prev and (len(I) >= cap or err <= 10 * tol):
                break
        Uc = _orth_left(C, 0.5 * tol, cap)
        I = maxvol(Uc)
        Ix = list(I) + kick_indices(n1, min(kick, n1 - len(I)), seed, 2 * s + 1, I)
        R = evalF(np.array(Ix), cols)
        prev = (Uc, I, R[:len(I), :])
        Vr = _orth_left(R.T, 0.5 * tol, cap)
        Jn = maxvol(Vr)
        if len(Jn) >= cap and set(Jn) == set(J):
            break  # rank cap reached with stationary pivots: no further gain
        J = Jn
    Uc, I, RI = prev
    A = np.linalg.solve(Uc[I, :].T, Uc.T).T
    Y, rinfo = T.round_tt((A, RI.T.copy()), tol, cap)
    if return_info:
        return Y, dict(sweeps=sweeps, err=err, rank=rinfo["rank"])
    return Y
