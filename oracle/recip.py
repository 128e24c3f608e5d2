"""Oracle B, Taylor-series TT reciprocal (Algorithm 1, Sec. 4.2).

Oracle code (test infrastructure only).

With x_avg = sum(x)/N and x~ = round(1 - x/x_avg), 1/x = (1/x_avg) sum_k x~^k;
the loop adds the terms dy_k = round(dy_{k-1} o x~) until
Err = ||dy||_F / sqrt(N) <= eps (checked after each update; N = numel).
"""
import numpy as np

from . import tt as T


def reciprocal(x, tol, cap, max_iter=50):
    """Returns (y, iters) with y ~ 1/x entrywise."""
    n1, n2 = x[0].shape[0], x[1].shape[0]
    N = n1 * n2
    x_avg = T.tsum(x) / N
    y = T.const(1.0, n1, n2)
    dy = T.const(1.0, n1, n2)
    xt = T.rnd(T.add([(1.0, T.const(1.0, n1, n2)), (-1.0 / x_avg, x)]), tol, cap)
    err = 1.0
    it = 0
    while err > tol and it < max_iter:
        dy = T.rnd(T.hadamard(dy, xt), tol, cap)
        y = T.rnd(T.add([(1.0, y), (1.0, dy)]), tol, cap)
        err = T.fro(dy) / np.sqrt(N)
        it += 1
    return T.scale(1.0 / x_avg, y), it
