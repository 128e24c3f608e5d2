"""Plane waves amp cos(kx x + ky y - omega t + phase) as problem input: exact
cell averages on the grid (and on ghost cells outside it) and as TT cores.

A list of waves is a list of (field, amp, kx, ky, omega, phase).  A plane
wave's average over a dx x dy cell centred at (xc, yc) is its value there
times sinc(kx dx / 2) sinc(ky dy / 2), and it is a rank-2 TT:
cos(a + b) = cos a cos b - sin a sin b.
"""
import numpy as np


def _sinc(z):
    return 1.0 if z == 0.0 else float(np.sin(z) / z)


def waves_cellavg(waves, field, n, t, length=1.0, rows=None, ny=None):
    """Exact cell averages of the waves of `field` at time t on the n x n grid
    of [0, length]^2 -- or, with `rows`, on the cells of those x indices (any
    integers, ghost cells included) times all ny = n y cells."""
    ny = n if ny is None else ny
    dx = length / n
    xi = np.arange(n) if rows is None else np.asarray(rows)
    xc = (xi + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    out = np.zeros((len(xc), ny))
    for c, amp, kx, ky, om, ph in waves:
        if c != field:
            continue
        s = _sinc(kx * dx / 2) * _sinc(ky * dx / 2)
        out += amp * s * np.cos(kx * xc[:, None] + ky * yc[None, :] - om * t + ph)
    return out


def waves_tt(waves, field, n, t, length=1.0):
    """The cell averages of waves_cellavg as TT cores (A, B), rank 2 per wave
    (a zero rank-1 TT when the field has no wave)."""
    dx = length / n
    xc = (np.arange(n) + 0.5) * dx
    A, B = [], []
    for c, amp, kx, ky, om, ph in waves:
        if c != field:
            continue
        sx, sy = _sinc(kx * dx / 2), _sinc(ky * dx / 2)
        a = kx * xc
        b = ky * xc - om * t + ph
        A += [sx * np.cos(a), -sx * np.sin(a)]
        B += [amp * sy * np.cos(b), amp * sy * np.sin(b)]
    if not A:
        return np.zeros((n, 1)), np.zeros((n, 1))
    return np.stack(A, axis=1), np.stack(B, axis=1)
