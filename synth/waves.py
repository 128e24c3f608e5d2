"""Plane waves amp cos(kx x + ky y - omega t + phase) as problem input: exact
cell averages on the grid (and on ghost cells outside it) and as TT cores.

A list of waves is a list of (field, amp, kx, ky, omega, phase), or
(field, amp, kx, ky, omega, phase, decay) for a wave damped in x,
amp exp(-decay x) cos(kx x + ky y - omega t + phase) (the coastal Kelvin
wave's profile, Sec. 5.1).  A plane wave's average over a dx x dy cell
centred at (xc, yc) is its value there times sinc(kx dx / 2) sinc(ky dy / 2),
and it is a rank-2 TT: cos(a + b) = cos a cos b - sin a sin b.  With a decay
the x factors exp(-decay x) cos(kx x) and exp(-decay x) sin(kx x) are
averaged exactly as the real and imaginary parts of the integral of
exp(z x), z = -decay + i kx, over the cell.
"""
import numpy as np


def _sinc(z):
    return 1.0 if z == 0.0 else float(np.sin(z) / z)


def _decay(w):
    return float(w[6]) if len(w) > 6 else 0.0


def _x_factors(kx, decay, xi, dx):
    """Cell averages over [i dx, (i + 1) dx] of exp(-decay x) cos(kx x) and
    exp(-decay x) sin(kx x) for the integers i of xi."""
    xi = np.asarray(xi, dtype=float)
    if decay == 0.0:
        s = _sinc(kx * dx / 2)
        a = kx * (xi + 0.5) * dx
        return s * np.cos(a), s * np.sin(a)
    z = complex(-decay, kx)
    # integral of exp(z x) over the cell = exp(z x1) (exp(z dx) - 1) / z, with
    # exp(z dx) - 1 formed without cancellation
    ed = np.expm1(-decay * dx)
    d = complex(ed * np.cos(kx * dx) - 2.0 * np.sin(kx * dx / 2) ** 2, np.exp(-decay * dx) * np.sin(kx * dx))
    x1 = xi * dx
    e1 = np.exp(-decay * x1) * (np.cos(kx * x1) + 1j * np.sin(kx * x1))
    avg = e1 * d / z / dx
    return avg.real, avg.imag


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
    for wv in waves:
        c, amp, kx, ky, om, ph = wv[:6]
        if c != field:
            continue
        dk = _decay(wv)
        if dk == 0.0:
            s = _sinc(kx * dx / 2) * _sinc(ky * dx / 2)
            out += amp * s * np.cos(kx * xc[:, None] + ky * yc[None, :] - om * t + ph)
        else:
            cx, sx = _x_factors(kx, dk, xi, dx)
            b = ky * yc - om * t + ph
            sy = amp * _sinc(ky * dx / 2)
            out += sy * (cx[:, None] * np.cos(b)[None, :] - sx[:, None] * np.sin(b)[None, :])
    return out


def waves_tt(waves, field, n, t, length=1.0):
    """The cell averages of waves_cellavg as TT cores (A, B), rank 2 per wave
    (a zero rank-1 TT when the field has no wave)."""
    dx = length / n
    xc = (np.arange(n) + 0.5) * dx
    A, B = [], []
    for wv in waves:
        c, amp, kx, ky, om, ph = wv[:6]
        if c != field:
            continue
        cx, snx = _x_factors(kx, _decay(wv), np.arange(n), dx)
        sy = _sinc(ky * dx / 2)
        b = ky * xc - om * t + ph
        A += [cx, -snx]
        B += [amp * sy * np.cos(b), amp * sy * np.sin(b)]
    if not A:
        return np.zeros((n, 1)), np.zeros((n, 1))
    return np.stack(A, axis=1), np.stack(B, axis=1)
