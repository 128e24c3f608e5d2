"""The linear SWE on a domain bounded in x with exact-solution boundary
values (Sec. 5.3's barotropic tide; periodic in y): Oracle A with ghost cells
holding the exact solution's cell averages converges to the tide at the
formal orders 3 / 5 / 5 in every field, and fails to when the boundary is
treated as periodic or the ghost rows are misplaced; Oracle B's TT form
(cores extended by the exact solution's ghost rows, non-periodic stencils on
the x-core) equals Oracle A's step on states of nontrivial TT rank."""
import math

import numpy as np
import pytest

from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_scales
from synth import kelvin, tide, waves

W = tide.tide_waves()
P = tide.tide_params()
G0 = FA.GHOST


def ghost_cells(n, t, shift=0):
    rows_l = np.arange(-G0, 0) + shift
    rows_r = np.arange(n, n + G0) + shift
    return ([waves.waves_cellavg(W, c, n, t, rows=rows_l) for c in range(3)],
            [waves.waves_cellavg(W, c, n, t, rows=rows_r) for c in range(3)])


def tide_errors(scheme, n, T_end=0.05, bc="exact"):
    dx = 1.0 / n
    c = math.sqrt(P["g"] * P["H"])
    dt0 = 0.4 * dx / c if scheme == "up3" else 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / c
    nst = int(math.ceil(T_end / dt0))
    dt = T_end / nst
    Q = [waves.waves_cellavg(W, k, n, 0.0) for k in range(3)]
    if bc == "exact":
        fun = lambda t: ghost_cells(n, t)  # noqa: E731
    elif bc == "shifted":
        fun = lambda t: ghost_cells(n, t, shift=1)  # noqa: E731
    else:
        fun = None
    t = 0.0
    for _ in range(nst):
        Q = FA.ssprk3_step(Q, "linear", scheme, P, dt, t=t, bc=fun)
        t += dt
    ex = [waves.waves_cellavg(W, k, n, t) for k in range(3)]
    return [np.linalg.norm(Q[k] - ex[k]) / np.linalg.norm(ex[k]) for k in range(3)]


@pytest.mark.parametrize("scheme,order,lo", [("up3", 3, 2.8), ("up5", 5, 4.7), ("weno5", 5, 4.6)])
def test_tide_converges_with_exact_boundary_cells(scheme, order, lo):
    e = [tide_errors(scheme, n) for n in (16, 32, 64)]
    for c in range(3):
        o = math.log2(e[1][c] / e[2][c])
        assert lo < o < order + 0.5, (scheme, c, e, o)


@pytest.mark.parametrize("bc", ["periodic", "shifted"])
def test_wrong_boundary_treatment_fails_to_converge(bc):
    e = [tide_errors("up5", n, bc=bc) for n in (16, 32)]
    assert max(e[1]) > 1e-2 or min(math.log2(e[0][c] / e[1][c]) for c in range(3)) < 2.0, (bc, e)


def rich_state(n):
    """The tide at t = 0 plus a y-dependent smooth perturbation (TT rank > 1)."""
    x = (np.arange(n) + 0.5) / n
    bump = np.exp(-((x[:, None] - 0.4) ** 2) / 0.02) * np.cos(2 * np.pi * x[None, :])
    base = [waves.waves_cellavg(W, k, n, 0.0) for k in range(3)]
    return [base[0] + 0.005 * bump, base[1] + 0.002 * bump.T + 0.001 * bump, base[2] - 0.001 * bump]


@pytest.mark.parametrize("scheme", ["up3", "up5"])
def test_tt_bounded_step_equals_full_tensor_step(scheme):
    n = 32
    dt = 0.4 / n / math.sqrt(P["g"]) * 0.5
    p = dict(P, dt=dt)
    Q = [T.tt_svd(f, 1e-15, n) for f in rich_state(n)]
    assert min(T.rank(q) for q in Q) > 1
    w = dict(eqn="linear", scheme=scheme, n=n, tol=1e-13, cap=n, bc_x="exact", boundary=W)
    t = 0.03
    out = TB.step(Q, w, p, seed=0, t=t)
    ref = FA.ssprk3_step([T.full(q) for q in Q], "linear", scheme, p, dt, t=t, bc=lambda s: ghost_cells(n, s))
    check_fields(out, ref, 1e-11, field_scales(ref, "linear", p, dt))


# ---------------------------------------------------------------- Kelvin wave
KW = kelvin.kelvin_waves()
KP = kelvin.kelvin_params()


def kelvin_point(waves_list, c, x, y, t):
    v = 0.0
    for f, amp, kx, ky, om, ph, dk in waves_list:
        if f == c:
            v = v + amp * np.exp(-dk * x) * np.cos(kx * x + ky * y - om * t + ph)
    return v


def swe_residuals(waves_list, p, x, y, t, h=1e-5):
    """The linear SWE's three residuals at (x, y, t) by central differences of
    the point values: eta_t + H (u_x + v_y), u_t - f v + g eta_x,
    v_t + f u + g eta_y (Sec. 2.1 with the Coriolis source)."""
    q = lambda c, dx=0.0, dy=0.0, dt=0.0: kelvin_point(waves_list, c, x + dx, y + dy, t + dt)  # noqa: E731
    d = lambda c, ax: ((q(c, **{ax: h}) - q(c, **{ax: -h})) / (2 * h))  # noqa: E731
    g, H, f = p["g"], p["H"], p["f"]
    return (d(0, "dt") + H * (d(1, "dx") + d(2, "dy")),
            d(1, "dt") - f * q(2) + g * d(0, "dx"),
            d(2, "dt") + f * q(1) + g * d(0, "dy"))


def test_kelvin_wave_solves_the_linear_swe():
    rng = np.random.default_rng(3)
    scale = max(abs(a) for _, a, *_ in KW) * max(abs(w[3]) * math.sqrt(KP["g"] * KP["H"]) for w in KW)
    for _ in range(20):
        x, y, t = rng.uniform(0.0, 1.0), rng.uniform(0.0, 1.0), rng.uniform(0.0, 1.0)
        r = swe_residuals(KW, KP, x, y, t)
        assert max(abs(v) for v in r) < 1e-6 * scale, r
    # a wrong decay length (R != c / f) or a wrong sign of v breaks it
    bad_f = dict(KP, f=1.2 * KP["f"])
    assert max(abs(v) for v in swe_residuals(KW, bad_f, 0.3, 0.4, 0.1)) > 1e-4 * scale
    flipped = [(f, -a if f == 2 else a, *rest) for f, a, *rest in KW]
    assert max(abs(v) for v in swe_residuals(flipped, KP, 0.3, 0.4, 0.1)) > 1e-4 * scale


def test_kelvin_cell_averages_are_exact():
    """The damped waves' cell averages (on the grid and on the ghost cells)
    equal a 12-point Gauss-Legendre quadrature of the point values, and their
    TT (Oracle B's cores) reconstructs them."""
    n, t = 16, 0.3
    xg, wg = np.polynomial.legendre.leggauss(12)
    rows = np.arange(-3, n + 3)
    for c in (0, 2):
        ca = waves.waves_cellavg(KW, c, n, t, rows=rows)
        q = np.zeros_like(ca)
        for ii, i in enumerate(rows):
            xs = (i + 0.5 + 0.5 * xg) / n
            for j in range(n):
                ys = (j + 0.5 + 0.5 * xg) / n
                vals = kelvin_point(KW, c, xs[:, None], ys[None, :], t)
                q[ii, j] = 0.25 * (wg[:, None] * wg[None, :] * vals).sum()
        assert np.abs(ca - q).max() <= 1e-14 * np.abs(q).max(), c
        A, B = TB.waves_tt(KW, c, n, n, t, 1.0, 1.0, rows=rows)
        assert np.abs(A @ B.T - ca).max() <= 1e-15 * np.abs(q).max(), c


def kelvin_ghost(n, t):
    g0 = FA.GHOST
    return ([waves.waves_cellavg(KW, c, n, t, rows=np.arange(-g0, 0)) for c in range(3)],
            [waves.waves_cellavg(KW, c, n, t, rows=np.arange(n, n + g0)) for c in range(3)])


def kelvin_errors(scheme, n, T_end=0.05):
    dx = 1.0 / n
    c = math.sqrt(KP["g"] * KP["H"])
    dt0 = 0.4 * dx / c if scheme == "up3" else 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / c
    nst = int(math.ceil(T_end / dt0))
    dt = T_end / nst
    Q = [waves.waves_cellavg(KW, k, n, 0.0) for k in range(3)]
    t = 0.0
    for _ in range(nst):
        Q = FA.ssprk3_step(Q, "linear", scheme, KP, dt, t=t, bc=lambda s: kelvin_ghost(n, s))
        t += dt
    ex = [waves.waves_cellavg(KW, k, n, t) for k in range(3)]
    # u = 0 exactly: its error relative to eta's scale
    return [np.linalg.norm(Q[0] - ex[0]) / np.linalg.norm(ex[0]),
            np.linalg.norm(Q[1]) / np.linalg.norm(ex[2]),
            np.linalg.norm(Q[2] - ex[2]) / np.linalg.norm(ex[2])]


@pytest.mark.parametrize("scheme,order,lo", [("up3", 3, 2.8), ("up5", 5, 4.6), ("weno5", 5, 4.5)])
def test_kelvin_wave_converges_with_exact_boundary_cells(scheme, order, lo):
    e = [kelvin_errors(scheme, n) for n in (16, 32, 64)]
    for c in range(3):
        o = math.log2(e[1][c] / e[2][c])
        assert lo < o < order + 0.7, (scheme, c, e, o)


@pytest.mark.parametrize("scheme", ["up3", "up5"])
def test_tt_bounded_step_equals_full_tensor_step_kelvin(scheme):
    n = 32
    dt = 0.4 / n / math.sqrt(KP["g"]) * 0.5
    p = dict(KP, dt=dt)
    full = [waves.waves_cellavg(KW, k, n, 0.0) for k in range(3)]
    full = [full[0] + 0.002 * rich_state(n)[0] - 0.002 * waves.waves_cellavg(W, 0, n, 0.0), full[1], full[2]]
    Q = [T.tt_svd(f, 1e-15, n) if np.linalg.norm(f) > 0 else (np.zeros((n, 1)), np.zeros((n, 1))) for f in full]
    w = dict(eqn="linear", scheme=scheme, n=n, tol=1e-13, cap=n, bc_x="exact", boundary=KW)
    t = 0.03
    out = TB.step(Q, w, p, seed=0, t=t)
    ref = FA.ssprk3_step([T.full(q) for q in Q], "linear", scheme, p, dt, t=t, bc=lambda s: kelvin_ghost(n, s))
    check_fields(out, ref, 1e-11, field_scales(ref, "linear", p, dt))
