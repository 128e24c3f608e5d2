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
from synth import tide, waves

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
