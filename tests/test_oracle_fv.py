"""Pins of Oracle A (full-tensor finite volume, Sec. 2) against the closed-form
inertia-gravity wave (Sec. 5.2), conservation and steady states."""
import math

import numpy as np
import pytest

from oracle import fv_full as FA
from synth import igw_cellavg, initial_tt, tt_to_full, workload

G, H, F = 9.81, 1.0, 1.0


def _igw_error(scheme, n, T=0.02):
    p = dict(g=G, H=H, f=F, lx=1.0, ly=1.0)
    dx = 1.0 / n
    c = math.sqrt(G * H)
    if scheme == "up3":
        dt0 = 0.4 * dx / c
    else:  # dt proportional to dx^(5/3) (Sec. 5) so the RK3 error stays O(dx^5)
        dt0 = 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / c
    nst = int(math.ceil(T / dt0))
    dt = T / nst
    Q = igw_cellavg(n, 0.0, g=G, H=H, f=F)
    for _ in range(nst):
        Q = FA.ssprk3_step(Q, "linear", scheme, p, dt)
    ex = igw_cellavg(n, T, g=G, H=H, f=F)
    return np.linalg.norm(Q[0] - ex[0]) / np.linalg.norm(ex[0])


@pytest.mark.parametrize("scheme,order,lo", [("up3", 3, 2.8), ("up5", 5, 4.7), ("weno5", 5, 4.7)])
def test_igw_convergence_order(scheme, order, lo):
    e = [_igw_error(scheme, n) for n in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert orders[-1] > lo, (scheme, e, orders)
    assert orders[-1] < order + 0.5


def test_igw_closed_form_satisfies_dispersion():
    # the closed form solves the linear SWE: its time derivative by central
    # differences matches -(H du/dx ...) computed spectrally on a fine grid
    n = 64
    dt = 1e-5
    a = igw_cellavg(n, dt)
    b = igw_cellavg(n, -dt)
    dQ = [(a[c] - b[c]) / (2 * dt) for c in range(3)]
    Q = igw_cellavg(n, 0.0)
    k = 2 * np.pi * np.fft.fftfreq(n, d=1.0 / n)

    def ddx(f, axis):
        return np.real(np.fft.ifft(1j * k.reshape((-1, 1) if axis == 0 else (1, -1)) *
                                   np.fft.fft(f, axis=axis), axis=axis))
    eta, u, v = Q
    r0 = -(H * ddx(u, 0) + H * ddx(v, 1))
    r1 = -G * ddx(eta, 0) + F * v
    r2 = -G * ddx(eta, 1) - F * u
    for c, r in enumerate((r0, r1, r2)):
        assert np.max(np.abs(dQ[c] - r)) < 1e-6 * np.max(np.abs(r))


@pytest.mark.parametrize("scheme", ["up3", "up5", "weno5"])
def test_mass_conservation_nonlinear(scheme):
    w = workload("nonlinear256_weno5", n=32, scheme=scheme)
    Qt, p = initial_tt(w)
    Q = [tt_to_full(*q) for q in Qt]
    m0 = Q[0].sum()
    for _ in range(3):
        Q = FA.ssprk3_step(Q, "nonlinear", scheme, p, p["dt"])
    assert abs(Q[0].sum() - m0) <= 1e-13 * abs(m0)
    # momentum is conserved too with f = 0 (telescoping fluxes, no source)
    assert abs(Q[1].sum()) <= 1e-12 * np.abs(Q[1]).sum()


@pytest.mark.parametrize("scheme", ["up3", "up5", "weno5"])
def test_lake_at_rest_is_steady(scheme):
    n = 16
    p = dict(g=G, H=1.0, f=0.5, lx=1.0, ly=1.0)
    Q = [np.full((n, n), 1.3), np.zeros((n, n)), np.zeros((n, n))]
    L = FA.rhs(Q, "nonlinear", scheme, p)
    for c in range(3):
        assert np.max(np.abs(L[c])) < 1e-12


def test_x_y_symmetry():
    # a field and its transpose evolve into transposes (with u <-> v)
    w = workload("nonlinear256_weno5", n=24, scheme="weno5")
    Qt, p = initial_tt(w)
    Q = [tt_to_full(*q) for q in Qt]
    Q[1] = 0.01 * np.sin(2 * np.pi * np.arange(24) / 24)[:, None] * np.ones((1, 24))
    QT = [Q[0].T.copy(), Q[2].T.copy(), Q[1].T.copy()]
    a = FA.euler(Q, "nonlinear", "weno5", p, p["dt"])
    b = FA.euler(QT, "nonlinear", "weno5", p, p["dt"])
    np.testing.assert_allclose(a[0].T, b[0], atol=1e-14)
    np.testing.assert_allclose(a[1].T, b[2], atol=1e-14)


def test_planted_sign_error_breaks_convergence(monkeypatch):
    # a plausible slip -- using the "-" side stencil on the "+" side -- must
    # fail the convergence pin
    orig = FA.step1

    def wrong(v, axis, scheme, side, eps):
        return orig(v, axis, scheme, "-", eps)
    monkeypatch.setattr(FA, "step1", wrong)
    e = [_igw_error("up3", n) for n in (16, 32)]
    assert math.log2(e[0] / e[1]) < 2.5 or e[1] > 1e-2


def test_weno5_step_data_has_no_new_extrema():
    # a periodic box profile (two unit jumps): the WENO5 reconstructions of
    # Steps 1 and 2 stay within the cell averages' range up to O(eps), eps =
    # dx^2 (Sec. 2.3), while the linear Upwind5/Upwind3 stencils overshoot
    # by 17-18 %; a WENO weight that fell back to the linear weights fails
    n = 64
    x = (np.arange(n) + 0.5) / n
    v = np.where((x > 0.25) & (x < 0.6), 1.0, 0.0)[:, None] * np.ones((1, n))
    eps = (1.0 / n) ** 2
    for side in ("-", "+"):
        f = FA.step1(v, 0, "weno5", side, eps)
        assert f.min() >= -eps and f.max() <= 1.0 + eps, side
        for lin in ("up5", "up3"):
            g = FA.step1(v, 0, lin, side, eps)
            assert g.min() < -0.1 and g.max() > 1.1, (lin, side)
    pts = FA.step2(v, 0, "weno5", eps)
    assert np.min(pts) >= -eps and np.max(pts) <= 1.0 + eps
    lin = FA.step2(v, 0, "up5", eps)
    assert np.min(lin) < -0.1 and np.max(lin) > 1.1

