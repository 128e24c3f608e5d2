"""Pins of Oracle A's nonlinear physical flux, LLF wave speed and source term
(Sec. 2.1, Eq. nonlinear-SWE; Sec. 2.4, Eq. LLF) against facts of the
shallow water equations that do not come from the oracle's own formulas:

* characteristic speeds: the flux Jacobians dF/dQ and dG/dQ have the
  eigenvalues u_n - c, u_n, u_n + c with c = sqrt(g h) (the textbook
  eigenstructure of the SWE; Sec. 2.4 takes lambda as the largest of them);
* an exact nonlinear solution: a 1-D simple wave (constant Riemann invariant
  u_n - 2c, straight characteristics of speed u_n + c) running along the
  diagonal with a constant tangential velocity, so every flux term -- the
  advective hu^2/h, hv^2/h, the cross term hu hv / h and the pressure
  g h^2 / 2 in both directions -- is exercised; the full-tensor scheme must
  converge to it at the formal orders 3 / 5 / 5 in every field;
* an exact steady state with rotation: a diagonal geostrophic jet
  h = h(x + y) with the velocity along the isolines and g grad h balanced by
  the Coriolis term (0, f hv, -f hu); the discrete operator must vanish at
  the formal order.

Each pin is paired with planted mistakes (a wrong 1/2 on g h^2, a missing
1/h, the cross term in the wrong component, a wrong source sign, a wrong
wave speed) that it must catch.
"""
import math

import numpy as np
import pytest

from oracle import fv_full as FA

G = 9.81


# ---------------------------------------------------------------- exact solutions

def simple_wave_cellavg(n, t, a=0.1, ut=0.3, g=G, npts=6):
    """Exact cell averages of (h, hu, hv) of a smooth simple wave at time t.

    Dependence on s = x + y only (period 1 on the unit square), normal
    n = (1, 1)/sqrt(2), tangent (-1, 1)/sqrt(2).  Along the normal
    coordinate sigma = s / sqrt(2) the 1-D SWE keeps the Riemann invariant
    u_n - 2c constant (= -2 sqrt(g)), so c = sqrt(g h) is carried along
    straight characteristics of speed u_n + c = -2 sqrt(g) + 3c:
    c(s, t) = c0(s0) with s = s0 + sqrt(2) (-2 sqrt(g) + 3 c0(s0)) t
    (solved for s0 by Newton).  The tangential velocity u_t is constant
    (it is advected).  h0(s) = 1 + a sin(2 pi s); the characteristics
    first cross near t = 0.23 for a = 0.1."""
    R = -2.0 * math.sqrt(g)
    x, w = np.polynomial.legendre.leggauss(npts)
    dx = 1.0 / n
    k = np.arange(n)
    # s at the Gauss points of the cells (i, j) with i + j = k (mod n)
    s = (k[:, None, None] + 1.0) * dx + 0.5 * dx * (x[None, :, None] + x[None, None, :])
    s0 = s.copy()
    for _ in range(60):
        c0 = np.sqrt(g * (1.0 + a * np.sin(2 * np.pi * s0)))
        F = s0 + math.sqrt(2.0) * (R + 3.0 * c0) * t - s
        dF = 1.0 + 3.0 * math.sqrt(2.0) * t * g * (2 * np.pi * a * np.cos(2 * np.pi * s0)) / (2.0 * c0)
        d = F / dF
        s0 = s0 - d
        if np.max(np.abs(d)) < 1e-15:
            break
    c = np.sqrt(g * (1.0 + a * np.sin(2 * np.pi * s0)))
    h = c * c / g
    un = R + 2.0 * c
    u = (un - ut) / math.sqrt(2.0)
    v = (un + ut) / math.sqrt(2.0)
    W = 0.25 * w[None, :, None] * w[None, None, :]
    avg = [np.sum(W * q, axis=(1, 2)) for q in (h, h * u, h * v)]
    idx = (k[:, None] + k[None, :]) % n
    return [q[idx] for q in avg]


def geostrophic_jet_cellavg(n, a=0.1, f=10.0, g=G):
    """Exact cell averages of a steady diagonal jet of the rotating nonlinear
    SWE: h = 1 + a sin(2 pi s), s = x + y, velocity (u, v) = alpha (1, -1)
    along the isolines with g h'(s) = -f alpha, so the pressure gradient
    balances the Coriolis source and the advection u.grad vanishes.  The
    cell average of a function of x + y with wavenumber 2 pi m is its value
    at the cell centre times sinc(pi m dx)^2."""
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    S = xc[:, None] + xc[None, :]

    def sinc2(m):
        z = math.pi * m * dx
        return (math.sin(z) / z) ** 2
    h = 1.0 + a * np.sin(2 * np.pi * S) * sinc2(1)
    # alpha = -(g/f) h' = -(g/f) 2 pi a cos;  h alpha = -(g/f) 2 pi a (cos + (a/2) sin 2)
    c = -(g / f) * 2 * np.pi * a
    halpha = c * (np.cos(2 * np.pi * S) * sinc2(1) + 0.5 * a * np.sin(4 * np.pi * S) * sinc2(2))
    return [h, halpha, -halpha]


# ---------------------------------------------------------------- helpers

def simple_wave_errors(scheme, n, T=0.04):
    """Per-field relative L2 errors of Oracle A (nonlinear, f = 0) against the
    exact simple wave at time T; dt ~ dx (Upwind3) or dx^(5/3) (5th order,
    Sec. 5) so that SSP-RK3 stays below the spatial error."""
    p = dict(g=G, H=1.0, f=0.0, lx=1.0, ly=1.0)
    dx = 1.0 / n
    smax = 0.35 + math.sqrt(G * 1.1)
    if scheme == "up3":
        dt0 = 0.4 * dx / smax
    else:
        dt0 = 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / smax
    nst = int(math.ceil(T / dt0))
    dt = T / nst
    Q = simple_wave_cellavg(n, 0.0)
    for _ in range(nst):
        Q = FA.ssprk3_step(Q, "nonlinear", scheme, p, dt)
    ex = simple_wave_cellavg(n, T)
    return [np.linalg.norm(Q[c] - ex[c]) / np.linalg.norm(ex[c]) for c in range(3)]


def jet_residuals(scheme, n, f=10.0):
    """max over fields of ||L(Q)||_2 / sqrt(cells) at the exact steady jet."""
    p = dict(g=G, H=1.0, f=f, lx=1.0, ly=1.0)
    Q = geostrophic_jet_cellavg(n, f=f)
    L = FA.rhs(Q, "nonlinear", scheme, p)
    return max(np.linalg.norm(L[c]) / n for c in range(3))


def numeric_jacobian(Q, direction, eps=1e-6):
    """dF/dQ (3 x 3) of Oracle A's physical flux by central differences."""
    p = dict(g=G, H=1.0, f=0.0)
    J = np.zeros((3, 3))
    for k in range(3):
        d = eps * max(1.0, abs(Q[k]))
        qp = [np.array([q + (d if i == k else 0.0)]) for i, q in enumerate(Q)]
        qm = [np.array([q - (d if i == k else 0.0)]) for i, q in enumerate(Q)]
        fp = FA.phys_flux(qp, direction, "nonlinear", p)
        fm = FA.phys_flux(qm, direction, "nonlinear", p)
        for c in range(3):
            J[c, k] = (fp[c][0] - fm[c][0]) / (2 * d)
    return J


def random_states(count=40, seed=5):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.2, 3.0, count)
    u = rng.uniform(-2.0, 2.0, count)
    v = rng.uniform(-2.0, 2.0, count)
    return [(h[i], h[i] * u[i], h[i] * v[i]) for i in range(count)]


# ---------------------------------------------------------------- the pins

@pytest.mark.parametrize("direction", ["x", "y"])
def test_flux_jacobian_has_the_swe_characteristic_speeds(direction):
    for h, hu, hv in random_states():
        J = numeric_jacobian((h, hu, hv), direction)
        un = (hu if direction == "x" else hv) / h
        c = math.sqrt(G * h)
        ev = np.sort(np.linalg.eigvals(J).real)
        np.testing.assert_allclose(ev, [un - c, un, un + c], rtol=0, atol=2e-6 * (abs(un) + c))


@pytest.mark.parametrize("direction", ["x", "y"])
def test_llf_speed_is_the_largest_jacobian_eigenvalue(direction):
    # lambda of Eq. LLF: the largest |eigenvalue| over the two face states
    st = random_states(count=40, seed=9)
    for (qa, qb) in zip(st[::2], st[1::2]):
        Qm = [np.array([x]) for x in qa]
        Qp = [np.array([x]) for x in qb]
        lam = float(FA.max_speed(Qm, Qp, direction, "nonlinear", dict(g=G, H=1.0))[0])
        want = max(np.max(np.abs(np.linalg.eigvals(numeric_jacobian(q, direction)))) for q in (qa, qb))
        assert abs(lam - want) <= 2e-6 * want


@pytest.mark.parametrize("scheme,order,lo", [("up3", 3, 2.8), ("up5", 5, 4.6), ("weno5", 5, 4.6)])
def test_simple_wave_convergence_order_every_field(scheme, order, lo):
    e = [simple_wave_errors(scheme, n) for n in (16, 32, 64)]
    for c in range(3):
        o = math.log2(e[1][c] / e[2][c])
        assert lo < o < order + 0.5, (scheme, c, e, o)


@pytest.mark.parametrize("scheme,order,lo", [("up3", 3, 2.7), ("up5", 5, 4.5), ("weno5", 5, 4.5)])
def test_geostrophic_jet_is_steady_to_formal_order(scheme, order, lo):
    r = [jet_residuals(scheme, n) for n in (16, 32, 64)]
    o = math.log2(r[1] / r[2])
    assert lo < o < order + 0.7, (scheme, r, o)


# ---------------------------------------------------------------- planted mistakes

def _flux_variant(kind):
    orig = FA.phys_flux

    def flux(Q, direction, eqn, p):
        if eqn != "nonlinear":
            return orig(Q, direction, eqn, p)
        g = p["g"]
        h, hu, hv = Q
        if kind == "pressure":  # g h^2 instead of g h^2 / 2
            return (hu, hu * hu / h + g * h * h, hu * hv / h) if direction == "x" else \
                (hv, hu * hv / h, hv * hv / h + g * h * h)
        if kind == "no_inv_h":  # (hu)^2 without 1/h, everywhere
            return (hu, hu * hu + 0.5 * g * h * h, hu * hv) if direction == "x" else \
                (hv, hu * hv, hv * hv + 0.5 * g * h * h)
        if kind == "cross_swapped":  # the cross term in the wrong component of G
            return orig(Q, direction, eqn, p) if direction == "x" else \
                (hv, hv * hv / h, hu * hv / h + 0.5 * g * h * h)
        raise ValueError(kind)
    return flux


@pytest.mark.parametrize("kind", ["pressure", "no_inv_h", "cross_swapped"])
def test_planted_flux_mistakes_fail_the_pins(monkeypatch, kind):
    monkeypatch.setattr(FA, "phys_flux", _flux_variant(kind))
    caught = []
    # eigenvalue pin
    bad = False
    for direction in ("x", "y"):
        for h, hu, hv in random_states(count=6):
            J = numeric_jacobian((h, hu, hv), direction)
            un = (hu if direction == "x" else hv) / h
            c = math.sqrt(G * h)
            ev = np.sort(np.linalg.eigvals(J).real)
            if np.max(np.abs(ev - [un - c, un, un + c])) > 2e-6 * (abs(un) + c):
                bad = True
    caught.append(bad)
    # simple-wave convergence pin (Upwind5 at 16, 32: the exact scheme has
    # order 4.6 there and errors below 3e-5)
    e = [simple_wave_errors("up5", n, T=0.02) for n in (16, 32)]
    caught.append(any(math.log2(e[0][c] / e[1][c]) < 4.0 or e[1][c] > 1e-4 for c in range(3)))
    assert all(caught), (kind, caught)


def test_planted_source_sign_fails_the_jet(monkeypatch):
    orig = FA.rhs

    def rhs(Q, eqn, scheme, p):
        # the Coriolis source with the opposite sign: S = (0, -f hv, f hu)
        out = orig(Q, eqn, scheme, p)
        out[1] = out[1] - 2 * p["f"] * Q[2]
        out[2] = out[2] + 2 * p["f"] * Q[1]
        return out
    monkeypatch.setattr(FA, "rhs", rhs)
    r = [jet_residuals("up5", n) for n in (16, 32)]
    assert r[1] > 1e-2 and math.log2(r[0] / r[1]) < 1.0


@pytest.mark.parametrize("kind", ["velocity_not_divided", "no_g", "min_not_max"])
def test_planted_speed_mistakes_fail_the_eigenvalue_pin(monkeypatch, kind):
    def speed(Qm, Qp, direction, eqn, p):
        g = p["g"]
        k = 1 if direction == "x" else 2
        if kind == "velocity_not_divided":
            lm, lp = np.abs(Qm[k]) + np.sqrt(g * Qm[0]), np.abs(Qp[k]) + np.sqrt(g * Qp[0])
        elif kind == "no_g":
            lm, lp = np.abs(Qm[k] / Qm[0]) + np.sqrt(Qm[0]), np.abs(Qp[k] / Qp[0]) + np.sqrt(Qp[0])
        else:
            lm, lp = np.abs(Qm[k] / Qm[0]) + np.sqrt(g * Qm[0]), np.abs(Qp[k] / Qp[0]) + np.sqrt(g * Qp[0])
            return np.minimum(lm, lp)
        return np.maximum(lm, lp)
    monkeypatch.setattr(FA, "max_speed", speed)
    with pytest.raises(AssertionError):
        test_llf_speed_is_the_largest_jacobian_eigenvalue("x")


def test_exact_solutions_are_consistent():
    # the simple wave conserves mass and momentum exactly (periodic), and at
    # t = 0 reduces to the initial profile; the jet has zero divergence of
    # mass flux (hu = -hv)
    a0 = simple_wave_cellavg(32, 0.0)
    a1 = simple_wave_cellavg(32, 0.04)
    for c in range(3):
        assert abs(a1[c].sum() - a0[c].sum()) <= 1e-11 * np.abs(a0[c]).sum()
    n = 32
    xc = (np.arange(n) + 0.5) / n
    z = math.pi / n
    np.testing.assert_allclose(a0[0], 1.0 + 0.1 * np.sin(2 * np.pi * (xc[:, None] + xc[None, :])) *
                               (math.sin(z) / z) ** 2, atol=1e-13)
    j = geostrophic_jet_cellavg(n)
    np.testing.assert_array_equal(j[1], -j[2])
