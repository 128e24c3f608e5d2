"""The manufactured solution of the nonlinear SWE (Sec. 5.4): the forcing
derived symbolically in synth/mms.py makes Oracle A converge to the
manufactured fields at the formal orders 3 / 5 / 5 (without it the scheme
does not converge to them at all), and Oracle B's TT step with the same
forcing stays within the truncation bar of Oracle A's."""
import math

import numpy as np
import pytest

from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_scales

pytest.importorskip("sympy")
from synth import mms  # noqa: E402

W = mms.forcing_waves()
E = mms.exact_waves()
P = dict(g=mms.MMS_DEFAULT["g"], H=mms.MMS_DEFAULT["H"], f=mms.MMS_DEFAULT["f"], lx=1.0, ly=1.0)


def setup(scheme, n, T_end):
    dx = 1.0 / n
    smax = 0.15 + math.sqrt(P["g"] * 1.1)
    dt0 = 0.4 * dx / smax if scheme == "up3" else 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / smax
    nst = int(math.ceil(T_end / dt0))
    return nst, T_end / nst


def oracle_a_errors(scheme, n, T_end=0.02, forcing=True):
    nst, dt = setup(scheme, n, T_end)
    src = (lambda t: [mms.waves_cellavg(W, c, n, t) for c in range(3)]) if forcing else None
    Q = [mms.waves_cellavg(E, c, n, 0.0) for c in range(3)]
    t = 0.0
    for _ in range(nst):
        Q = FA.ssprk3_step(Q, "nonlinear", scheme, P, dt, source=src, t=t)
        t += dt
    ex = [mms.waves_cellavg(E, c, n, nst * dt) for c in range(3)]
    return [np.linalg.norm(Q[c] - ex[c]) / np.linalg.norm(ex[c]) for c in range(2)]


@pytest.mark.parametrize("scheme,order,lo", [("up3", 3, 2.7), ("up5", 5, 4.6), ("weno5", 5, 4.6)])
def test_forced_oracle_a_converges_to_the_manufactured_solution(scheme, order, lo):
    e = [oracle_a_errors(scheme, n) for n in (16, 32, 64)]
    for c in range(2):
        o = math.log2(e[1][c] / e[2][c])
        assert lo < o < order + 0.5, (scheme, c, e, o)


def test_without_the_forcing_there_is_no_convergence():
    e = [oracle_a_errors("up5", n, forcing=False) for n in (16, 32)]
    assert e[1][1] > 0.1 and abs(math.log2(e[0][1] / e[1][1])) < 0.5


def test_forcing_is_the_pde_residual_of_the_exact_fields():
    # independent of the symbolic algebra: dQ/dt by central differences in t
    # plus dF/dx + dG/dy by spectral derivatives on a fine grid, minus the
    # Coriolis source, equals the forcing waves (point values)
    n = 64
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x, indexing="ij")

    def fields(t):
        out = [np.zeros((n, n)) for _ in range(3)]
        for c, amp, kx, ky, om, ph in E:
            out[c] += amp * np.cos(kx * X + ky * Y - om * t + ph)
        return out
    k = 2 * np.pi * np.fft.fftfreq(n, d=1.0 / n)

    def d(fun, axis):
        kk = k.reshape((-1, 1) if axis == 0 else (1, -1))
        return np.real(np.fft.ifft(1j * kk * np.fft.fft(fun, axis=axis), axis=axis))
    t0, h = 0.013, 1e-5
    Qp, Qm, Q = fields(t0 + h), fields(t0 - h), fields(t0)
    hh, hu, hv = Q
    g, f = P["g"], P["f"]
    F = [hu, hu * hu / hh + 0.5 * g * hh * hh, hu * hv / hh]
    G = [hv, hu * hv / hh, hv * hv / hh + 0.5 * g * hh * hh]
    S = [0 * hh, f * hv, -f * hu]
    for c in range(3):
        res = (Qp[c] - Qm[c]) / (2 * h) + d(F[c], 0) + d(G[c], 1) - S[c]
        want = np.zeros((n, n))
        for cc, amp, kx, ky, om, ph in W:
            if cc == c:
                want += amp * np.cos(kx * X + ky * Y - om * t0 + ph)
        assert np.max(np.abs(res - want)) < 1e-6 * max(1.0, np.max(np.abs(want))), c


@pytest.mark.parametrize("scheme", ["up5", "weno5"])
def test_forced_tt_step_matches_full_tensor(scheme):
    n = 32
    nst, dt = setup(scheme, n, 0.02)
    p = dict(P, dt=dt)
    w = dict(eqn="nonlinear", scheme=scheme, n=n, tol=1e-8, cap=24, forcing=W)
    Q = [T.tt_svd(mms.waves_cellavg(E, c, n, 0.0), 1e-15, n) if c < 2 else (np.zeros((n, 1)), np.zeros((n, 1)))
         for c in range(3)]
    t = 0.05
    out = TB.step(Q, w, p, seed=0, t=t)
    src = lambda tt: [mms.waves_cellavg(W, c, n, tt) for c in range(3)]  # noqa: E731
    ref = FA.ssprk3_step([T.full(q) for q in Q], "nonlinear", scheme, p, dt, source=src, t=t)
    check_fields(out, ref, 3 * 10 * w["tol"], field_scales(ref, "nonlinear", p, dt))
