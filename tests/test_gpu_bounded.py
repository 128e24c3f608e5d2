"""The linear SWE on a domain bounded in x with exact-solution boundary cells
(bc_x = TT_BC_EXACT; Sec. 5.3's barotropic tide and Sec. 5.1's coastal Kelvin
wave, damped in x), through the C ABI:

* three steps from a state of TT rank > 1 (the tide plus a y-dependent
  perturbation) against Oracle B's bounded TT step (tol 1e-12, equal ranks:
  1e-10 of each field's scale S_c) and Oracle A's full-tensor step with ghost
  cells (30 tol per step of S_c);
* the tide converges at the formal orders 3 / 5 (Upwind3 / Upwind5) in every
  field, dt ~ dx (Upwind3) and dt ~ dx^(5/3) (Upwind5), and so does the
  Kelvin wave in eta and v (the same three-step parity against Oracles B and A);
* a bounded solver refuses to step before its boundary is set, and WENO5 or
  the nonlinear SWE with a bounded x are refused at init.
"""
import math

import numpy as np
import pytest

from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_scales
from synth import kelvin, tide, waves

pytestmark = pytest.mark.gpu

W = tide.tide_waves()
P = tide.tide_params()
NW = max(sum(w[0] == c for w in W) for c in range(3))


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def ghost_cells(n, t):
    g = FA.GHOST
    return ([waves.waves_cellavg(W, c, n, t, rows=np.arange(-g, 0)) for c in range(3)],
            [waves.waves_cellavg(W, c, n, t, rows=np.arange(n, n + g)) for c in range(3)])


def solver(api, Q, scheme, n, dt, tol, cap, t0=0.0):
    q0 = [api.DevTT.from_cores(A, B, cap=cap) for A, B in Q]
    s = api.Solver(q0, "linear", scheme, n, dt, tol, cap, g=P["g"], H=P["H"], f=P["f"], bc_x="exact",
                   boundary_waves=NW)
    s.set_boundary(W, t0=t0)
    return s


def rich_state(n):
    x = (np.arange(n) + 0.5) / n
    bump = np.exp(-((x[:, None] - 0.4) ** 2) / 0.02) * np.cos(2 * np.pi * x[None, :])
    base = [waves.waves_cellavg(W, k, n, 0.0) for k in range(3)]
    return [base[0] + 0.005 * bump, base[1] + 0.002 * bump.T + 0.001 * bump, base[2] - 0.001 * bump]


@pytest.mark.parametrize("scheme", ["up3", "up5"])
def test_bounded_steps_match_oracles(api, scheme):
    n, tol, cap = 32, 1e-12, 32
    dt = 0.2 / n / math.sqrt(P["g"])
    p = dict(P, dt=dt)
    full = rich_state(n)
    Q = [T.tt_svd(f, 1e-15, n) for f in full]
    w = dict(eqn="linear", scheme=scheme, n=n, tol=tol, cap=cap, bc_x="exact", boundary=W)
    s = solver(api, Q, scheme, n, dt, tol, cap)
    Qb, Qa, t = Q, full, 0.0
    for k in range(3):
        s.step(1)
        Qb = TB.step(Qb, w, p, seed=0, t=t)
        Qa = FA.ssprk3_step(Qa, "linear", scheme, p, dt, t=t, bc=lambda tt: ghost_cells(n, tt))
        t += dt
        got = s.get()
        assert [g.rank for g in got] == [T.rank(q) for q in Qb], k
        check_fields(got, Qb, 1e-10, field_scales(Qb, "linear", p, dt), what=("B", scheme, k))
        errs = check_fields(got, Qa, 30 * tol * (k + 1) + 1e-12, field_scales(Qa, "linear", p, dt),
                            what=("A", scheme, k))
        print("bounded", scheme, "step", k + 1, "ranks", [g.rank for g in got], "rel L2 vs A", errs)
    assert s.stats()["device_status"] == 0
    s.close()


@pytest.mark.parametrize("scheme,order", [("up3", 3), ("up5", 5)])
def test_tide_converges_through_the_gpu(api, scheme, order):
    errs = []
    for n in (16, 32, 64):
        dx = 1.0 / n
        c = math.sqrt(P["g"] * P["H"])
        dt0 = 0.4 * dx / c if scheme == "up3" else 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / c
        T_end = 0.05
        nst = int(math.ceil(T_end / dt0))
        dt = T_end / nst
        Q = [T.tt_svd(waves.waves_cellavg(W, k, n, 0.0), 1e-15, n) if k != 1 else (np.zeros((n, 1)), np.zeros((n, 1)))
             for k in range(3)]
        s = solver(api, Q, scheme, n, dt, 1e-12, 16)
        s.step(nst)
        got = s.get()
        assert s.stats()["device_status"] == 0
        s.close()
        ex = [waves.waves_cellavg(W, k, n, nst * dt) for k in range(3)]
        errs.append([float(np.linalg.norm(got[k].full().numpy() - ex[k]) / np.linalg.norm(ex[k])) for k in range(3)])
    print("tide", scheme, errs)
    for k in range(3):
        o = math.log2(errs[1][k] / errs[2][k])
        assert order - 0.3 < o < order + 0.5, (scheme, k, errs, o)


def test_bounded_solver_argument_checks(api):
    from paper_2408_03483_gb300 import capi
    n = 16
    Q = [T.tt_svd(waves.waves_cellavg(W, k, n, 0.0), 1e-15, n) if k != 1 else (np.zeros((n, 1)), np.zeros((n, 1)))
         for k in range(3)]
    q0 = [api.DevTT.from_cores(A, B, cap=8) for A, B in Q]
    s = api.Solver(q0, "linear", "up5", n, 1e-3, 1e-10, 8, f=P["f"], bc_x="exact", boundary_waves=NW)
    with pytest.raises(capi.TTError):
        s.step(1)  # no boundary set yet
    with pytest.raises(capi.TTError):
        s.set_boundary(W + W)  # more waves per field than boundary_waves
    s.set_boundary(W)
    s.step(1)
    s.close()
    for eqn, scheme in (("linear", "weno5"), ("nonlinear", "up5")):
        with pytest.raises(capi.TTError):
            api.Solver(q0, eqn, scheme, n, 1e-3, 1e-10, 8, bc_x="exact", boundary_waves=NW)


# ---------------------------------------------------------------- Kelvin wave
# Sec. 5.1's coastal Kelvin wave: damped in x (exp(-x/R), five decay lengths
# across the domain), travelling along the coast at x = 0 in y; its ghost
# cells are the damped waves' exact cell averages.
KW = kelvin.kelvin_waves()
KP = kelvin.kelvin_params()
KNW = max(sum(w[0] == c for w in KW) for c in range(3))


def kelvin_state(n, t=0.0):
    out = []
    for k in range(3):
        f = waves.waves_cellavg(KW, k, n, t)
        out.append(T.tt_svd(f, 1e-15, n) if np.linalg.norm(f) > 0 else (np.zeros((n, 1)), np.zeros((n, 1))))
    return out


def kelvin_solver(api, Q, scheme, n, dt, tol, cap, t0=0.0):
    q0 = [api.DevTT.from_cores(A, B, cap=cap) for A, B in Q]
    s = api.Solver(q0, "linear", scheme, n, dt, tol, cap, g=KP["g"], H=KP["H"], f=KP["f"], bc_x="exact",
                   boundary_waves=KNW)
    s.set_boundary(KW, t0=t0)
    return s


@pytest.mark.parametrize("scheme", ["up3", "up5"])
def test_kelvin_steps_match_oracles(api, scheme):
    n, tol, cap = 32, 1e-12, 32
    dt = 0.2 / n / math.sqrt(KP["g"])
    p = dict(KP, dt=dt)
    Q = kelvin_state(n)
    full = [T.full(q) for q in Q]
    w = dict(eqn="linear", scheme=scheme, n=n, tol=tol, cap=cap, bc_x="exact", boundary=KW)
    s = kelvin_solver(api, Q, scheme, n, dt, tol, cap)
    g0 = FA.GHOST
    ghost = lambda tt: ([waves.waves_cellavg(KW, c, n, tt, rows=np.arange(-g0, 0)) for c in range(3)],  # noqa: E731
                        [waves.waves_cellavg(KW, c, n, tt, rows=np.arange(n, n + g0)) for c in range(3)])
    Qb, Qa, t = Q, full, 0.0
    for k in range(3):
        s.step(1)
        Qb = TB.step(Qb, w, p, seed=0, t=t)
        Qa = FA.ssprk3_step(Qa, "linear", scheme, p, dt, t=t, bc=ghost)
        t += dt
        got = s.get()
        assert [g.rank for g in got] == [T.rank(q) for q in Qb], k
        check_fields(got, Qb, 1e-10, field_scales(Qb, "linear", p, dt), what=("B", scheme, k))
        errs = check_fields(got, Qa, 30 * tol * (k + 1) + 1e-12, field_scales(Qa, "linear", p, dt),
                            what=("A", scheme, k))
        print("kelvin", scheme, "step", k + 1, "ranks", [g.rank for g in got], "rel L2 vs A", errs)
    assert s.stats()["device_status"] == 0
    s.close()


@pytest.mark.parametrize("scheme,order", [("up3", 3), ("up5", 5)])
def test_kelvin_wave_converges_through_the_gpu(api, scheme, order):
    errs = []
    c = math.sqrt(KP["g"] * KP["H"])
    for n in (16, 32, 64):
        dx = 1.0 / n
        dt0 = 0.4 * dx / c if scheme == "up3" else 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / c
        T_end = 0.05
        nst = int(math.ceil(T_end / dt0))
        dt = T_end / nst
        s = kelvin_solver(api, kelvin_state(n), scheme, n, dt, 1e-12, 16)
        s.step(nst)
        got = s.get()
        assert s.stats()["device_status"] == 0
        s.close()
        ex = [waves.waves_cellavg(KW, k, n, nst * dt) for k in range(3)]
        errs.append([float(np.linalg.norm(got[k].full().numpy() - ex[k]) / np.linalg.norm(ex[k])) for k in (0, 2)])
    print("kelvin", scheme, errs)
    for k in range(2):
        o = math.log2(errs[1][k] / errs[2][k])
        assert order - 0.3 < o < order + 0.7, (scheme, k, errs, o)
