"""The adaptive truncation tolerance of Sec. 4.4 on the GPU (eps_rule =
TT_EPS_ADAPTIVE): per-field eps_u = min(1e-3, C V^(1/2) dx^(p-1/2) / ||u||_F)
for a variable's own forward-Euler and SSP rounds (Eq.
modified-eps-tt-formula) and eps_TT over max_q ||q||_F for every other
rounding (Eq. eps-tt-formula), set at the start of each step.

* the step's tolerances and states equal Oracle B's under the same rule
  (tolerances to 1e-12 relative, ranks equal, fields within 30 x the step's
  largest tolerance -- 1e-10 at least -- of their scale S_c);
* the inertia-gravity wave of Sec. 5.2 (the closed form of synth.igw_cellavg,
  doubly periodic, Coriolis on) run through the GPU TT solver keeps the
  formal orders 3 / 5 / 5 of Upwind3 / Upwind5 / WENO5 with dt ~ dx
  (Upwind3) and dt ~ dx^(5/3) (fifth order, Sec. 5) and Table 1's C_eps for
  this case (1, 1, 500).
"""
import math

import numpy as np
import pytest

from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_scales
from synth import igw_cellavg, initial_tt, workload

pytestmark = pytest.mark.gpu

G, H, F = 9.81, 1.0, 1.0


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def igw_setup(scheme, n, T_end=0.02):
    p = dict(g=G, H=H, f=F, lx=1.0, ly=1.0)
    dx = 1.0 / n
    c = math.sqrt(G * H)
    dt0 = 0.4 * dx / c if scheme == "up3" else 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / c
    nst = int(math.ceil(T_end / dt0))
    p["dt"] = T_end / nst
    Q = [T.tt_svd(q, 1e-15, n) for q in igw_cellavg(n, 0.0, g=G, H=H, f=F)]
    return Q, p, nst


def make(api, Q, w, p):
    q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
    return api.Solver(q0, w["eqn"], w["scheme"], w["n"], p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"],
                      f=p["f"], seed=0, eps_rule="adaptive", c_eps=w["c_eps"])


@pytest.mark.parametrize("case", ["igw_up5", "bumps_up3"])
def test_adaptive_tolerances_and_states_match_oracle_b(api, case):
    if case == "igw_up5":
        n = 32
        Q, p, _ = igw_setup("up5", n)
        w = dict(eqn="linear", scheme="up5", n=n, tol=0.0, cap=24, eps_rule="adaptive", c_eps=1.0)
    else:
        w = workload("nonlinear256_weno5", n=32, scheme="up3", cap=24, eps_rule="adaptive", c_eps=1.0)
        Q, p = initial_tt(w)
    s = make(api, Q, w, p)
    Qb = Q
    for k in range(3):
        # the rule applied to the GPU's own state at the start of the step
        mine = Q if k == 0 else [(q.cores()[0].numpy(), q.cores()[1].numpy()) for q in s.get()]
        eps_tt, eps_u = TB.step_tolerances(mine, w, p)
        s.step(1)
        st = s.stats()
        assert abs(st["eps_tt"] - eps_tt) <= 1e-12 * eps_tt, (k, st["eps_tt"], eps_tt)
        for c in range(3):
            assert abs(st["eps_u"][c] - eps_u[c]) <= 1e-12 * eps_u[c], (k, c, st["eps_u"], eps_u)
        Qb = TB.step(Qb, w, p, seed=0)
        got = s.get()
        assert [g.rank for g in got] == [T.rank(q) for q in Qb], k
        # truncation decides at the step's own tolerances (momentum from rest
        # rounds at the 1e-3 clip in step 1), so the bar is 10 x the largest
        # of them per stage, never below the 1e-10 round-off bar
        bar = max(1e-10, 3 * 10 * max([eps_tt] + list(eps_u)))
        check_fields(got, Qb, bar, field_scales(Qb, w["eqn"], p, p["dt"]), what=(case, k))
    if case == "bumps_up3":
        # momentum starts at rest: its own tolerance is clipped at 1e-3 in step 1
        assert TB.step_tolerances(Q, w, p)[1][1] == 1e-3
    assert s.stats()["device_status"] == 0
    s.close()


@pytest.mark.parametrize("scheme,order,c_eps,sizes", [("up3", 3, 1.0, (16, 32, 64)),
                                                      ("up5", 5, 1.0, (16, 32, 64)),
                                                      ("weno5", 5, 500.0, (16, 32, 64))])
def test_igw_convergence_through_the_gpu_solver(api, scheme, order, c_eps, sizes):
    errs = []
    for n in sizes:
        Q, p, nst = igw_setup(scheme, n)
        w = dict(eqn="linear", scheme=scheme, n=n, tol=0.0, cap=min(n, 32), c_eps=c_eps)
        s = make(api, Q, w, p)
        s.step(nst)
        got = s.get()
        assert s.stats()["device_status"] == 0
        s.close()
        ex = igw_cellavg(n, nst * p["dt"], g=G, H=H, f=F)
        errs.append(float(np.linalg.norm(got[0].full().numpy() - ex[0]) / np.linalg.norm(ex[0])))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    print("igw", scheme, "errors", errs, "orders", orders)
    assert order - 0.4 < orders[-1] < order + 0.6, (scheme, errs, orders)
