"""GPU parity of the full TT finite-volume stage (tt_fv_init / tt_fv_stage /
tt_fv_step through the C ABI) against Oracle B (TT stage) and Oracle A
(full-tensor stage).

Tolerances, per field (tests/parity.py), each on the field's scale
S_c = ||u_c|| + 2 dt/dx ||F_c|| + 2 dt/dy ||G_c||, the size of the tensors
whose roundings reach it (for h its own norm; for momentum from rest the
pressure flux g h^2/2 dominates): with no rank cap binding and truncation
decided by tol, GPU and Oracle B run the same algorithm at the same ranks,
so each field agrees to a small multiple of the FP64 round-off of the
roundings (asserted 1e-10 of S_c for the upwind schemes, whose roundings
sit at clear spectral gaps); against Oracle A's exact full-tensor result,
and for WENO5 (cross pivots may differ), each field is within 10 x tol of
S_c per stage.
"""
import numpy as np
import pytest

from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_scales
from synth import initial_tt, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def make_solver(api, w, Q, p):
    q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
    return api.Solver(q0, w["eqn"], w["scheme"], w["n"], p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"],
                      f=p["f"], kick=w.get("kick", 4), max_sweeps=w.get("max_sweeps", 10), seed=0)


def test_linear_64_up3_matches_oracle_b_and_a(api):
    # the 64^2 linear Upwind3 workload (tol 1e-10, cap 8), 5 full steps
    w = workload("linear64_up3")
    Q, p = initial_tt(w)
    s = make_solver(api, w, Q, p)
    Qb = Q
    Qa = [T.full(q) for q in Q]
    for n in range(5):
        s.step(1)
        Qb = TB.step(Qb, w, p, seed=0)
        Qa = FA.ssprk3_step(Qa, "linear", "up3", p, p["dt"])
        got = s.get()
        assert [g.rank for g in got] == [T.rank(q) for q in Qb]
        check_fields(got, Qb, 1e-10, field_scales(Qb, "linear", p, p["dt"]), what=("oracle B", n))
        # eta starts as a bump, u = v = 0: every field has its own scale
        check_fields(got, Qa, 3 * 10 * w["tol"] * (n + 1), field_scales(Qa, "linear", p, p["dt"]),
                     what=("oracle A", n))
    st = s.stats()
    assert st["device_status"] == 0 and st["rounds"] > 0
    s.close()


@pytest.mark.parametrize("scheme,n", [("up3", 32), ("up5", 40)])
def test_nonlinear_upwind_stages_match_oracle_b(api, scheme, n):
    w = workload("nonlinear256_weno5", n=n, scheme=scheme, cap=40, tol=1e-8)
    Q, p = initial_tt(w)
    s = make_solver(api, w, Q, p)
    Qn, Qs = Q, Q
    for k in range(3):
        s.stage(k)
        out = TB.stage(Qn, Qs, k, w, p, seed=1000 * k)
        Qs = out
        got = s.get()
        check_fields(got, out, 1e-10, field_scales(out, "nonlinear", p, p["dt"]), what=(scheme, k))
    s.close()


def test_nonlinear_weno5_stage_matches_full_tensor(api):
    n = 32
    w = workload("nonlinear256_weno5", n=n, cap=32, tol=1e-8)
    Q, p = initial_tt(w)
    s = make_solver(api, w, Q, p)
    s.stage(0)
    got = s.get()
    full = FA.ssprk3_stage([T.full(q) for q in Q], [T.full(q) for q in Q], 0, "nonlinear", "weno5", p, p["dt"])
    S = field_scales(full, "nonlinear", p, p["dt"])
    check_fields(got, full, 10 * w["tol"], S, what="oracle A")
    ref = TB.stage(Q, Q, 0, w, p, seed=0)
    check_fields(got, ref, 10 * w["tol"], S, what="oracle B")
    s.close()


def test_weno5_256_step_at_bench_configuration_matches_full_tensor(api):
    # the 256^2 WENO5 workload itself (rank cap 32, tol 1e-8, the stage graph
    # on its 16 workers): one SSP-RK3 step against Oracle A's exact
    # full-tensor step, per field within the WENO5 bar per stage (10 tol of
    # the field's truncation scale) times the three stages
    w = workload("nonlinear256_weno5")
    Q, p = initial_tt(w)
    s = make_solver(api, w, Q, p)
    s.step(1)
    got = s.get()
    ref = FA.ssprk3_step([T.full(q) for q in Q], "nonlinear", "weno5", p, p["dt"])
    check_fields(got, ref, 3 * 10 * w["tol"], field_scales(ref, "nonlinear", p, p["dt"]))
    st = s.stats()
    assert st["device_status"] == 0 and st["qb_uncertified"] == 0
    s.close()


def test_checkpoint_resume_is_bit_exact(api):
    w = workload("nonlinear256_weno5", n=32, scheme="up3", cap=24)
    Q, p = initial_tt(w)
    s1 = make_solver(api, w, Q, p)
    s1.step(2)
    snap = s1.get()
    s1.step(1)
    a = s1.get()
    s2 = make_solver(api, w, Q, p)
    s2.set(snap)
    s2.step(1)
    b = s2.get()
    for c in range(3):
        assert a[c].rank == b[c].rank
        assert np.array_equal(a[c].full().numpy(), b[c].full().numpy())
    s1.close()
    s2.close()


@pytest.mark.parametrize("scheme,n", [("up5", 40), ("weno5", 32)])
def test_lf_cross_flux_stages_match_oracles(api, scheme, n):
    # the LF-cross form of the nonlinear flux (one cross of the whole LLF
    # flux vector per direction, Sec. 4.2): three stages against Oracle A's
    # exact stages and Oracle B's LF-cross stages, per field within the
    # cross bar (10 tol of S_c per stage)
    w = workload("nonlinear256_weno5", n=n, scheme=scheme, cap=32, tol=1e-8, flux="cross")
    Q, p = initial_tt(w)
    q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
    s = api.Solver(q0, "nonlinear", scheme, n, p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"], f=p["f"],
                   seed=0, flux="cross")
    Qn = Qs = Q
    Qa_n = [T.full(q) for q in Q]
    Qa_s = Qa_n
    for k in range(3):
        s.stage(k)
        Qs = TB.stage(Qn, Qs, k, w, p, seed=1000 * k)
        Qa_s = FA.ssprk3_stage(Qa_n, Qa_s, k, "nonlinear", scheme, p, p["dt"])
        got = s.get()
        S = field_scales(Qa_s, "nonlinear", p, p["dt"])
        check_fields(got, Qa_s, 10 * w["tol"] * (k + 1), S, what=("A", scheme, k))
        check_fields(got, Qs, 10 * w["tol"] * (k + 1), S, what=("B", scheme, k))
    st = s.stats()
    assert st["device_status"] == 0 and st["taylor_iters"] == 0 and st["cross_calls"] > 0
    s.close()
