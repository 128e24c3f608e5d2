"""GPU parity of the precision forms (tt_fv_params.precision = TT_FP32,
TT_TF32, TT_BF16): every rounding contraction (Hadamard formation,
range-finder products, TSQR and its applications) runs in FP32 -- the large
products of the range finder on tcgen05 tensor cores for TF32/BF16, with
operands split into parts that reach FP32 accuracy -- while the small SVDs
and all cores stay FP64.

Bar.  FP32 round-off of a formed face tensor or residual is a few units of
2^-24 = 6e-8 relative to its norm, so the form never truncates below
tol_eff = max(tol, 1e-6) (below that it would keep round-off directions).
It is compared with Oracle B run at the same tol_eff: the truncation decides
the ranks, so each field must agree within 10 x tol_eff of its truncation
scale (tests/parity.py; the bar used for truncation-decided results), and
with Oracle A's exact full-tensor stage within the same bar.
"""
import numpy as np
import pytest

from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_scales
from synth import initial_tt, workload

pytestmark = pytest.mark.gpu

TOL_EFF_FP32 = 1e-6


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def make_solver(api, w, Q, p, precision):
    q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
    return api.Solver(q0, w["eqn"], w["scheme"], w["n"], p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"],
                      f=p["f"], seed=0, precision=precision)


def check(got, ref_full, p, what):
    """Per-field bar 10 tol_eff on each field's truncation scale."""
    return check_fields(got, ref_full, 10 * TOL_EFF_FP32, field_scales(ref_full, "nonlinear", p, p["dt"]), what)


def smooth_state(n, r):
    """A smooth periodic state of TT rank about r in every field (h > 0),
    so that Hadamard products of the faces exceed 112 columns."""
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="ij")
    F = [np.exp(0.6 * np.sin(2 * np.pi * (X + Y) + ph) + 0.3 * np.cos(2 * np.pi * (X - 2 * Y) + ph))
         for ph in (0.3, 1.1, 2.0)]
    h = 1.0 + 0.05 * F[0]
    return [T.tt_svd(h, 1e-14, r), T.tt_svd(0.02 * F[1], 1e-14, r), T.tt_svd(0.02 * F[2], 1e-14, r)]


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("scheme,n,state", [("up5", 128, "smooth"), ("up5", 128, "vortex"),
                                            ("up3", 40, "bumps")])
def test_precision_form_stages_match_oracles(api, scheme, n, state, precision):
    # "smooth" (ranks ~14) at 128^2: Hadamard products reach R > 112 and take
    # the range-finder route; the vortex and the bumps stay on the factored
    # and direct routes
    base = "vortex1024_up5" if state == "vortex" else "nonlinear256_weno5"
    w = workload(base, n=n, scheme=scheme, tol=1e-8, cap=48)
    Q, p = initial_tt(w)
    if state == "smooth":
        Q = smooth_state(n, 14)
    s = make_solver(api, w, Q, p, precision)
    wb = dict(w, tol=max(w["tol"], TOL_EFF_FP32))
    Qn, Qs = Q, Q
    Qa_n = [T.full(q) for q in Q]
    Qa_s = Qa_n
    for k in range(3):
        s.stage(k)
        Qs = TB.stage(Qn, Qs, k, wb, p, seed=1000 * k)
        Qa_s = FA.ssprk3_stage(Qa_n, Qa_s, k, w["eqn"], scheme, p, p["dt"])
        got = s.get()
        check(got, [T.full(q) for q in Qs], p, ("oracle B", scheme, k))
        check(got, Qa_s, p, ("oracle A", scheme, k))
        # no rank inflation from FP32 round-off
        assert all(g.rank <= T.rank(q) + 2 for g, q in zip(got, Qs)), ([g.rank for g in got],
                                                                     [T.rank(q) for q in Qs])
    st = s.stats()
    assert st["device_status"] == 0
    s.close()


def test_fp32_form_step_close_to_fp64_path(api):
    # one full SSP-RK3 step of the 128^2 vortex: the FP32 form and the FP64
    # path at the same tol_eff agree within the truncation bar
    w = workload("vortex1024_up5", n=128, tol=TOL_EFF_FP32, cap=48)
    Q, p = initial_tt(w)
    s32 = make_solver(api, w, Q, p, "fp32")
    s64 = make_solver(api, w, Q, p, "fp64")
    s32.step(1)
    s64.step(1)
    a, b = s32.get(), s64.get()
    ref = [q.full().numpy() for q in b]
    check(a, ref, p, "fp64 path")
    s32.close()
    s64.close()


_ref_cache = {}


def _smooth1024_refs():
    """Oracle B's first stage at tol_eff and Oracle A's exact first stage of
    the rank-14 smooth state at 1024^2 (computed once)."""
    if not _ref_cache:
        n = 1024
        w = workload("vortex1024_up5", tol=1e-8, cap=48)
        Q = smooth_state(n, 14)
        _, p = initial_tt(w)
        wb = dict(w, tol=TOL_EFF_FP32)
        full = [T.full(q) for q in Q]
        _ref_cache.update(Q=Q, p=p, w=w, b=TB.stage(Q, Q, 0, wb, p, seed=0),
                          a=FA.ssprk3_stage(full, full, 0, "nonlinear", "up5", p, p["dt"]))
    return _ref_cache


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_precision_forms_round_products_through_the_cores_at_1024(api, precision):
    # faces of rank ~14 on 1024 x 3072: their Hadamard products (R ~ 200
    # columns) are rounded by the range finder through the Khatri-Rao cores,
    # whose Grams, sketch and projections run on the tensor cores under
    # TF32 / BF16 (FP32 on CUDA cores for the FP32 form)
    r = _smooth1024_refs()
    s = make_solver(api, r["w"], r["Q"], r["p"], precision)
    s.stage(0)
    got = s.get()
    check(got, [T.full(q) for q in r["b"]], r["p"], ("oracle B", precision))
    errs = check(got, r["a"], r["p"], ("oracle A", precision))
    print("smooth1024", precision, "per-field rel L2 vs A", errs)
    st = s.stats()
    assert st["device_status"] == 0 and st["qb_attempts"] > 0
    s.close()
