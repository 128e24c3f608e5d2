"""GPU parity at the sizes the workloads state: the 1024^2 geostrophic vortex
(Upwind5) in FP64 and in each precision form, one SSP-RK3 step of the
4096^2 WENO5 case, and one step of the 256-instance ensemble.

Oracle A runs in its C form (oracle/fv_full.c, pinned to the numpy form)
except on the 4096^2 patches.  Bars, per field on the field's scale S_c (tests/parity.py): 30 x tol per
step (10 x tol per stage, three stages) against Oracle A's exact
full-tensor result, and against Oracle B where truncation decides the ranks;
1e-10 of S_c against Oracle B at equal ranks.  The precision forms truncate
at tol_eff = 1e-6 and are held to 30 x tol_eff per step against Oracle B
run at tol_eff and against Oracle A.

At 4096^2 the full-tensor oracle is sampled: Oracle A's exact step on
seeded patches with a 12-cell halo (one step reads 9 cells on either side,
so the periodically wrapped patch is exact in its interior; pinned by
tests/test_bench_helpers.py).
"""
import functools

import numpy as np
import pytest

import bench
from oracle import fv_c as FC
from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_errors, field_scales
from synth import ensemble, initial_tt, workload

pytestmark = pytest.mark.gpu

TOL_EFF = 1e-6
VORTEX_STEPS = 2


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def solver(api, w, Q, p, precision="fp64"):
    q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
    return api.Solver(q0, w["eqn"], w["scheme"], w["n"], p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"],
                      f=p["f"], seed=0, precision=precision)


@functools.lru_cache(maxsize=None)
def vortex_oracle_a():
    """Oracle A's exact states after 1..VORTEX_STEPS steps of the 1024^2 vortex."""
    w = workload("vortex1024_up5")
    Q, p = initial_tt(w)
    out, Qa = [], [T.full(q) for q in Q]
    for _ in range(VORTEX_STEPS):
        Qa = FC.ssprk3_steps(Qa, w["eqn"], w["scheme"], p, p["dt"], 1)
        out.append(Qa)
    return out


@functools.lru_cache(maxsize=None)
def vortex_oracle_b(tol):
    w = workload("vortex1024_up5", tol=tol)
    Q, p = initial_tt(w)
    out, Qb = [], Q
    for _ in range(VORTEX_STEPS):
        Qb = TB.step(Qb, w, p, seed=0)
        out.append(Qb)
    return out


def test_vortex1024_fp64_matches_oracles(api):
    w = workload("vortex1024_up5")
    Q, p = initial_tt(w)
    s = solver(api, w, Q, p)
    for k in range(VORTEX_STEPS):
        s.step(1)
        got = s.get()
        qb = vortex_oracle_b(w["tol"])[k]
        qa = vortex_oracle_a()[k]
        if [g.rank for g in got] == [T.rank(q) for q in qb]:
            check_fields(got, qb, 1e-10, field_scales(qb, "nonlinear", p, p["dt"]), what=("B equal ranks", k))
        else:
            check_fields(got, qb, 30 * w["tol"] * (k + 1), field_scales(qb, "nonlinear", p, p["dt"]),
                         what=("B", k))
        errs = check_fields(got, qa, 30 * w["tol"] * (k + 1), field_scales(qa, "nonlinear", p, p["dt"]),
                            what=("A", k))
        print("vortex1024 fp64 step", k + 1, "per-field rel L2 vs A", errs)
    assert s.stats()["device_status"] == 0
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_vortex1024_precision_forms_match_oracles(api, precision):
    w = workload("vortex1024_up5")
    Q, p = initial_tt(w)
    s = solver(api, w, Q, p, precision)
    for k in range(VORTEX_STEPS):
        s.step(1)
        got = s.get()
        qb = vortex_oracle_b(TOL_EFF)[k]
        qa = vortex_oracle_a()[k]
        check_fields(got, qb, 30 * TOL_EFF * (k + 1), field_scales(qb, "nonlinear", p, p["dt"]), what=("B", k))
        errs = check_fields(got, qa, 30 * TOL_EFF * (k + 1), field_scales(qa, "nonlinear", p, p["dt"]),
                            what=("A", k))
        print("vortex1024", precision, "step", k + 1, "per-field rel L2 vs A", errs)
    assert s.stats()["device_status"] == 0
    s.close()


def patch_arrays(start, after, w, p, npatch=12, size=48, halo=12, seed=11):
    """(got, ref) per field: the patch interiors of `after` and of Oracle A's
    exact step from `start`, side by side."""
    rng = np.random.default_rng(seed)
    n = w["n"]
    m = size + 2 * halo
    pp = dict(p, lx=m / n, ly=m / n)
    got = [[], [], []]
    ref = [[], [], []]
    for _ in range(npatch):
        i0, j0 = (int(v) for v in rng.integers(0, n, size=2))
        rows = (i0 - halo + np.arange(m)) % n
        cols = (j0 - halo + np.arange(m)) % n
        P = [A[rows] @ B[cols].T for A, B in start]
        R = FA.ssprk3_step(P, w["eqn"], w["scheme"], pp, p["dt"])
        for c in range(3):
            A, B = after[c]
            got[c].append(A[rows[halo:-halo]] @ B[cols[halo:-halo]].T)
            ref[c].append(R[c][halo:-halo, halo:-halo])
    return [np.hstack(g) for g in got], [np.hstack(r) for r in ref]


def test_weno5_4096_step_matches_oracle_a_on_patches(api):
    # the 4096^2 WENO5 workload (rank cap 64, tol 1e-8): steps 1 and 3 (the
    # second from the GPU's own state after step 2) against Oracle A's exact
    # step, sampled on patches; the patches include the bumps' flanks
    w = workload("nonlinear4096_weno5")
    Q, p = initial_tt(w)
    s = solver(api, w, Q, p)
    n = w["n"]
    start = Q
    for k in range(3):
        s.step(1)
        got = s.get()
        after = [bench.host_tt(q) for q in got]
        if k in (0, 2):
            g, r = patch_arrays(start, after, w, p, seed=11 + k)
            S = field_scales(r, "nonlinear", p, p["dt"], d=(1.0 / n, 1.0 / n))
            errs = check_fields(g, r, 30 * w["tol"], S, what=("4096 step", k + 1))
            print("weno5 4096 step", k + 1, "per-field rel L2 vs A (patches)", errs)
        start = after
    st = s.stats()
    assert st["device_status"] == 0
    s.close()


def test_ensemble256_step_matches_oracles_on_sampled_instances(api):
    # all 256 instances (grids 128^2-1024^2, caps 8-64, up3/up5/weno5 in
    # thirds) advanced one step together in the batched form; a seeded sample
    # of 4 instances per scheme is compared with the oracles
    ws = ensemble(256)
    insts = []
    for w in ws:
        Q, p = initial_tt(w)
        q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
        insts.append((q0, dict(eqn=w["eqn"], scheme=w["scheme"], n=w["n"], dt=p["dt"], tol=w["tol"],
                               rank_cap=w["cap"], g=p["g"], H=p["H"], f=p["f"], seed=0)))
    b = api.Batch(insts, precision="fp64", workers=16)
    b.step(1)
    rng = np.random.default_rng(4)
    for scheme in ("up3", "up5", "weno5"):
        idx = [i for i, w in enumerate(ws) if w["scheme"] == scheme]
        for i in rng.choice(idx, size=4, replace=False):
            w = ws[i]
            Q, p = initial_tt(w)
            got = b.get(int(i))
            assert b.stats(int(i))["device_status"] == 0
            qa = FC.ssprk3_steps([T.full(q) for q in Q], "nonlinear", scheme, p, p["dt"], 1)
            S = field_scales(qa, "nonlinear", p, p["dt"])
            check_fields(got, qa, 30 * w["tol"], S, what=("ensemble A", int(i), scheme, w["n"], w["cap"]))
            if scheme != "weno5":
                qb = TB.step(Q, w, p, seed=0)
                if [g.rank for g in got] == [T.rank(q) for q in qb]:
                    check_fields(got, qb, 1e-10, field_scales(qb, "nonlinear", p, p["dt"]),
                                 what=("ensemble B", int(i)))
            print("ensemble instance", int(i), scheme, w["n"], "cap", w["cap"], "rel L2 vs A",
                  field_errors(got, qa))
    b.close()


@pytest.mark.slow
def test_weno5_256_all_500_steps_match_oracle_a(api):
    # the 256^2 WENO5 workload over its full 500 steps, against the C form of
    # Oracle A advanced the same 500 steps without truncation; the bar grows
    # linearly with the steps (30 tol of S_c per step); per-field errors are
    # reported every 100 steps
    w = workload("nonlinear256_weno5")
    Q, p = initial_tt(w)
    s = solver(api, w, Q, p)
    Qa = [T.full(q) for q in Q]
    done = 0
    for k in (100, 200, 300, 400, 500):
        s.step(k - done)
        Qa = FC.ssprk3_steps(Qa, "nonlinear", "weno5", p, p["dt"], k - done)
        done = k
        got = s.get()
        errs = check_fields(got, Qa, 30 * w["tol"] * k, field_scales(Qa, "nonlinear", p, p["dt"]), what=k)
        print("weno5 256 after", k, "steps: ranks", [g.rank for g in got], "per-field rel L2 vs A", errs)
    st = s.stats()
    assert st["device_status"] == 0
    s.close()
