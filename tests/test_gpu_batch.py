"""GPU parity of the batched form (tt_fv_batch_*): an ensemble of instances
with uneven grid sizes, rank caps and reconstructions advanced together.

Every instance runs the same kernels as a single solver on its own stream,
and every kernel is deterministic, so each instance must match a solver
advanced alone bit for bit, whatever the worker count; against the oracle
the single-solver bars apply per field on the field's scale S_c of
tests/parity.py (upwind at 1e-10 of S_c against Oracle B at equal ranks,
WENO5 by cross within 10 x tol of S_c per stage against Oracle A's exact
result, so 30 x tol after the three stages of a step; their caps equal n,
so only the tolerance truncates).
"""
import numpy as np
import pytest

from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from parity import check_fields, field_scales
from synth import initial_tt

pytestmark = pytest.mark.gpu

CASES = [("up3", 32, 12, 1), ("up5", 40, 16, 2), ("weno5", 32, 32, 3), ("up3", 48, 8, 1), ("up5", 64, 20, 2),
         ("weno5", 40, 40, 1)]


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def instances(api):
    out = []
    for k, (scheme, n, cap, nb) in enumerate(CASES):
        w = dict(eqn="nonlinear", scheme=scheme, n=n, steps=1, tol=1e-8, cap=cap, ic="bumps", amp=0.1,
                 amp_range=(0.01, 0.1), nbumps=nb, seed=500 + k, cfl=0.4, f=0.0)
        Q, p = initial_tt(w)
        d = dict(eqn="nonlinear", scheme=scheme, n=n, dt=p["dt"], tol=w["tol"], rank_cap=cap, g=p["g"],
                 H=p["H"], f=p["f"], seed=0)
        out.append((w, Q, p, d))
    return out


def dev(api, Q, cap):
    return [api.DevTT.from_cores(A, B, cap=cap) for A, B in Q]


@pytest.mark.parametrize("workers,inner", [(3, False), (6, True)])
def test_batch_matches_single_solvers_bitwise(api, workers, inner):
    inst = instances(api)
    b = api.Batch([(dev(api, Q, d["rank_cap"]), d) for w, Q, p, d in inst], workers=workers, inner_tasks=inner)
    b.step(2)
    for i, (w, Q, p, d) in enumerate(inst):
        s = api.Solver(dev(api, Q, d["rank_cap"]), "nonlinear", d["scheme"], d["n"], d["dt"], d["tol"],
                       d["rank_cap"], g=d["g"], H=d["H"], f=d["f"], seed=0)
        s.step(2)
        a, c = b.get(i), s.get()
        for qa, qc in zip(a, c):
            assert qa.rank == qc.rank
            assert np.array_equal(qa.full().numpy(), qc.full().numpy()), (i, d["scheme"])
        assert b.stats(i)["device_status"] == 0
        s.close()
    b.close()


def test_batch_one_step_matches_oracles(api):
    inst = instances(api)
    b = api.Batch([(dev(api, Q, d["rank_cap"]), d) for w, Q, p, d in inst], workers=4)
    b.step(1)
    for i, (w, Q, p, d) in enumerate(inst):
        got = b.get(i)
        if d["scheme"] == "weno5":
            ref = FA.ssprk3_step([T.full(q) for q in Q], "nonlinear", "weno5", p, p["dt"])
            check_fields(got, ref, 3 * 10 * w["tol"], field_scales(ref, "nonlinear", p, p["dt"]), i)
        else:
            ref = TB.step(Q, w, p, seed=0)
            check_fields(got, ref, 1e-10, field_scales(ref, "nonlinear", p, p["dt"]), what=i)
    b.close()


def test_batch_tune_picks_a_candidate(api):
    inst = instances(api)
    b = api.Batch([(dev(api, Q, d["rank_cap"]), d) for w, Q, p, d in inst], workers=1)
    w, inner = b.tune(workers=(2, 6), steps_per_trial=1)
    assert w in (2, 6) and inner in (False, True)
    b.step(1)
    for i, (_, _, _, d) in enumerate(inst):
        st = b.stats(i)
        assert st["device_status"] == 0 and max(st["rank"]) <= d["rank_cap"]
    b.close()


def test_every_tile_shape_matches_oracle_b(api):
    """Each TSQR tile shape (leaf rows, merge fan-in) only reorders the
    rounding's round-off: an Upwind5 step at 256^2 (faces 256 x 768, so the
    cores' TSQR trees have several leaves and merge levels) matches Oracle B
    at equal ranks under every shape."""
    shapes = api.tile_shapes()
    assert shapes[0] == (2, 0)
    w = dict(eqn="nonlinear", scheme="up5", n=256, steps=1, tol=1e-8, cap=24, ic="bumps", amp=0.1,
             amp_range=(0.01, 0.1), nbumps=3, seed=77, cfl=0.4, f=0.0)
    Q, p = initial_tt(w)
    ref = TB.step(Q, w, p, seed=0)
    scales = field_scales(ref, "nonlinear", p, p["dt"])
    for k in range(len(shapes)):
        s = api.Solver(dev(api, Q, w["cap"]), "nonlinear", "up5", 256, p["dt"], w["tol"], w["cap"], g=p["g"],
                       H=p["H"], f=p["f"], seed=0)
        s.set_tile_shape(k)
        s.step(1)
        check_fields(s.get(), ref, 1e-10, scales, what=("shape", k, shapes[k]))
        s.close()


def test_batch_tile_tuner_gives_each_member_a_shape(api):
    inst = instances(api)
    b = api.Batch([(dev(api, Q, d["rank_cap"]), d) for w, Q, p, d in inst], workers=4)
    K = len(api.tile_shapes())
    shape_of, rates = b.tune_tiles(steps_per_trial=1, rounds=1)
    assert len(shape_of) == len(inst) and all(0 <= k < K for k in shape_of)
    assert sorted(rates) == list(range(K)) and all(r > 0 for r in rates.values())
    b.step(1)
    for i, (_, _, _, d) in enumerate(inst):
        st = b.stats(i)
        assert st["device_status"] == 0 and max(st["rank"]) <= d["rank_cap"]
    b.close()
