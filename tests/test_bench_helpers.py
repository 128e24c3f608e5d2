"""Host-side helpers of bench.py: the patch-sampled Oracle A check used at
4096^2 must equal the full-grid Oracle A step, and the replica throughput
counts every rank's work."""
import numpy as np

import bench
from oracle import fv_full as FA
from oracle import tt as T
from oracle import tt_fv as TB
from synth import initial_tt, workload


def test_patch_sampled_step_is_exact():
    # a full-tensor Oracle A step as the "after" state: the patch check (one
    # step on periodically wrapped patches with a 12-cell halo) must agree
    # with it to round-off, whatever the scheme
    for scheme in ("weno5", "up5"):
        w = workload("nonlinear256_weno5", n=96, scheme=scheme)
        Q, p = initial_tt(w)
        full = [T.full(q) for q in Q]
        ref = FA.ssprk3_step(full, "nonlinear", scheme, p, p["dt"])
        after = [T.tt_svd(r, 1e-15, 96) for r in ref]
        errs = bench.oracle_a_patches(Q, after, w, p, npatch=6, size=24, halo=12)
        assert max(errs) < 1e-12, (scheme, errs)


def test_patch_check_sees_a_tt_step_error():
    # Oracle B's truncated step differs from the exact step at the level of
    # its truncation: the patch check reports it per field
    w = workload("nonlinear256_weno5", n=64)
    Q, p = initial_tt(w)
    after = TB.step(Q, w, p, seed=0)
    errs = bench.oracle_a_patches(Q, after, w, p, npatch=6, size=24, halo=12)
    assert 1e-12 < errs[0] < 1e-6 and all(e < 1e-4 for e in errs), errs


def test_halo_below_the_step_reach_is_not_exact():
    # 6 cells of halo are fewer than one step reads (9): the wrapped patch
    # edge then reaches the interior and the check is no longer exact
    w = workload("nonlinear256_weno5", n=96, scheme="up5")
    Q, p = initial_tt(w)
    ref = FA.ssprk3_step([T.full(q) for q in Q], "nonlinear", "up5", p, p["dt"])
    after = [T.tt_svd(r, 1e-15, 96) for r in ref]
    errs = bench.oracle_a_patches(Q, after, w, p, npatch=6, size=24, halo=6)
    assert max(errs) > 1e-9, errs


def test_replica_value_counts_all_ranks():
    assert bench.replica_value(100, 4, 2000.0) == 200.0
    assert np.isclose(bench.replica_value(4096 ** 2 * 20, 1, 1e4), 4096 ** 2 * 2)
