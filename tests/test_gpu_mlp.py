"""GPU parity of the learned-pivot network (tt_mlp_*) against the FP64 oracle
(oracle/mlp.py), and of the solver's learned-pivot crosses.

Bars.  The GPU runs every product with BF16 operands and FP32 accumulation,
the oracle with the same BF16 operands and exact accumulation; FP32 sums of
<= 256 (forward) or m (weight gradients) terms, plus the rare operand that
sits on a BF16 rounding boundary and rounds the other way after an FP32
rather than FP64 pre-activation, keep scores within 2e-3 max|s| and each
gradient within 5e-3 relative Frobenius norm.  Features are FP64 on both
sides, stored as FP32 (1e-5).  Top-k selection is exact on distinct scores.
"""
import numpy as np
import pytest

from oracle import fv_full as FA
from oracle import mlp as M
from oracle import tt as T
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


def params(seed):
    P = M.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    P["b1"] = (0.1 * rng.standard_normal(M.HIDDEN)).astype(np.float32)
    P["b2"] = (0.1 * rng.standard_normal(M.HIDDEN)).astype(np.float32)
    P["b3"] = np.array([0.05], np.float32)
    return P


def to_dev(X):
    import torch
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m", [1, 77, 300, 1030])
def test_forward_matches_oracle(api, m):
    rng = np.random.default_rng(m)
    X = rng.standard_normal((m, M.F_IN)).astype(np.float32)
    P = params(1)
    net = api.PivotNet(P)
    s = net.forward(to_dev(X)).cpu().numpy()
    ref, _ = M.forward(P, X.astype(np.float64), bf16_ops=True)
    assert np.max(np.abs(s - ref)) <= 2e-3 * np.max(np.abs(ref)) + 1e-5


@pytest.mark.parametrize("m", [64, 300, 2000])
def test_gradients_and_loss_match_oracle(api, m):
    rng = np.random.default_rng(10 + m)
    X = rng.standard_normal((m, M.F_IN)).astype(np.float32)
    y = (rng.random(m) < 0.2).astype(np.float32)
    P = params(2)
    net = api.PivotNet(P)
    loss = float(net.grad(to_dev(X), to_dev(y)).cpu().numpy()[0])
    s, cache = M.forward(P, X.astype(np.float64), bf16_ops=True)
    g = M.backward(s, y.astype(np.float64), cache)
    assert loss == pytest.approx(M.loss(s, y), rel=2e-3)
    for k in M.init_params(0):
        got = net.g[k].cpu().numpy().reshape(g[k].shape)
        err = np.linalg.norm(got - g[k]) / max(np.linalg.norm(g[k]), 1e-30)
        assert err <= 5e-3, (k, err)


def test_adam_matches_oracle(api):
    rng = np.random.default_rng(7)
    X = rng.standard_normal((256, M.F_IN)).astype(np.float32)
    y = (rng.random(256) < 0.3).astype(np.float32)
    P = params(3)
    net = api.PivotNet(P)
    state = {}
    Pc = {k: v.copy() for k, v in P.items()}
    for t in range(1, 4):
        net.grad(to_dev(X), to_dev(y))
        g = {k: net.g[k].cpu().numpy().astype(np.float64) for k in P}
        net.adam_step(1e-3)
        Pc = M.adam(Pc, g, state, lr=1e-3, t=t)
        got = net.host()
        for k in P:
            assert np.allclose(got[k], Pc[k], rtol=1e-5, atol=1e-7), (k, t)
        # continue both from the GPU's parameters (same gradients next step)
        Pc = {k: got[k].copy() for k in P}


def test_features_match_oracle(api):
    rng = np.random.default_rng(11)
    for n1, n2, r, prev in ((40, 300, 6, [0, 17, 299]), (64, 97, 1, []), (200, 768, 12, [5, 6, 400, 767])):
        A = rng.standard_normal((n1, r))
        B = rng.standard_normal((n2, r)) * (0.7 ** np.arange(r))
        x0 = api.DevTT.from_cores(A, B)
        got = api.tt_mlp_features(x0, prev).cpu().numpy()
        ref = M.features(A, B, prev)
        assert np.allclose(got, ref, rtol=1e-5, atol=1e-5), np.max(np.abs(got - ref))


def test_topk_exact(api):
    import torch
    rng = np.random.default_rng(12)
    s = rng.permutation(5000).astype(np.float32) / 7.0
    for k in (1, 17, 64, 128):
        got = api.tt_mlp_topk(torch.from_numpy(s).cuda(), k).cpu().numpy()
        assert list(got) == list(M.top_indices(s.astype(np.float64), k))
    t = np.array([0.5, 2.0, 2.0, -1.0, 2.0, 0.5], np.float32)
    assert list(api.tt_mlp_topk(torch.from_numpy(t).cuda(), 4).cpu().numpy()) == [0, 1, 2, 4]


def test_training_lowers_the_loss(api):
    # a separable synthetic task: label = leverage feature above 1.2
    rng = np.random.default_rng(13)
    X = rng.standard_normal((4096, M.F_IN)).astype(np.float32)
    X[:, 0] = 1.0 + 0.5 * rng.standard_normal(4096)
    y = (X[:, 0] > 1.2).astype(np.float32)
    net = api.PivotNet(M.init_params(4))
    Xd, yd = to_dev(X), to_dev(y)
    first = float(net.grad(Xd, yd).cpu()[0])
    for _ in range(200):
        last = float(net.train_step(Xd, yd, 3e-3).cpu()[0])
    assert last < 0.5 * first, (first, last)


def _weno_setup(api, n=40):
    w = workload("nonlinear256_weno5", n=n, cap=16)
    Q, p = initial_tt(w)
    q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
    return w, Q, p, q0


def test_learned_solver_stage_is_exact_whatever_the_proposals(api):
    # an untrained network proposes poor pivots; the maxvol sweeps still
    # decide, so the stage stays within the WENO5 bar of Oracle A
    w, Q, p, q0 = _weno_setup(api)
    s = api.Solver(q0, "nonlinear", "weno5", w["n"], p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"], f=p["f"],
                   seed=0, pivots="learned")
    net = api.PivotNet(M.init_params(5))
    s.set_pivot_net(net)
    s.stage(0)
    got = s.get()
    ref = FA.ssprk3_stage([T.full(q) for q in Q], [T.full(q) for q in Q], 0, "nonlinear", "weno5", p, p["dt"])
    check_fields(got, ref, 10 * w["tol"], field_scales(ref, "nonlinear", p, p["dt"]))
    st = s.stats()
    assert st["learned_calls"] > 0 and st["device_status"] == 0
    s.close()


def test_recording_captures_labelled_rows(api):
    w, Q, p, q0 = _weno_setup(api)
    s = api.Solver(q0, "nonlinear", "weno5", w["n"], p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"], f=p["f"],
                   seed=0)
    s.record_pivots(True)
    s.stage(0)
    X, y = s.take_pivots()
    st = s.stats()
    assert X.shape[1] == M.F_IN and X.shape[0] == y.shape[0] > 0
    assert np.all(np.isfinite(X)) and set(np.unique(y)) <= {0.0, 1.0} and y.sum() > 0
    assert y.shape[0] >= st["cross_calls"] * w["n"]
    s.close()


def test_shipped_network_gain_over_plain_maxvol(api):
    # the trained network (train_pivots.py, seeds 20000+) on held-out 256^2
    # WENO5 instances: fewer cross sweeps than the plain maxvol start, and the
    # same accuracy class against the exact full-tensor stage
    import importlib
    tp = importlib.import_module("paper_2408_03483_gb300.train_pivots")
    net = api.PivotNet.shipped()
    sweeps = {"maxvol": 0, "learned": 0}
    for seed in (30000, 30003):
        w, Q, p = tp.instance(256, seed)
        for mode in ("maxvol", "learned"):
            s = tp.solver(api, w, Q, p, pivots=mode)
            if mode == "learned":
                s.set_pivot_net(net)
            s.step(1)  # stages 1 and 2 start from the site pivots of the stage before
            st = s.stats()
            sweeps[mode] += st["cross_sweeps"]
            if mode == "learned":
                # every cross starts from the network's proposal except the
                # lambda crosses of stages 1 and 2 (2 directions each), which
                # start from the previous stage's lambda by maxvol
                assert st["learned_calls"] == st["cross_calls"] - 4 > 0
                got = s.get()
                ref = FA.ssprk3_step([T.full(q) for q in Q], "nonlinear", "weno5", p, p["dt"])
                # the WENO5 bar per stage and field, three stages
                check_fields(got, ref, 3 * 10 * w["tol"], field_scales(ref, "nonlinear", p, p["dt"]))
            s.close()
    assert sweeps["learned"] < sweeps["maxvol"], sweeps
