"""GPU parity of the TT primitives against the FP64 CPU oracle, through the C ABI.

Tolerances: the exact routes (rounding at a clear spectral gap, stencils,
Khatri-Rao products) reproduce the oracle's reconstructed tensor to relative
L2 <= 1e-11; the range-finder rounding route stops at a certified residual of
1e-11 and is held to the 1e-10 parity bar; the cross is judged by its
approximation error against the exactly evaluated function (<= 10 tol).
"""
import numpy as np
import pytest

from oracle import cross as CR
from oracle import fv_full as FA
from oracle import recip as RC
from oracle import tt as T
from oracle import tt_fv as TB
from synth import initial_tt, random_tt, workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def dev(api, X, cap=None):
    return api.DevTT.from_cores(X[0], X[1], cap=cap)


# ------------------------------------------------------------------ rounding

@pytest.mark.parametrize("n1,n2,R,route", [
    (60, 90, 12, "factored"),
    (256, 768, 48, "factored"),
    (768, 256, 40, "factored"),
    (64, 64, 72, "direct"),
    (96, 300, 130, "direct"),
    (256, 768, 200, "range-finder"),
    (770, 257, 150, "range-finder"),
    # R > 112 with modes large enough that sketching through the cores costs
    # fewer flops than forming the n1 x n2 tensor: the range finder on cores
    (1024, 3072, 150, "range-finder"),
    (3000, 1100, 130, "range-finder"),
])
def test_round_matches_oracle(api, n1, n2, R, route):
    # decay 0.75: the spectrum falls below 1e-11 within 112 singular values,
    # so the range-finder route certifies its residual
    X = random_tt(n1, n2, R, seed=R + n1, decay=0.75)
    for tol, cap in ((1e-8, 64), (1e-4, 64), (1e-12, 20)):
        ref, info = T.round_tt(X, tol, cap)
        y, err = api.tt_round(dev(api, X), tol, cap)
        assert y.rank == info["rank"], (route, tol, cap)
        # exact routes agree to round-off; the range finder stops at a certified
        # residual of 1e-11, inside the 1e-10 parity bar
        bar = 1e-10 if route == "range-finder" else 1e-11
        assert rel(y.full().numpy(), T.full(ref)) < bar, (route, tol, cap)
        assert abs(err - info["err"]) <= 1e-10 * np.linalg.norm(info["sigma"]) + 1e-3 * info["err"]


def test_round_flat_spectrum_is_near_optimal(api):
    # decay 0.85 leaves more than 112 singular values above 1e-11: the range
    # finder cannot certify its residual; the result must still be as good as
    # the exact truncation up to a small residual
    X = random_tt(300, 500, 220, seed=11, decay=0.85)
    F = T.full(X)
    for tol, cap in ((1e-8, 40), (1e-3, 40)):
        ref, info = T.round_tt(X, tol, cap)
        y, err = api.tt_round(dev(api, X), tol, cap)
        e_opt = np.linalg.norm(T.full(ref) - F)
        e_gpu = np.linalg.norm(y.full().numpy() - F)
        assert y.rank == info["rank"]
        assert e_gpu <= e_opt + 1e-9 * np.linalg.norm(F)


def test_round_exact_recovery_and_edges(api):
    X = random_tt(100, 140, 9, seed=1)
    y, _ = api.tt_round(dev(api, X), 1e-14, 50)
    assert y.rank == 9
    assert rel(y.full().numpy(), T.full(X)) < 1e-13
    Z = (np.zeros((30, 3)), np.zeros((40, 3)))
    y, _ = api.tt_round(dev(api, Z), 1e-8, 5)
    assert y.rank == 1 and np.all(y.full().numpy() == 0.0)


def smooth_tt(n1, n2, phase, r):
    """TT-SVD (oracle) of a smooth periodic field; singular values fall off
    geometrically without clusters, like the solver's face fields."""
    x = (np.arange(n1) + 0.5) / n1
    y = (np.arange(n2) + 0.5) / n2
    X, Y = np.meshgrid(x, y, indexing="ij")
    F = np.exp(0.6 * np.sin(2 * np.pi * (X + Y) + phase) + 0.3 * np.cos(2 * np.pi * (X - 2 * Y)))
    return T.tt_svd(F, 1e-15, r)


@pytest.mark.parametrize("n1,n2,r1,r2", [(40, 70, 6, 5), (256, 768, 16, 16), (768, 256, 24, 20),
                                         (100, 100, 12, 10),
                                         # products of R = 120-144 columns on 1024-3072 modes: the
                                         # range finder through the Khatri-Rao cores
                                         (1024, 3072, 12, 12), (3072, 1024, 12, 10)])
def test_round_hadamard_matches_oracle(api, n1, n2, r1, r2):
    X = smooth_tt(n1, n2, 0.3, r1)
    Z = smooth_tt(n1, n2, 1.1, r2)
    for tol, cap in ((1e-8, 48), (1e-12, 32), (1e-3, 48)):
        ref, info = T.round_tt(T.hadamard(X, Z), tol, cap)
        y = api.tt_round_hadamard(dev(api, X), dev(api, Z), tol, cap)
        assert y.rank == info["rank"]
        assert rel(y.full().numpy(), T.full(ref)) < 1e-10


# ------------------------------------------------------------------ stencils

@pytest.mark.parametrize("scheme", ["up3", "up5"])
@pytest.mark.parametrize("direction", [0, 1])
def test_recon_linear_matches_oracle(api, scheme, direction):
    from paper_2408_03483_gb300 import capi
    X = random_tt(37, 53, 5, seed=7)  # ragged sizes, not multiples of any tile
    qm, qp = api.tt_recon_linear(dev(api, X), direction, capi.SCHEMES[scheme])
    rm, rp = TB.recon_linear(X, "x" if direction == 0 else "y", scheme)
    for got, ref in ((qm, rm), (qp, rp)):
        A, B = got.cores()
        np.testing.assert_allclose(A.numpy(), ref[0], rtol=0, atol=1e-13)
        np.testing.assert_allclose(B.numpy(), ref[1], rtol=0, atol=1e-13)


# ------------------------------------------------------------------ reciprocal

@pytest.mark.parametrize("n,stack", [(64, 1), (48, 3), (256, 3)])
def test_reciprocal_matches_oracle(api, n, stack):
    w = workload("nonlinear256_weno5", n=n)
    Q, _ = initial_tt(w)
    h = (Q[0][0], np.vstack([Q[0][1]] * stack))
    tol, cap = 1e-8, 32
    ref, it_ref = RC.reciprocal(h, tol, cap)
    y, it = api.tt_reciprocal(dev(api, h, cap), tol, cap)
    assert it == it_ref
    assert rel(y.full().numpy(), T.full(ref)) < 1e-10
    assert rel(y.full().numpy(), 1.0 / T.full(h)) < 1e-7


# ------------------------------------------------------------------ cross

@pytest.mark.parametrize("n1,n2,r", [(70, 90, 1), (70, 90, 7), (256, 768, 20)])
def test_cross_exact_recovery(api, n1, n2, r):
    from paper_2408_03483_gb300 import capi
    X = random_tt(n1, n2, r, seed=r)
    x0 = random_tt(n1, n2, 2, seed=5)
    y, sweeps = api.tt_cross(capi.TT_FN_ENTRY, [dev(api, X)], dev(api, x0), [], 1e-12, 40, n1, n2,
                             kick=4, max_sweeps=12, seed=3)
    assert rel(y.full().numpy(), T.full(X)) < 1e-11
    assert y.rank == r


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("side", [-1.0, 1.0])
def test_cross_weno_step1(api, mode, side):
    from paper_2408_03483_gb300 import capi
    n = 64
    w = workload("nonlinear256_weno5", n=n)
    Q, _ = initial_tt(w)
    X = Q[0]
    eps = (1.0 / n) ** 2
    ref = FA.step1(T.full(X), mode, "weno5", "-" if side < 0 else "+", eps)
    tol = 1e-10
    y, _ = api.tt_cross(capi.TT_FN_WENO_S1, [dev(api, X)], dev(api, X), [eps, side, mode], tol, 40, n, n,
                        seed=9)
    assert rel(y.full().numpy(), ref) <= 10 * tol
    # the oracle's own cross reaches the same accuracy
    ev = TB._weno_step1_eval(X, mode, "-" if side < 0 else "+", eps)
    yo = CR.cross2d(ev, n, n, X, tol, 40, 4, 10, seed=9)
    assert rel(T.full(yo), ref) <= 10 * tol


@pytest.mark.parametrize("mode", [1, 0])
def test_cross_weno_step2(api, mode):
    from paper_2408_03483_gb300 import capi
    n = 48
    w = workload("nonlinear256_weno5", n=n)
    Q, _ = initial_tt(w)
    V = Q[0]
    eps = (1.0 / n) ** 2
    axis = 1 if mode == 1 else 0
    pts = FA.step2(T.full(V), axis, "weno5", eps)  # (3, n, n)
    ref = np.hstack(list(pts)) if mode == 1 else np.vstack(list(pts))
    n1, n2 = ref.shape
    x0 = (V[0], np.vstack([V[1]] * 3)) if mode == 1 else (np.vstack([V[0]] * 3), V[1])
    tol = 1e-10
    y, _ = api.tt_cross(capi.TT_FN_WENO_S2, [dev(api, V)], dev(api, x0), [eps, mode, 3], tol, 40, n1, n2,
                        seed=2)
    assert rel(y.full().numpy(), ref) <= 10 * tol


def test_cross_llf_lambda(api):
    from paper_2408_03483_gb300 import capi
    n = 80
    g = 9.81
    rng = np.random.default_rng(6)
    u = [rng.uniform(0.0, 1.0, (n, 1)) for _ in range(4)]
    v = [rng.uniform(0.0, 1.0, (2 * n, 1)) for _ in range(4)]
    one1, one2 = np.ones((n, 1)), np.ones((2 * n, 1))
    hm = (np.hstack([one1, 0.01 * u[0]]), np.hstack([one2, v[0]]))
    hp = hm
    qm = (np.hstack([0.1 * one1, 0.05 * u[2]]), np.hstack([one2, v[2]]))
    # qp > qm > 0 everywhere: the max picks the + side, lambda is smooth
    qp = (np.hstack([0.11 * one1, 0.05 * u[2]]), np.hstack([one2, v[2]]))
    F = [T.full(t) for t in (hm, qm, hp, qp)]
    ref = np.maximum(np.abs(F[1] / F[0]) + np.sqrt(g * F[0]), np.abs(F[3] / F[2]) + np.sqrt(g * F[2]))
    tol = 1e-9
    y, _ = api.tt_cross(capi.TT_FN_LLF_LAMBDA, [dev(api, t) for t in (hm, qm, hp, qp)], dev(api, hp), [g],
                        tol, 40, n, 2 * n, seed=4)
    ev = TB._lambda_eval(hm, qm, hp, qp, g)
    yo = CR.cross2d(ev, n, 2 * n, hp, tol, 40, 4, 10, seed=4)
    e_oracle = rel(T.full(yo), ref)
    assert rel(y.full().numpy(), ref) <= max(10 * tol, 2 * e_oracle)
