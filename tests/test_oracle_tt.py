"""Pins of Oracle B (TT algebra, rounding, cross, Taylor reciprocal, TT stage)
against library SVDs, brute force on full matrices, closed forms and Oracle A."""
import math

import numpy as np
import pytest

from conftest import golden_path
from oracle import cross as CR
from oracle import fv_full as FA
from oracle import recip as RC
from oracle import tt as T
from oracle import tt_fv as TB
from synth import initial_tt, random_tt, tt_to_full, workload


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ---------------------------------------------------------------- rounding

@pytest.mark.parametrize("n1,n2,r", [(40, 60, 7), (64, 192, 30), (33, 17, 50)])
def test_round_exact_recovery(n1, n2, r):
    A, B = random_tt(n1, n2, r, seed=r)
    X = (A, B)
    Y, info = T.round_tt(X, 1e-13, 10 ** 6)
    assert info["rank"] == min(r, n1, n2)
    assert rel(T.full(Y), T.full(X)) < 1e-13


@pytest.mark.parametrize("tol,cap", [(1e-3, 100), (1e-6, 100), (1e-6, 5), (0.5, 100)])
def test_round_is_eckart_young(tol, cap):
    A, B = random_tt(50, 70, 25, seed=2, decay=0.5)
    F = A @ B.T
    Y, info = T.round_tt((A, B), tol, cap)
    U, s, Vt = np.linalg.svd(F)
    # library SVD of the full matrix: same rank rule, same truncated matrix
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
    k = next((i for i in range(1, len(s) + 1) if (tail[i] if i < len(s) else 0.0) <= tol * np.linalg.norm(s)), len(s))
    k = min(k, cap)
    assert info["rank"] == k
    Fk = (U[:, :k] * s[:k]) @ Vt[:k]
    assert rel(T.full(Y), Fk) < 1e-12
    err = np.linalg.norm(T.full(Y) - F)
    if cap >= 100:
        assert err <= tol * np.linalg.norm(F) * (1 + 1e-12)
    assert abs(err - info["err"]) <= 1e-10 * np.linalg.norm(F)


def test_truncation_rule_edges():
    assert T.truncation_rank(np.zeros(5), 1e-8, 10) == 1
    assert T.truncation_rank(np.array([1.0, 0.0, 0.0]), 1e-8, 10) == 1
    assert T.truncation_rank(np.array([1.0, 1.0, 1.0]), 1e-8, 2) == 2
    # tail exactly at the bound is kept out (<=)
    s = np.array([3.0, 4.0])
    assert T.truncation_rank(s, 4.0 / 5.0, 10) == 1
    assert T.truncation_rank(s, 4.0 / 5.0 - 1e-12, 10) == 2


def test_round_zero_tensor():
    Y, info = T.round_tt((np.zeros((8, 3)), np.zeros((9, 3))), 1e-8, 5)
    assert info["rank"] == 1 and np.all(T.full(Y) == 0.0)


# ---------------------------------------------------------------- algebra

def test_hadamard_sum_scale_shift_match_full():
    X = random_tt(20, 30, 3, seed=4)
    Y = random_tt(20, 30, 4, seed=5)
    FX, FY = T.full(X), T.full(Y)
    assert T.rank(T.hadamard(X, Y)) == 12
    np.testing.assert_allclose(T.full(T.hadamard(X, Y)), FX * FY, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(T.full(T.add([(2.0, X), (-0.5, Y)])), 2 * FX - 0.5 * FY, atol=1e-13)
    np.testing.assert_allclose(T.full(T.shift(X, 2, 0)), np.roll(FX, -2, axis=0), atol=1e-14)
    np.testing.assert_allclose(T.full(T.shift(X, -3, 1)), np.roll(FX, 3, axis=1), atol=1e-14)
    assert abs(T.tsum(X) - FX.sum()) < 1e-11 * np.abs(FX).sum()
    assert abs(T.fro(X) - np.linalg.norm(FX)) < 1e-12 * np.linalg.norm(FX)


def test_linear_tt_recon_matches_full():
    # Upwind TT reconstruction on cores (Sec. 4.3.1) equals the full-tensor
    # dimension-by-dimension reconstruction (Sec. 2.3) entry by entry
    n = 24
    X = random_tt(n, n, 3, seed=8)
    F = T.full(X)
    for scheme in ("up3", "up5"):
        for direction in ("x", "y"):
            Qm_tt, Qp_tt = TB.recon_linear(X, direction, scheme)
            Qm, Qp = FA.face_states(F, direction, scheme, 1.0 / n, 1.0 / n)
            nq = Qm.shape[0]
            fm, fp = T.full(Qm_tt), T.full(Qp_tt)
            for m in range(nq):
                if direction == "x":
                    np.testing.assert_allclose(fm[:, m * n:(m + 1) * n], Qm[m], atol=1e-13)
                    np.testing.assert_allclose(fp[:, m * n:(m + 1) * n], Qp[m], atol=1e-13)
                else:
                    np.testing.assert_allclose(fm[m * n:(m + 1) * n, :], Qm[m], atol=1e-13)
                    np.testing.assert_allclose(fp[m * n:(m + 1) * n, :], Qp[m], atol=1e-13)


# ---------------------------------------------------------------- reciprocal

@pytest.mark.parametrize("amp", [0.05, 0.3])
def test_reciprocal_within_geometric_tail(amp):
    w = workload("nonlinear256_weno5", n=48, amp=amp)
    Q, _ = initial_tt(w)
    h = Q[0]
    tol = 1e-10
    y, it = RC.reciprocal(h, tol, 64)
    F = T.full(h)
    ref = 1.0 / F
    xavg = F.mean()
    q = np.max(np.abs(1.0 - F / xavg))
    # ||1/x - y|| <= (1/x_avg) * (Err q/(1-q) * sqrt(N) + rounding); rounding at
    # tol per operation, a few dozen operations
    N = F.size
    bound = (1.0 / xavg) * (tol * q / (1 - q) * math.sqrt(N) + 50 * tol * math.sqrt(N) * 2)
    assert np.linalg.norm(T.full(y) - ref) <= bound
    assert it <= math.ceil(math.log(tol) / math.log(q)) + 2


def test_reciprocal_constant_is_exact_in_one_iteration():
    X = (np.full((10, 1), 2.0), np.full((12, 1), 1.5))  # 3.0 everywhere
    y, it = RC.reciprocal(X, 1e-12, 4)
    assert it == 1
    np.testing.assert_allclose(T.full(y), np.full((10, 12), 1.0 / 3.0), rtol=1e-15)


def test_reciprocal_of_rank1_h_matches_rank1_cross():
    # h = f(x) g(y) > 0 is rank 1, so 1/h = (1/f)(1/g) is rank 1 too: the
    # cross of 1/h recovers it exactly (1e-12) from one fibre pair, and
    # Algorithm 1 reaches the same tensor to its geometric tail and rounds
    # back to (numerical) rank 1
    n1, n2 = 40, 56
    xs = (np.arange(n1) + 0.5) / n1
    ys = (np.arange(n2) + 0.5) / n2
    f = (1.0 + 0.04 * np.sin(2 * np.pi * xs))[:, None]
    g = (1.0 + 0.03 * np.cos(2 * np.pi * ys))[:, None]
    h = (f, g)
    F = T.full(h)
    Yc = CR.cross2d(lambda I, J: 1.0 / F[np.ix_(I, J)], n1, n2, h, 1e-12, 8, kick=4, max_sweeps=8)
    assert rel(T.full(Yc), 1.0 / F) < 1e-12
    y, it = RC.reciprocal(h, 1e-10, 16)
    assert rel(T.full(y), T.full(Yc)) < 1e-8
    assert T.rank(T.round_tt(y, 1e-9, 16)[0]) == 1


def test_planted_taylor_sign_error_is_caught(monkeypatch):
    # flipping the sign of x~ (1 + x/x_avg) must break the 1/h pin
    orig = T.add

    def flipped(terms):
        if len(terms) == 2 and terms[0][0] == 1.0 and T.rank(terms[0][1]) == 1 and terms[1][0] < 0:
            terms = [terms[0], (-terms[1][0], terms[1][1])]
        return orig(terms)
    w = workload("nonlinear256_weno5", n=32)
    Q, _ = initial_tt(w)
    monkeypatch.setattr(T, "add", flipped)
    y, _ = RC.reciprocal(Q[0], 1e-10, 32, max_iter=5)
    monkeypatch.setattr(T, "add", orig)
    assert rel(T.full(y), 1.0 / T.full(Q[0])) > 1e-3


# ---------------------------------------------------------------- cross

def test_splitmix64_reference_values():
    with open(golden_path("splitmix64_reference.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    g = 0x9E3779B97F4A7C15
    for k, hexv in rows:
        assert CR.splitmix64(int(k) * g) == int(hexv, 16)


def test_maxvol_invariant_and_volume():
    rng = np.random.default_rng(0)
    U = rng.standard_normal((80, 6))
    I = CR.maxvol(U, delta=1e-2)
    B = U @ np.linalg.inv(U[I, :])
    assert np.max(np.abs(B)) <= 1.0 + 1e-2 + 1e-12
    # brute force on a tiny case: maxvol reaches a submatrix within a factor of
    # the optimum volume (dominance |B|<=1+d bounds the ratio by (1+d)^r r^{r/2})
    U = rng.standard_normal((9, 3))
    I = CR.maxvol(U, delta=0.0)
    import itertools
    best = max(abs(np.linalg.det(U[list(c), :])) for c in itertools.combinations(range(9), 3))
    assert abs(np.linalg.det(U[I, :])) >= best / (3 ** 1.5) - 1e-12


@pytest.mark.parametrize("r", [1, 5, 12])
def test_cross_recovers_low_rank(r):
    n1, n2 = 70, 90
    A, B = random_tt(n1, n2, r, seed=10 + r)
    F = A @ B.T
    x0 = random_tt(n1, n2, 2, seed=99)
    Y, info = CR.cross2d(lambda I, J: F[np.ix_(I, J)], n1, n2, x0, 1e-12, 40, kick=4,
                         max_sweeps=12, return_info=True)
    assert rel(T.full(Y), F) < 1e-11
    assert info["rank"] == r


def test_cross_cap_limited_stops_on_stagnation():
    # singular values 0.7^k: at cap 10 the skeleton cannot reach tol 1e-12;
    # the cross stops once a sweep no longer halves its prediction error,
    # well before max_sweeps, with an error within a small factor of the
    # best rank-10 approximation's (sigma_10 / ||F|| ~ 2.8e-2 here)
    n1, n2, r = 90, 120, 40
    rng = np.random.default_rng(31)
    U, _ = np.linalg.qr(rng.standard_normal((n1, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n2, r)))
    s = 0.7 ** np.arange(r)
    F = (U * s) @ V.T
    best = np.sqrt(np.sum(s[10:] ** 2)) / np.linalg.norm(s)
    x0 = random_tt(n1, n2, 2, seed=5)
    Y, info = CR.cross2d(lambda I, J: F[np.ix_(I, J)], n1, n2, x0, 1e-12, 10, kick=4,
                         max_sweeps=30, return_info=True)
    assert info["rank"] == 10
    assert info["sweeps"] < 30
    assert best <= rel(T.full(Y), F) <= 10 * best


def test_cross_plateau_just_above_tol_stops():
    # a rank-3 field plus full-rank noise of relative size ~3e-9: with tol
    # 1e-9 the skeleton's prediction error plateaus at the noise, above tol;
    # the cross stops once a sweep no longer halves it (within 10 tol)
    # instead of running all max_sweeps, and its result carries the noise's
    # error only
    n1, n2 = 80, 100
    A, B = random_tt(n1, n2, 3, seed=41)
    F0 = A @ B.T
    rng = np.random.default_rng(42)
    N = rng.standard_normal((n1, n2))
    F = F0 + 3e-9 * np.linalg.norm(F0) / np.linalg.norm(N) * N
    x0 = random_tt(n1, n2, 2, seed=43)
    Y, info = CR.cross2d(lambda I, J: F[np.ix_(I, J)], n1, n2, x0, 1e-9, 40, kick=4,
                         max_sweeps=30, return_info=True)
    assert info["sweeps"] < 30
    assert info["err"] <= 10 * 1e-9
    assert rel(T.full(Y), F) <= 10 * 1e-9


def test_cross_weno_step1_against_full():
    n = 40
    w = workload("nonlinear256_weno5", n=n)
    Q, _ = initial_tt(w)
    X = Q[0]
    F = T.full(X)
    eps = (1.0 / n) ** 2
    for side in ("-", "+"):
        ref = FA.step1(F, 0, "weno5", side, eps)
        ev = TB._weno_step1_eval(X, 0, side, eps)
        assert np.allclose(ev(np.arange(n), np.arange(n)), ref, atol=1e-14, rtol=0)
        Y = CR.cross2d(ev, n, n, X, 1e-10, 40, 4, 12, seed=3)
        assert rel(T.full(Y), ref) <= 10 * 1e-10


# ---------------------------------------------------------------- TT stage

@pytest.mark.parametrize("scheme", ["up3", "up5"])
def test_tt_stage_linear_matches_full(scheme):
    w = workload("linear64_up3", n=32, scheme=scheme)
    Q, p = initial_tt(w)
    Qf = [T.full(q) for q in Q]
    for k, (Qn, Qs) in enumerate([(Q, Q)]):
        a = TB.stage(Qn, Qs, 0, w, p)
        b = FA.ssprk3_stage([T.full(q) for q in Qn], [T.full(q) for q in Qs], 0, "linear", scheme, p, p["dt"])
        for c in range(3):
            assert rel(T.full(a[c]), b[c]) < 1e-12
    step_tt = TB.step(Q, w, p)
    step_full = FA.ssprk3_step(Qf, "linear", scheme, p, p["dt"])
    for c in range(3):
        assert rel(T.full(step_tt[c]), step_full[c]) < 1e-12


@pytest.mark.parametrize("scheme", ["up3", "weno5"])
def test_tt_stage_nonlinear_matches_full(scheme):
    # no rank cap binds and tol is tight: the TT stage reproduces the
    # full-tensor stage to a small multiple of tol relative to ||Q||
    w = workload("nonlinear256_weno5", n=24, scheme=scheme, tol=1e-11, cap=24)
    Q, p = initial_tt(w)
    a = TB.stage(Q, Q, 0, w, p)
    b = FA.ssprk3_stage([T.full(q) for q in Q], [T.full(q) for q in Q], 0, "nonlinear", scheme, p, p["dt"])
    scale = np.linalg.norm(b[0])
    for c in range(3):
        assert np.linalg.norm(T.full(a[c]) - b[c]) <= 1e3 * 1e-11 * scale


# ---------------------------------------------------------------- LF-cross flux

def test_lf_cross_flux_matches_the_exact_llf_flux():
    # the LF-cross of Sec. 4.2 (one cross of the whole flux vector, components
    # stacked along the first mode) against Oracle A's LLF flux evaluated on
    # the full face tensors: within the cross's tolerance class (10 tol of the
    # stacked flux), per direction
    w = workload("nonlinear256_weno5", n=32, scheme="up5", flux="cross")
    Q, p = initial_tt(w)
    # a state with flow: momentum from one forward-Euler stage
    Q = TB.forward_euler(Q, dict(w, flux="products"), p, p["dt"])
    for direction in ("x", "y"):
        faces = [TB.recon_linear(q, direction, "up5") for q in Q]
        Qm = [f[0] for f in faces]
        Qp = [f[1] for f in faces]
        F = TB.flux_cross(Qm, Qp, direction, p, w, seed=3)
        ex = FA.llf([T.full(q) for q in Qm], [T.full(q) for q in Qp], direction, "nonlinear", p)
        num = sum(np.linalg.norm(T.full(F[c]) - ex[c]) ** 2 for c in range(3)) ** 0.5
        den = sum(np.linalg.norm(ex[c]) ** 2 for c in range(3)) ** 0.5
        assert num <= 10 * w["tol"] * den, (direction, num / den)
        # the three components share the second core
        assert F[0][1] is F[1][1] is F[2][1]


@pytest.mark.parametrize("scheme", ["up3", "weno5"])
def test_lf_cross_step_matches_full_tensor(scheme):
    from parity import check_fields, field_scales
    w = workload("nonlinear256_weno5", n=32, scheme=scheme, flux="cross")
    Q, p = initial_tt(w)
    out = TB.step(Q, w, p, seed=0)
    ref = FA.ssprk3_step([T.full(q) for q in Q], "nonlinear", scheme, p, p["dt"])
    check_fields(out, ref, 3 * 10 * w["tol"], field_scales(ref, "nonlinear", p, p["dt"]))


def test_planted_lf_cross_mistake_fails(monkeypatch):
    # a dissipation term with the wrong sign in the stacked evaluator must
    # fail the exact-flux pin
    orig = TB._llf_flux_eval

    def wrong(Qm, Qp, direction, g):
        ev = orig(Qm, Qp, direction, g)
        n1 = Qm[0][0].shape[0]

        def ev2(I, J):
            I = np.asarray(I)
            out = ev(I, J)
            comp, rows = I // n1, I % n1
            for c in range(3):
                sel = np.nonzero(comp == c)[0]
                if sel.size:
                    qm = TB._entries(Qm[c], rows[sel], J)
                    qp = TB._entries(Qp[c], rows[sel], J)
                    out[sel] += (qp - qm) * 5.0
            return out
        return ev2
    monkeypatch.setattr(TB, "_llf_flux_eval", wrong)
    with pytest.raises(AssertionError):
        test_lf_cross_flux_matches_the_exact_llf_flux()
