"""Oracle B, one SSP-RK3 stage of the TT finite-volume solver (Sec. 4).

Oracle code (test infrastructure only).

Composition (Sec. 4.1-4.4):
  * reconstruction on cores: Upwind3/Upwind5 by stencils on one core at a
    time (Sec. 4.3.1); WENO5 by two crosses per side (Algorithms 2 and 3,
    Sec. 4.3.2), the Step-2 result stored as a TT of size
    N_x x (N_q N_y) (x faces) or (N_q N_x) x N_y (y faces), quadrature index
    outermost ([m][j] blocks);
  * LLF flux in TT (Eq. LLF-TT): linear SWE by plain TT sums with
    lambda = sqrt(gH) and no rounding; nonlinear SWE with 1/h by Algorithm 1,
    products by TT Hadamard products rounded after each product and sum,
    lambda = max(|u-|+sqrt(g h-), |u+|+sqrt(g h+)) by cross -- or, with
    w["flux"] == "cross", the whole flux vector by one cross (the LF-cross
    alternative of Sec. 4.2);
  * face quadrature sum over the stacked index, then (T - 1)/dx on the core
    normal to the face (Eq. SWE-system-TT), plus the source term;
  * forward Euler F(u) = round(u + dt L(u)) and the SSP-RK3 combinations of
    Eq. tt-ssprk3, every round at the workload's (tol, cap).

Face convention: the face TT at row (x faces) index i is the face x_{i-1/2};
Qm there is cell i-1's right-face value, Qp is cell i's left-face value.
"""
import numpy as np

from . import coeffs
from . import cross as CR
from . import fv_full as FA
from . import recip as RC
from . import tt as T


# ---------------------------------------------------------------------------
# Linear reconstruction on cores (Sec. 4.3.1)
# ---------------------------------------------------------------------------

def _step2_core(C, scheme):
    """Step 2 applied to one core: for each Gauss point m the candidates
    v^(r)_m = sum_l c^m_{rl} C[j-r+l] combined with the linear weights (sigma
    split at m=2 of the 3-point rule); blocks stacked [m][j]."""
    nq = FA.nq_of(scheme)
    k = nq - 1
    Cs = coeffs.step2_C(nq)
    gam = coeffs.step2_gamma(nq)
    out = []
    for m in range(nq):
        cand = [sum(Cs[m][r, l] * np.roll(C, r - l, axis=0) for l in range(k + 1))
                for r in range(k + 1)]
        if gam[m] is not None:
            out.append(sum(gam[m][r] * cand[r] for r in range(k + 1)))
        else:
            gp, gm, sp, sm = coeffs.step2_split()
            out.append(sp * sum(gp[r] * cand[r] for r in range(3))
                       - sm * sum(gm[r] * cand[r] for r in range(3)))
    return np.vstack(out)


def recon_linear(X, direction, scheme):
    """Face TTs (Qm, Qp) of X for Upwind3/Upwind5: Step 1 on the core normal to
    the face, Step 2 on the other core (ranks unchanged)."""
    order = 3 if scheme == "up3" else 5
    right = coeffs.step1_linear(order, "-")
    left = coeffs.step1_linear(order, "+")
    A, B = X
    if direction == "x":
        Am = np.roll(T.core_stencil(A, right), 1, axis=0)  # cell i-1's right face
        Ap = T.core_stencil(A, left)
        Bs = _step2_core(B, scheme)
        return (Am, Bs), (Ap, Bs.copy())
    Bm = np.roll(T.core_stencil(B, right), 1, axis=0)
    Bp = T.core_stencil(B, left)
    As = _step2_core(A, scheme)
    return (As, Bm), (As.copy(), Bp)


GHOST = FA.GHOST


def _window_stencil(C, stencil, first, count):
    """sum_s c_s C[i+s, :] for i = first .. first+count-1 (no wrap: the rows
    read must exist)."""
    out = np.zeros((count, C.shape[1]))
    for s, c in stencil.items():
        out += float(c) * C[first + s:first + s + count]
    return out


def extend_x(X, ghost):
    """The TT of X with GHOST rows of an exact solution above and below in x:
    ghost = (Al, Ar, Be) with the exact solution's first-core rows of the
    cells -3..-1 (Al) and nx..nx+2 (Ar) and its second core Be; the cores are
    concatenated (rank r + r_E), X's columns zero on the ghost rows and the
    exact solution's zero on the real rows."""
    A, B = X
    Al, Ar, Be = ghost
    r, re = A.shape[1], Al.shape[1]
    top = np.hstack([np.zeros((GHOST, r)), Al])
    mid = np.hstack([A, np.zeros((A.shape[0], re))])
    bot = np.hstack([np.zeros((GHOST, r)), Ar])
    return (np.vstack([top, mid, bot]), np.hstack([B, Be]))


def recon_linear_bounded(X, ghost, direction, scheme):
    """Face TTs (Qm, Qp) of X for Upwind3/Upwind5 on a domain bounded in x
    with exact-solution ghost cells (periodic in y): x faces are the nx + 1
    faces x_{-1/2} .. x_{nx-1/2} (Qm: the right-face value of the cell
    below, Qp: the left-face value of the cell above, ghost or real); y faces
    are those of the nx real rows, their Step 2 in x reading the ghost rows."""
    order = 3 if scheme == "up3" else 5
    right = coeffs.step1_linear(order, "-")
    left = coeffs.step1_linear(order, "+")
    Ae, Be = extend_x(X, ghost)
    nx = X[0].shape[0]
    if direction == "x":
        Am = _window_stencil(Ae, right, GHOST - 1, nx + 1)  # cells -1 .. nx-1
        Ap = _window_stencil(Ae, left, GHOST, nx + 1)       # cells 0 .. nx
        Bs = _step2_core(Be, scheme)
        return (Am, Bs), (Ap, Bs.copy())
    Bm = np.roll(T.core_stencil(Be, right), 1, axis=0)
    Bp = T.core_stencil(Be, left)
    nq = FA.nq_of(scheme)
    k = nq - 1
    Cs = coeffs.step2_C(nq)
    gam = coeffs.step2_gamma(nq)
    blocks = []
    for m in range(nq):
        cand = [sum(Cs[m][r, l] * Ae[GHOST - r + l:GHOST - r + l + nx] for l in range(k + 1))
                for r in range(k + 1)]
        if gam[m] is not None:
            blocks.append(sum(gam[m][r] * cand[r] for r in range(k + 1)))
        else:
            gp, gm, sp, sm = coeffs.step2_split()
            blocks.append(sp * sum(gp[r] * cand[r] for r in range(3)) - sm * sum(gm[r] * cand[r] for r in range(3)))
    As = np.vstack(blocks)
    return (As, Bm), (As.copy(), Bp)


# ---------------------------------------------------------------------------
# WENO5 reconstruction by cross (Algorithms 2 and 3)
# ---------------------------------------------------------------------------

def _entries(X, I, J):
    return X[0][I, :] @ X[1][J, :].T


def _weno_step1_eval(X, mode, side, eps):
    n1, n2 = X[0].shape[0], X[1].shape[0]

    def ev(I, J):
        if mode == 0:
            S = [_entries(X, (I + s) % n1, J) for s in (-2, -1, 0, 1, 2)]
        else:
            S = [_entries(X, I, (J + s) % n2) for s in (-2, -1, 0, 1, 2)]
        if side == "-":
            return FA.weno5_step1(*S, eps)
        return FA.weno5_step1(*S[::-1], eps)
    return ev


def _weno_step2_eval(V, mode, nq, eps):
    """funWENOquad over the stacked index: mode 1 (x faces) the columns are
    (m, j) = m*n2 + j with the stencil along j; mode 0 (y faces) the rows are
    (m, i) = m*n1 + i with the stencil along i."""
    n1, n2 = V[0].shape[0], V[1].shape[0]

    def ev(I, J):
        I = np.asarray(I)
        J = np.asarray(J)
        out = np.empty((len(I), len(J)))
        if mode == 1:
            m_of, j_of = J // n2, J % n2
            for m in range(nq):
                sel = np.nonzero(m_of == m)[0]
                if len(sel) == 0:
                    continue
                S = [_entries(V, I, (j_of[sel] + s) % n2) for s in (-2, -1, 0, 1, 2)]
                out[:, sel] = FA.step2_point(S, m, "weno5", eps)
        else:
            m_of, i_of = I // n1, I % n1
            for m in range(nq):
                sel = np.nonzero(m_of == m)[0]
                if len(sel) == 0:
                    continue
                S = [_entries(V, (i_of[sel] + s) % n1, J) for s in (-2, -1, 0, 1, 2)]
                out[sel, :] = FA.step2_point(S, m, "weno5", eps)
        return out
    return ev


def recon_weno(X, direction, w, dx, dy, seed_base=0, stats=None):
    """Face TTs (Qm, Qp) of X for WENO5: Algorithm 2 (Step 1 by two crosses)
    then Algorithm 3 (Step 2 at all quadrature points by one cross per side)."""
    tol, cap = w["tol"], w["cap"]
    kick, sweeps = w.get("kick", 4), w.get("max_sweeps", 10)
    nq = 3
    n1, n2 = X[0].shape[0], X[1].shape[0]
    mode1 = 0 if direction == "x" else 1
    e1, e2 = (dx * dx, dy * dy) if direction == "x" else (dy * dy, dx * dx)
    out = {}
    for k, side in enumerate(("-", "+")):
        ev1 = _weno_step1_eval(X, mode1, side, e1)
        Vt, i1 = CR.cross2d(ev1, n1, n2, X, tol, cap, kick, sweeps,
                            seed=seed_base + 4 * k, return_info=True)
        if direction == "x":
            x0 = (Vt[0], np.vstack([Vt[1]] * nq))
            ev2 = _weno_step2_eval(Vt, 1, nq, e2)
            V, i2 = CR.cross2d(ev2, n1, nq * n2, x0, tol, cap, kick, sweeps,
                               seed=seed_base + 4 * k + 1, return_info=True)
        else:
            x0 = (np.vstack([Vt[0]] * nq), Vt[1])
            ev2 = _weno_step2_eval(Vt, 0, nq, e2)
            V, i2 = CR.cross2d(ev2, nq * n1, n2, x0, tol, cap, kick, sweeps,
                               seed=seed_base + 4 * k + 1, return_info=True)
        if stats is not None:
            stats.setdefault("cross", []).extend([i1, i2])
        out[side] = V
    Vm, Vp = out["-"], out["+"]
    if direction == "x":
        Qm = (np.roll(Vm[0], 1, axis=0), Vm[1])
    else:
        Qm = (Vm[0], np.roll(Vm[1], 1, axis=0))
    return Qm, Vp


# ---------------------------------------------------------------------------
# Fluxes (Sec. 4.2)
# ---------------------------------------------------------------------------

def _lambda_eval(hm, hum, hp, hup, g):
    def ev(I, J):
        a = _entries(hm, I, J)
        b = _entries(hum, I, J)
        c = _entries(hp, I, J)
        d = _entries(hup, I, J)
        return np.maximum(np.abs(b / a) + np.sqrt(g * a), np.abs(d / c) + np.sqrt(g * c))
    return ev


def flux_linear(Qm, Qp, direction, p):
    """LLF flux of the linear SWE in TT: F(Q) is linear and lambda = sqrt(gH)
    is a constant, so every term is a TT sum (no rounding, Sec. 4.2)."""
    g, H = p["g"], p["H"]
    lam = np.sqrt(g * H)
    k = 1 if direction == "x" else 2
    # F(Q) = (H q_k, g eta e_k): component 0 gets H q_k, component k gets g eta
    out = []
    for c in range(3):
        terms = []
        if c == 0:
            terms += [(0.5 * H, Qm[k]), (0.5 * H, Qp[k])]
        elif c == k:
            terms += [(0.5 * g, Qm[0]), (0.5 * g, Qp[0])]
        terms += [(-0.5 * lam, Qp[c]), (0.5 * lam, Qm[c])]
        out.append(T.add(terms))
    return out


def flux_nonlinear(Qm, Qp, direction, p, w, stats=None, seed=0):
    """LLF flux of the nonlinear SWE in TT with the Taylor reciprocal of h."""
    g = p["g"]
    tol, cap = w["tol"], w["cap"]
    R = lambda X: T.rnd(X, tol, cap)  # noqa: E731
    k = 1 if direction == "x" else 2
    F = {}
    for side, Q in (("-", Qm), ("+", Qp)):
        h, hu, hv = Q
        rh, its = RC.reciprocal(h, tol, cap, w.get("max_iter", 50))
        if stats is not None:
            stats.setdefault("taylor_iters", []).append(its)
        u = R(T.hadamard(hu, rh))
        v = R(T.hadamard(hv, rh))
        hh = R(T.hadamard(h, h))
        if direction == "x":
            f1 = R(T.add([(1.0, R(T.hadamard(hu, u))), (0.5 * g, hh)]))
            f2 = R(T.hadamard(hu, v))
            F[side] = (hu, f1, f2)
        else:
            g1 = R(T.hadamard(hv, u))
            g2 = R(T.add([(1.0, R(T.hadamard(hv, v))), (0.5 * g, hh)]))
            F[side] = (hv, g1, g2)
    n1, n2 = Qm[0][0].shape[0], Qm[0][1].shape[0]
    ev = _lambda_eval(Qm[0], Qm[k], Qp[0], Qp[k], g)
    lam = CR.cross2d(ev, n1, n2, Qp[0], tol, cap, w.get("kick", 4),
                     w.get("max_sweeps", 10), seed=seed)
    out = []
    for c in range(3):
        d = R(T.add([(1.0, Qp[c]), (-1.0, Qm[c])]))
        ld = R(T.hadamard(lam, d))
        out.append(R(T.add([(0.5, F["-"][c]), (0.5, F["+"][c]), (-0.5, ld)])))
    return out


def _llf_flux_eval(Qm, Qp, direction, g):
    """Entries of the LLF flux vector of Eq. LLF at the faces with its three
    components stacked along the first mode: row c n1 + i, column j holds
    component c at face point (i, j), from the six face states' entries with
    Oracle A's physical flux and wave speed."""
    n1 = Qm[0][0].shape[0]
    prm = {"g": g}

    def ev(I, J):
        I = np.asarray(I)
        out = np.empty((len(I), len(J)))
        comp, rows = I // n1, I % n1
        for c in range(3):
            sel = np.nonzero(comp == c)[0]
            if sel.size == 0:
                continue
            qm = [_entries(q, rows[sel], J) for q in Qm]
            qp = [_entries(q, rows[sel], J) for q in Qp]
            Fm = FA.phys_flux(qm, direction, "nonlinear", prm)
            Fp = FA.phys_flux(qp, direction, "nonlinear", prm)
            lam = FA.max_speed(qm, qp, direction, "nonlinear", prm)
            out[sel] = 0.5 * (Fm[c] + Fp[c]) - 0.5 * lam * (qp[c] - qm[c])
        return out
    return ev


def flux_cross(Qm, Qp, direction, p, w, seed=0):
    """The LF-cross alternative of Sec. 4.2: the whole LLF flux vector of one
    direction by a single cross of the face states (components stacked along
    the first mode, initial guess the h- faces), split into one TT per
    component sharing the second core."""
    n1, n2 = Qm[0][0].shape[0], Qm[0][1].shape[0]
    ev = _llf_flux_eval(Qm, Qp, direction, p["g"])
    A, B = CR.cross2d(ev, 3 * n1, n2, Qm[0], w["tol"], w["cap"], w.get("kick", 4), w.get("max_sweeps", 10),
                      seed=seed)
    return [(A[c * n1:(c + 1) * n1].copy(), B) for c in range(3)]


def quad_and_difference(Fh, direction, nq, n, d, bounded=False):
    """Face average sum_m w_m over the stacked index, then (T - 1)/d on the
    core normal to the face: returns the TT of (F_{i+1/2} - F_{i-1/2})/d
    (bounded: the x faces are nx + 1 rows and the difference does not wrap)."""
    _, wts = coeffs.gauss_legendre(nq)
    A, B = Fh
    if direction == "x":
        Bq = sum(wts[m] * B[m * n:(m + 1) * n] for m in range(nq))
        Ad = (A[1:] - A[:-1]) / d if bounded else (np.roll(A, -1, axis=0) - A) / d
        return (Ad, Bq)
    Aq = sum(wts[m] * A[m * n:(m + 1) * n] for m in range(nq))
    Bd = (np.roll(B, -1, axis=0) - B) / d
    return (Aq, Bd)


def ghost_tt(waves, field, n1, n2, t, lx, ly):
    """(Al, Ar, Be) of the exact solution `waves` for field at time t: its
    first-core rows of the GHOST cells beyond each x boundary and its second
    core (waves_tt on those rows)."""
    rows = np.concatenate([np.arange(-GHOST, 0), np.arange(n1, n1 + GHOST)])
    E = waves_tt(waves, field, n1, n2, t, lx, ly, rows=rows)
    if E is None:
        return (np.zeros((GHOST, 1)), np.zeros((GHOST, 1)), np.zeros((n2, 1)))
    return (E[0][:GHOST], E[0][GHOST:], E[1])


def rhs_terms(Q, w, p, stats=None, seed=0, t=0.0):
    """TT terms of L(Q) for each component: list of lists of (coef, TT).
    With w["bc_x"] == "exact" (linear SWE, Upwind3/Upwind5) the domain is
    bounded in x and the ghost cells hold the exact solution w["boundary"]
    (plane waves) at time t."""
    n1, n2 = Q[0][0].shape[0], Q[0][1].shape[0]
    dx, dy = p["lx"] / n1, p["ly"] / n2
    scheme, eqn = w["scheme"], w["eqn"]
    nq = FA.nq_of(scheme)
    bounded = w.get("bc_x", "periodic") == "exact"
    terms = [[], [], []]
    if bounded:
        if eqn != "linear" or scheme == "weno5":
            raise ValueError("the bounded-x form is built for the linear SWE with Upwind3/Upwind5")
        gh = [ghost_tt(w["boundary"], c, n1, n2, t, p["lx"], p["ly"]) for c in range(3)]
    for di, (direction, n, d) in enumerate((("x", n2, dx), ("y", n1, dy))):
        if bounded:
            faces = [recon_linear_bounded(q, gh[c], direction, scheme) for c, q in enumerate(Q)]
            Qm = [f[0] for f in faces]
            Qp = [f[1] for f in faces]
            Fh = flux_linear(Qm, Qp, direction, p)
            for c in range(3):
                terms[c].append((-1.0, quad_and_difference(Fh[c], direction, nq, n, d, bounded=True)))
            continue
        if scheme == "weno5":
            faces = [recon_weno(q, direction, w, dx, dy, seed_base=seed + 64 * di + 8 * c,
                                stats=stats) for c, q in enumerate(Q)]
        else:
            faces = [recon_linear(q, direction, scheme) for q in Q]
        Qm = [f[0] for f in faces]
        Qp = [f[1] for f in faces]
        if eqn == "linear":
            Fh = flux_linear(Qm, Qp, direction, p)
        elif w.get("flux", "products") == "cross":
            Fh = flux_cross(Qm, Qp, direction, p, w, seed=seed + 64 * di + 44)
        else:
            Fh = flux_nonlinear(Qm, Qp, direction, p, w, stats, seed=seed + 64 * di + 40)
        for c in range(3):
            terms[c].append((-1.0, quad_and_difference(Fh[c], direction, nq, n, d)))
    f = p["f"]
    if f != 0.0:
        terms[1].append((f, Q[2]))
        terms[2].append((-f, Q[1]))
    return terms


def _tol_u(w, c):
    """Tolerance of field c's forward-Euler and SSP rounds: eps^u of the step
    (Eq. modified-eps-tt-formula) when set, else the fixed tol."""
    return w["tol_u"][c] if "tol_u" in w else w["tol"]


def waves_tt(waves, field, n1, n2, t, lx, ly, rows=None):
    """Cell averages of sum amp exp(-decay x) cos(kx x + ky y - omega t +
    phase) over the waves of `field` as TT cores (first core on the x cells
    `rows`, by default 0..n1-1).  A wave is (field, amp, kx, ky, omega,
    phase[, decay]); decay = 0 unless given (the coastal Kelvin wave of
    Sec. 5.1 has decay = 1/R).  cos(a + b) = cos a cos b - sin a sin b is rank
    2; the y factors average to their centre values times sinc(ky dy/2); the x
    factors exp(-decay x) cos(kx x) and -exp(-decay x) sin(kx x) average to
    the real and minus the imaginary part of (1/dx) times the integral of
    exp(w x), w = -decay + i kx, over the cell -- for decay = 0 their centre
    values times sinc(kx dx/2)."""
    dx, dy = lx / n1, ly / n2
    xi = np.arange(n1) if rows is None else np.asarray(rows)
    xc = (xi + 0.5) * dx
    yc = (np.arange(n2) + 0.5) * dy
    A, B = [], []
    for wave in waves:
        c, amp, kx, ky, om, ph = wave[:6]
        decay = wave[6] if len(wave) > 6 else 0.0
        if c != field:
            continue
        sy = np.sinc(ky * dy / (2 * np.pi))  # numpy's sinc is sin(pi z)/(pi z)
        if decay == 0.0:
            sx = np.sinc(kx * dx / (2 * np.pi))
            a = kx * xc
            fc, fs = sx * np.cos(a), sx * np.sin(a)
        else:
            wz = complex(-decay, kx)
            lo = xi * dx
            # (e^{w hi} - e^{w lo}) / (w dx) = e^{w lo} (e^{w dx} - 1) / (w dx)
            step = complex(np.expm1(-decay * dx) * np.cos(kx * dx) - 2.0 * np.sin(kx * dx / 2) ** 2,
                           np.exp(-decay * dx) * np.sin(kx * dx))
            val = np.exp(wz * lo) * step / (wz * dx)
            fc, fs = val.real, val.imag
        b = ky * yc - om * t + ph
        A += [fc, -fs]
        B += [amp * sy * np.cos(b), amp * sy * np.sin(b)]
    if not A:
        return None
    return (np.stack(A, axis=1), np.stack(B, axis=1))


def forward_euler(Q, w, p, dt, stats=None, seed=0, t=0.0):
    """F(u) = round(u + dt (L(u) + S_m(t)), eps^u) per component (Eq.
    tt-forward-euler), S_m the external source w["forcing"] (plane waves) at
    time t when present."""
    terms = rhs_terms(Q, w, p, stats, seed, t)
    n1, n2 = Q[0][0].shape[0], Q[0][1].shape[0]
    out = []
    for c in range(3):
        X = [(1.0, Q[c])] + [(dt * a, Y) for a, Y in terms[c]]
        if w.get("forcing"):
            Sm = waves_tt(w["forcing"], c, n1, n2, t, p["lx"], p["ly"])
            if Sm is not None:
                X.append((dt, Sm))
        out.append(T.rnd(T.add(X), _tol_u(w, c), w["cap"]))
    return out


STAGE_TIME = (0.0, 1.0, 0.5)  # stage k evaluates L at t^n + STAGE_TIME[k] dt


def stage(Qn, Qs, k, w, p, stats=None, seed=0, t=0.0):
    """Stage k (0, 1, 2) of the TT SSP-RK3 of Eq. tt-ssprk3 given u^n (Qn) and
    the stage input Qs (u^n, u^(1), u^(2)); t = t^n."""
    f = forward_euler(Qs, w, p, p["dt"], stats, seed, t + STAGE_TIME[k] * p["dt"])
    if k == 0:
        return f
    a, b = (0.75, 0.25) if k == 1 else (1.0 / 3.0, 2.0 / 3.0)
    return [T.rnd(T.add([(a, Qn[c]), (b, f[c])]), _tol_u(w, c), w["cap"]) for c in range(3)]


def step_tolerances(Qn, w, p):
    """(eps_TT, [eps^u per field]) of a step (Sec. 4.4).  With
    w["eps_rule"] == "adaptive": eps^u = min(1e-3, C V^(1/2) dx^(p-1/2) / ||u||_F)
    at the beginning of the step (Eq. modified-eps-tt-formula) for the
    variable's own forward-Euler and SSP rounds, and eps_TT of
    Eq. eps-tt-formula (the same numerator over max_q ||q||_F) for every
    other rounding; V is the domain area, p the scheme's order (3 for
    Upwind3, 5 for Upwind5 and WENO5), C = w["c_eps"].  Otherwise the fixed
    w["tol"] for both."""
    if w.get("eps_rule", "fixed") != "adaptive":
        return w["tol"], [w["tol"]] * 3
    order = 3 if w["scheme"] == "up3" else 5
    nx = Qn[0][0].shape[0]
    num = w["c_eps"] * np.sqrt(p["lx"] * p["ly"]) * (p["lx"] / nx) ** (order - 0.5)
    norms = [T.fro(q) for q in Qn]
    eps_u = [min(1e-3, num / nm) if nm > 0 else 1e-3 for nm in norms]
    big = max(norms)
    return (num / big if big > 0 else 1e-3), eps_u


def step(Qn, w, p, stats=None, seed=0, t=0.0):
    """One full SSP-RK3 step in TT format (Eq. tt-ssprk3) from time t, with the
    step's truncation tolerances of Sec. 4.4."""
    eps_tt, eps_u = step_tolerances(Qn, w, p)
    ws = dict(w, tol=eps_tt, tol_u=eps_u)
    u1 = stage(Qn, Qn, 0, ws, p, stats, seed, t)
    u2 = stage(Qn, u1, 1, ws, p, stats, seed + 1000, t)
    return stage(Qn, u2, 2, ws, p, stats, seed + 2000, t)
