"""Oracle A: plain full-tensor finite-volume discretisation (Sec. 2).

Oracle code (test infrastructure only).

Arrays are indexed U[i, j] with i the x cell (axis 0) and j the y cell
(axis 1) on a doubly periodic N_x x N_y grid of [0, lx] x [0, ly].
Periodicity is applied with np.roll.  A face array F[i] holds the flux on the
face x_{i-1/2} (between cells i-1 and i), so the flux difference of Eq. 2.11
is (F[i+1] - F[i]) / dx, i.e. (T^x - 1) F / dx of Eq. SWE-system-no-loop.
"""
import numpy as np

from . import coeffs

SCHEMES = ("up3", "up5", "weno5")


def nq_of(scheme):
    return 2 if scheme == "up3" else 3


# ---------------------------------------------------------------------------
# 1-D reconstruction along one axis
# ---------------------------------------------------------------------------

def _sh(v, s, axis):
    """v shifted so that out[i] = v[i+s] along `axis` (periodic)."""
    return np.roll(v, -s, axis=axis)


def weno5_step1(vm2, vm1, v0, vp1, vp2, eps):
    """WENO5 "-" side value at x_{i+1/2} from the 5-cell stencil (Sec. 2.3.1):
    printed candidates v^(r), ideal weights d_r, alpha_r = d_r/(beta_r+eps)^2,
    printed smoothness indicators beta_r."""
    q0 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0
    q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0
    q2 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0
    b0 = 13.0 / 12.0 * (v0 - 2.0 * vp1 + vp2) ** 2 + 0.25 * (3.0 * v0 - 4.0 * vp1 + vp2) ** 2
    b1 = 13.0 / 12.0 * (vm1 - 2.0 * v0 + vp1) ** 2 + 0.25 * (vm1 - vp1) ** 2
    b2 = 13.0 / 12.0 * (vm2 - 2.0 * vm1 + v0) ** 2 + 0.25 * (vm2 - 4.0 * vm1 + 3.0 * v0) ** 2
    a0 = 0.3 / (b0 + eps) ** 2
    a1 = 0.6 / (b1 + eps) ** 2
    a2 = 0.1 / (b2 + eps) ** 2
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)


def step1(v, axis, scheme, side, eps):
    """Step 1 "de-cell" averaging along `axis` (Sec. 2.3.1).

    side "-": value at the right face of each cell (x_{i+1/2}^-);
    side "+": value at the left face of each cell (x_{i-1/2}^+), the mirror
    image of the "-" side."""
    if scheme in ("up3", "up5"):
        st = coeffs.step1_linear(3 if scheme == "up3" else 5, side)
        out = np.zeros_like(v)
        for s, c in st.items():
            out += float(c) * _sh(v, s, axis)
        return out
    S = [_sh(v, s, axis) for s in (-2, -1, 0, 1, 2)]
    if side == "-":
        return weno5_step1(S[0], S[1], S[2], S[3], S[4], eps)
    return weno5_step1(S[4], S[3], S[2], S[1], S[0], eps)


def _betas(vm2, vm1, v0, vp1, vp2):
    """Step-2 smoothness indicators beta_0..2 (Sec. 2.3.2, printed)."""
    b0 = 13.0 / 12.0 * (v0 - 2.0 * vp1 + vp2) ** 2 + 0.25 * (3.0 * v0 - 4.0 * vp1 + vp2) ** 2
    b1 = 13.0 / 12.0 * (vm1 - 2.0 * v0 + vp1) ** 2 + 0.25 * (vm1 - vp1) ** 2
    b2 = 13.0 / 12.0 * (vm2 - 2.0 * vm1 + v0) ** 2 + 0.25 * (vm2 - 4.0 * vm1 + 3.0 * v0) ** 2
    return (b0, b1, b2)


def step2_point(S, m, scheme, eps):
    """Step-2 point value at Gauss point m from the stencil values
    S = (v_{j-2}, v_{j-1}, v_j, v_{j+1}, v_{j+2}) (entrywise arrays):
    Eq. fv-recon-step2 with candidates v^(r)_m = sum_l c^m_{rl} v_{j-r+l};
    Upwind3/Upwind5 use the linear weights, WENO5 the nonlinear weights
    alpha = gamma/(beta+eps)^2; the negative-weight point m=2 of the 3-point
    rule uses the sigma split of Eq. neg-coeff-treatment."""
    nq = nq_of(scheme)
    k = nq - 1
    Cs = coeffs.step2_C(nq)
    gam = coeffs.step2_gamma(nq)
    cand = [sum(Cs[m][r, l] * S[2 - r + l] for l in range(k + 1)) for r in range(k + 1)]
    if scheme == "weno5":
        beta = _betas(*S)
    if gam[m] is not None:
        if scheme == "weno5":
            alpha = [gam[m][r] / (beta[r] + eps) ** 2 for r in range(3)]
            return sum(alpha[r] * cand[r] for r in range(3)) / (alpha[0] + alpha[1] + alpha[2])
        return sum(gam[m][r] * cand[r] for r in range(k + 1))
    gp, gm, sp, sm = coeffs.step2_split()
    if scheme == "weno5":
        ap = [gp[r] / (beta[r] + eps) ** 2 for r in range(3)]
        am = [gm[r] / (beta[r] + eps) ** 2 for r in range(3)]
        up = sum(ap[r] * cand[r] for r in range(3)) / (ap[0] + ap[1] + ap[2])
        um = sum(am[r] * cand[r] for r in range(3)) / (am[0] + am[1] + am[2])
    else:
        up = sum(gp[r] * cand[r] for r in range(3))
        um = sum(gm[r] * cand[r] for r in range(3))
    return sp * up - sm * um


def step2(v, axis, scheme, eps):
    """Step 2 "de-cell" averaging along `axis` to the Gauss points
    (Sec. 2.3.2).  Returns shape (nq,) + v.shape: entry m is the point value
    at y_j + delta_m dy."""
    S = [_sh(v, s, axis) for s in (-2, -1, 0, 1, 2)]
    return np.stack([step2_point(S, m, scheme, eps) for m in range(nq_of(scheme))])


def face_states(U, direction, scheme, dx, dy):
    """Reconstructed states on the faces normal to `direction` ("x" or "y").

    Returns (Qm, Qp), each of shape (nq,) + U.shape, where for direction x
    Qm[m, i, j] is the state left of the face x_{i-1/2} (from cell i-1) and
    Qp[m, i, j] the state right of it (from cell i), at y_j + delta_m dy.
    Step 1 runs along the face normal, Step 2 along the face (Sec. 2.3)."""
    if direction == "x":
        a1, a2, e1, e2 = 0, 1, dx * dx, dy * dy
    else:
        a1, a2, e1, e2 = 1, 0, dy * dy, dx * dx
    right = step2(step1(U, a1, scheme, "-", e1), a2, scheme, e2)
    left = step2(step1(U, a1, scheme, "+", e1), a2, scheme, e2)
    Qm = np.roll(right, 1, axis=a1 + 1)  # cell i-1's right face value
    Qp = left
    return Qm, Qp


# ---------------------------------------------------------------------------
# Physical fluxes, eigenvalues, LLF (Sec. 2.1, Sec. 2.4)
# ---------------------------------------------------------------------------

def phys_flux(Q, direction, eqn, p):
    """F(Q) (direction x) or G(Q) (direction y) of Eq. linear-SWE /
    Eq. nonlinear-SWE.  Q = (q0, q1, q2)."""
    g = p["g"]
    if eqn == "linear":
        eta, u, v = Q
        H = p["H"]
        if direction == "x":
            return (H * u, g * eta, np.zeros_like(eta))
        return (H * v, np.zeros_like(eta), g * eta)
    h, hu, hv = Q
    if direction == "x":
        return (hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h)
    return (hv, hu * hv / h, hv * hv / h + 0.5 * g * h * h)


def max_speed(Qm, Qp, direction, eqn, p):
    """lambda of the LLF flux: sqrt(gH) (linear) or the entrywise max over the
    two face states of |u_n| + sqrt(g h) (nonlinear)."""
    g = p["g"]
    if eqn == "linear":
        return np.sqrt(g * p["H"])
    k = 1 if direction == "x" else 2
    lm = np.abs(Qm[k] / Qm[0]) + np.sqrt(g * Qm[0])
    lp = np.abs(Qp[k] / Qp[0]) + np.sqrt(g * Qp[0])
    return np.maximum(lm, lp)


def llf(Qm, Qp, direction, eqn, p):
    """Local Lax-Friedrichs flux, Eq. LLF / Sec. 2.4."""
    Fm = phys_flux(Qm, direction, eqn, p)
    Fp = phys_flux(Qp, direction, eqn, p)
    lam = max_speed(Qm, Qp, direction, eqn, p)
    return tuple(0.5 * (Fm[c] + Fp[c]) - 0.5 * lam * (Qp[c] - Qm[c]) for c in range(3))


GHOST = 3  # cells beyond each x boundary that one stage's stencils read


def rhs_bounded_x(Q, eqn, scheme, p, ghost):
    """L(Q) on a domain that is not periodic in x (Sec. 5.1, Sec. 5.3: the
    boundary values come from the exact solution), periodic in y.  ghost =
    (left, right): per field the cell averages of the GHOST cells beyond x = 0
    (cells -3..-1) and beyond x = lx (cells nx..nx+2), each GHOST x ny.  The
    fields are extended by these rows; the x faces are the nx + 1 faces
    x_{-1/2} .. x_{nx-1/2} between real or ghost cells, the y faces those of
    the nx real rows (their Step 2 in x reads the ghost rows)."""
    nx, ny = Q[0].shape
    dx, dy = p["lx"] / nx, p["ly"] / ny
    _, w = coeffs.gauss_legendre(nq_of(scheme))
    gl, gr = ghost
    E = [np.vstack([gl[c], Q[c], gr[c]]) for c in range(3)]
    g0 = GHOST
    out = [np.zeros_like(Q[0]) for _ in range(3)]
    # x faces: extended face i sits between extended cells i-1 and i; the
    # faces of the domain are i = GHOST .. GHOST + nx (no stencil there reads
    # a wrapped row)
    faces = [face_states(e, "x", scheme, dx, dy) for e in E]
    Qm = [f[0][:, g0:g0 + nx + 1] for f in faces]
    Qp = [f[1][:, g0:g0 + nx + 1] for f in faces]
    Fh = llf(Qm, Qp, "x", eqn, p)
    for c in range(3):
        Fq = np.tensordot(w, Fh[c], axes=(0, 0))  # (nx + 1) x ny
        out[c] -= (Fq[1:] - Fq[:-1]) / dx
    # y faces of the real rows
    faces = [face_states(e, "y", scheme, dx, dy) for e in E]
    Qm = [f[0][:, g0:g0 + nx] for f in faces]
    Qp = [f[1][:, g0:g0 + nx] for f in faces]
    Fh = llf(Qm, Qp, "y", eqn, p)
    for c in range(3):
        Fq = np.tensordot(w, Fh[c], axes=(0, 0))
        out[c] -= (np.roll(Fq, -1, axis=1) - Fq) / dy
    f = p["f"]
    out[1] += f * Q[2]
    out[2] -= f * Q[1]
    return out


def rhs(Q, eqn, scheme, p, ghost=None):
    """Semi-discrete operator L(Q) of Eq. SWE-system-cell-avg:
    -(F_{i+1/2}-F_{i-1/2})/dx - (G_{j+1/2}-G_{j-1/2})/dy + S (doubly periodic;
    with `ghost`, bounded in x: rhs_bounded_x)."""
    if ghost is not None:
        return rhs_bounded_x(Q, eqn, scheme, p, ghost)
    nx, ny = Q[0].shape
    dx, dy = p["lx"] / nx, p["ly"] / ny
    _, w = coeffs.gauss_legendre(nq_of(scheme))
    out = [np.zeros_like(Q[0]) for _ in range(3)]
    for direction, axis, d in (("x", 0, dx), ("y", 1, dy)):
        faces = [face_states(q, direction, scheme, dx, dy) for q in Q]
        Qm = [f[0] for f in faces]
        Qp = [f[1] for f in faces]
        Fh = llf(Qm, Qp, direction, eqn, p)  # each (nq, nx, ny)
        for c in range(3):
            Fq = np.tensordot(w, Fh[c], axes=(0, 0))  # face average, Sec. 2.2
            out[c] -= (np.roll(Fq, -1, axis=axis) - Fq) / d
    # source S = (0, f q2, -f q1): (0, fv, -fu) linear, (0, f hv, -f hu) nonlinear;
    # it is linear in Q, so its cell average is S(cell-averaged Q)
    f = p["f"]
    out[1] += f * Q[2]
    out[2] -= f * Q[1]
    return out


def euler(Q, eqn, scheme, p, dt, src=None, ghost=None):
    """Q + dt (L(Q) + src), src the cell averages of an external source at the
    stage's time (or None); ghost the x-boundary cells at that time (or None:
    periodic)."""
    L = rhs(Q, eqn, scheme, p, ghost)
    if src is None:
        return [Q[c] + dt * L[c] for c in range(3)]
    return [Q[c] + dt * (L[c] + src[c]) for c in range(3)]


def ssprk3_step(Q, eqn, scheme, p, dt, source=None, t=0.0, bc=None):
    """One SSP-RK3 step (Sec. 4.4, Eq. tt-ssprk3 without rounding) from time t;
    source(time) -> cell averages of an external source (a manufactured
    solution's forcing) and bc(time) -> the x-boundary ghost cells (an exact
    solution's), each evaluated at the stages' times t, t + dt, t + dt/2."""
    S = (lambda s: None) if source is None else source  # noqa: E731
    B = (lambda s: None) if bc is None else bc  # noqa: E731
    u1 = euler(Q, eqn, scheme, p, dt, S(t), B(t))
    f1 = euler(u1, eqn, scheme, p, dt, S(t + dt), B(t + dt))
    u2 = [0.75 * Q[c] + 0.25 * f1[c] for c in range(3)]
    f2 = euler(u2, eqn, scheme, p, dt, S(t + 0.5 * dt), B(t + 0.5 * dt))
    return [Q[c] / 3.0 + 2.0 / 3.0 * f2[c] for c in range(3)]


def ssprk3_stage(Qn, Qs, stage, eqn, scheme, p, dt):
    """Stage `stage` (0, 1, 2) of SSP-RK3 given u^n (Qn) and the current
    stage input Qs (u^n, u^(1), u^(2))."""
    f = euler(Qs, eqn, scheme, p, dt)
    if stage == 0:
        return f
    if stage == 1:
        return [0.75 * Qn[c] + 0.25 * f[c] for c in range(3)]
    return [Qn[c] / 3.0 + 2.0 / 3.0 * f[c] for c in range(3)]
