"""Reconstruction coefficients of Sec. 2.3 (Danis et al., arXiv 2408.03483).

Oracle code (test infrastructure only).

Coordinates are in cell units: cell j is the interval [-1/2, 1/2] around 0,
cell j+s is centred at s.  A reconstruction stencil "r" of a k-th order
candidate uses the cells j-r, ..., j-r+k (Sec. 2.3.2: v^(r)_m = sum_l
c^m_{rl} v_{j-r+l}).

The paper prints C^m and gamma as rationals that approximate irrational values
(Sec. 2.3.2); this module computes them exactly from their definition (the
cell-average-matching polynomial evaluated at a Gauss point) and keeps the
printed tables only as test fixtures.  The m=2 split weights and sigma^+- are
exact in the paper and are used as printed.
"""
from fractions import Fraction
from functools import lru_cache

import numpy as np


def gauss_legendre(nq):
    """Gauss-Legendre points delta_m (cell units, ascending: m=1 is the lowest)
    and weights w_m normalised to sum to 1 (the face average of Sec. 2.2)."""
    if nq == 2:
        d = 1.0 / (2.0 * np.sqrt(3.0))
        return np.array([-d, d]), np.array([0.5, 0.5])
    if nq == 3:
        d = np.sqrt(15.0) / 10.0
        return np.array([-d, 0.0, d]), np.array([5.0, 8.0, 5.0]) / 18.0
    raise ValueError("nq must be 2 or 3")


def _cell_moment(s, d):
    """Average of x**d over the cell [s-1/2, s+1/2] (exact rational)."""
    a = Fraction(2 * s - 1, 2)
    b = Fraction(2 * s + 1, 2)
    return (b ** (d + 1) - a ** (d + 1)) / (d + 1)


def cellavg_point_coeffs(cells, x):
    """Weights c_l with p(x) = sum_l c_l v_{cells[l]}, where p is the unique
    polynomial of degree len(cells)-1 whose averages over the given cells are
    v (the "best polynomial" of Sec. 2.3 that matches cell averages)."""
    k1 = len(cells)
    M = np.array([[float(_cell_moment(s, d)) for d in range(k1)] for s in cells])
    e = np.array([x ** d for d in range(k1)])
    # p(x) = e^T a with M a = v  =>  p(x) = (M^{-T} e)^T v
    return np.linalg.solve(M.T, e)


# ---------------------------------------------------------------------------
# Step 1 (Sec. 2.3.1): interface values of the 1-D reconstruction.
# "-" side: value at x_{i+1/2} (right face of cell i) -- printed in the paper.
# "+" side: value at x_{i-1/2} (left face of cell i) -- the mirror image, which
# the paper leaves to Shu (1998).
# ---------------------------------------------------------------------------

@lru_cache(maxsize=None)
def step1_candidates(order):
    """Printed candidate stencils v^(r)_{i+1/2} ("-" side) as dicts
    {offset: coefficient} and the ideal weights d_r (Sec. 2.3.1)."""
    if order == 3:
        cand = [
            {0: Fraction(1, 2), 1: Fraction(1, 2)},
            {-1: Fraction(-1, 2), 0: Fraction(3, 2)},
        ]
        d = [Fraction(2, 3), Fraction(1, 3)]
    elif order == 5:
        cand = [
            {0: Fraction(2, 6), 1: Fraction(5, 6), 2: Fraction(-1, 6)},
            {-1: Fraction(-1, 6), 0: Fraction(5, 6), 1: Fraction(2, 6)},
            {-2: Fraction(2, 6), -1: Fraction(-7, 6), 0: Fraction(11, 6)},
        ]
        d = [Fraction(3, 10), Fraction(3, 5), Fraction(1, 10)]
    else:
        raise ValueError("order must be 3 or 5")
    return cand, d


def mirror(stencil):
    """Mirror image of a stencil dict about the cell centre ("+" side)."""
    return {-s: c for s, c in stencil.items()}


@lru_cache(maxsize=None)
def step1_linear(order, side):
    """Combined linear (upwind) Step-1 stencil sum_r d_r v^(r): dict offset->coeff."""
    cand, d = step1_candidates(order)
    out = {}
    for st, w in zip(cand, d):
        if side == "+":
            st = mirror(st)
        for s, c in st.items():
            out[s] = out.get(s, Fraction(0)) + w * c
    return out


# ---------------------------------------------------------------------------
# Step 2 (Sec. 2.3.2): point values at the Gauss points y_j + delta_m dy.
# ---------------------------------------------------------------------------

@lru_cache(maxsize=None)
def step2_C(nq):
    """Exact coefficient matrices C^m (list over m of (k+1)x(k+1) arrays):
    row r holds c^m_{rl}, l=0..k, acting on v_{j-r+l}."""
    k = nq - 1
    delta, _ = gauss_legendre(nq)
    Cs = []
    for dm in delta:
        rows = []
        for r in range(k + 1):
            cells = [-r + l for l in range(k + 1)]
            rows.append(cellavg_point_coeffs(cells, dm))
        Cs.append(np.array(rows))
    return Cs


@lru_cache(maxsize=None)
def step2_gamma(nq):
    """Linear weights per quadrature point.

    nq=2 (Upwind3): omega^(r)_m = 1/2 (printed).
    nq=3 (Upwind5/WENO5): gamma_m for m=1,3 solved exactly as the weights that
    combine the three 3-cell point values into the 5-cell point value at
    delta_m; m=2 is returned as None (it uses the printed split, see
    step2_split)."""
    if nq == 2:
        return [np.array([0.5, 0.5]), np.array([0.5, 0.5])]
    delta, _ = gauss_legendre(3)
    Cs = step2_C(3)
    out = []
    for m, dm in enumerate(delta):
        if m == 1:
            out.append(None)
            continue
        c5 = cellavg_point_coeffs([-2, -1, 0, 1, 2], dm)
        # columns: candidate r embedded in the 5-cell positions (offset -2..2)
        E = np.zeros((5, 3))
        for r in range(3):
            for l in range(3):
                E[(-r + l) + 2, r] = Cs[m][r, l]
        g, res, _, _ = np.linalg.lstsq(E, c5, rcond=None)
        out.append(g)
    return out


def step2_split():
    """Printed split of the negative linear weights at m=2 (Sec. 2.3.2,
    Eq. neg-coeff-treatment; Shi, Hu & Shu 2002): gamma^+, gamma^-, sigma^+,
    sigma^-.  These values are exact."""
    gp = np.array([9.0 / 214.0, 98.0 / 107.0, 9.0 / 214.0])
    gm = np.array([9.0 / 67.0, 49.0 / 67.0, 9.0 / 67.0])
    return gp, gm, 107.0 / 40.0, 67.0 / 40.0


@lru_cache(maxsize=None)
def step2_linear_stencils(nq):
    """Combined linear Step-2 stencils, one 5-entry array per m over offsets
    -2..2 (nq=3) or 3-entry array over -1..1 (nq=2): sum_r omega_m^r C^m_r
    (with the sigma split at m=2 for nq=3)."""
    k = nq - 1
    Cs = step2_C(nq)
    gam = step2_gamma(nq)
    out = []
    for m in range(nq):
        if gam[m] is None:
            gp, gm, sp, sm = step2_split()
            wts = sp * gp - sm * gm
        else:
            wts = gam[m]
        st = np.zeros(2 * k + 1)
        for r in range(k + 1):
            for l in range(k + 1):
                st[(-r + l) + k] += wts[r] * Cs[m][r, l]
        out.append(st)
    return out
