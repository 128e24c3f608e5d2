"""Pins of the oracle's reconstruction coefficients (Sec. 2.3) against values
the paper prints, closed forms and polynomial exactness."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import coeffs
from oracle import fv_full as FA
from conftest import golden_path


def _load_printed():
    out = {}
    with open(golden_path("recon_coeffs_printed.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            name, row = parts[0], int(parts[1])
            vals = [float(Fraction(x)) for x in parts[2:]]
            out.setdefault(name, {})[row] = vals
    return {k: np.array([v[r] for r in sorted(v)]) for k, v in out.items()}


PRINTED = _load_printed()


def test_gauss_points_match_library():
    for nq in (2, 3):
        d, w = coeffs.gauss_legendre(nq)
        x, wl = np.polynomial.legendre.leggauss(nq)
        np.testing.assert_allclose(d, x / 2.0, atol=1e-15)
        np.testing.assert_allclose(w, wl / 2.0, atol=1e-15)


@pytest.mark.parametrize("nq,tag", [(2, "up3"), (3, "up5")])
def test_C_matches_printed(nq, tag):
    Cs = coeffs.step2_C(nq)
    for m in range(nq):
        np.testing.assert_allclose(Cs[m], PRINTED[f"C_{tag}_m{m + 1}"], atol=2e-6, rtol=0)


def test_C_up3_row_structure():
    # U3 rows are the linear interpolants (1-d, d) and (-d, 1+d) at delta_m
    Cs = coeffs.step2_C(2)
    d, _ = coeffs.gauss_legendre(2)
    for m in range(2):
        np.testing.assert_allclose(Cs[m][0], [1 - d[m], d[m]], atol=1e-15)
        np.testing.assert_allclose(Cs[m][1], [-d[m], 1 + d[m]], atol=1e-15)


def test_gamma_matches_printed_and_is_exact():
    g = coeffs.step2_gamma(3)
    np.testing.assert_allclose(g[0], PRINTED["gamma_m1"][0], atol=2e-7, rtol=0)
    np.testing.assert_allclose(g[2], PRINTED["gamma_m3"][0], atol=2e-7, rtol=0)
    # exact weights sum to one; the printed ones do only to ~1.5e-7
    assert abs(g[0].sum() - 1.0) < 1e-14
    assert abs(PRINTED["gamma_m1"][0].sum() - 1.0) > 1e-7


def test_split_weights_reproduce_centre_value():
    gp, gm, sp, sm = coeffs.step2_split()
    np.testing.assert_allclose(gp, PRINTED["gamma_m2_plus"][0], atol=1e-16)
    np.testing.assert_allclose(gm, PRINTED["gamma_m2_minus"][0], atol=1e-16)
    np.testing.assert_allclose([sp, sm], PRINTED["sigma"][0], atol=1e-16)
    # combined weights (-9/80, 49/40, -9/80) and the classical 5-cell
    # point value at the cell centre (9, -116, 2134, -116, 9)/1920
    np.testing.assert_allclose(sp * gp - sm * gm, [-9 / 80, 49 / 40, -9 / 80], atol=1e-15)
    st = coeffs.step2_linear_stencils(3)[1]
    np.testing.assert_allclose(st, np.array([9, -116, 2134, -116, 9]) / 1920.0, atol=1e-15)


def _poly_cell_avgs(coef, cells):
    """Exact cell averages of sum_d coef[d] x^d over unit cells centred at `cells`."""
    out = []
    for s in cells:
        a, b = s - 0.5, s + 0.5
        out.append(sum(c * (b ** (d + 1) - a ** (d + 1)) / (d + 1) for d, c in enumerate(coef)))
    return np.array(out)


def _poly_val(coef, x):
    return sum(c * x ** d for d, c in enumerate(coef))


@pytest.mark.parametrize("order,deg", [(3, 2), (5, 4)])
def test_step1_linear_polynomial_exactness(order, deg):
    rng = np.random.default_rng(3)
    for side, x in (("-", 0.5), ("+", -0.5)):
        st = coeffs.step1_linear(order, side)
        for d in range(deg + 1):
            coef = np.zeros(d + 1)
            coef[d] = 1.0
            coef[:d] += rng.standard_normal(d)
            cells = sorted(st)
            avg = dict(zip(cells, _poly_cell_avgs(coef, cells)))
            val = sum(float(c) * avg[s] for s, c in st.items())
            assert abs(val - _poly_val(coef, x)) < 1e-13
    # one degree higher is not reproduced (the stencil is exactly of this order)
    coef = np.zeros(deg + 2)
    coef[-1] = 1.0
    st = coeffs.step1_linear(order, "-")
    avg = dict(zip(sorted(st), _poly_cell_avgs(coef, sorted(st))))
    assert abs(sum(float(c) * avg[s] for s, c in st.items()) - _poly_val(coef, 0.5)) > 1e-6


def test_step1_printed_upwind_stencils():
    st3 = coeffs.step1_linear(3, "-")
    assert st3 == {-1: Fraction(-1, 6), 0: Fraction(5, 6), 1: Fraction(1, 3)}
    st5 = coeffs.step1_linear(5, "-")
    assert {k: v * 60 for k, v in st5.items()} == {-2: 2, -1: -13, 0: 47, 1: 27, 2: -3}


@pytest.mark.parametrize("nq,deg", [(2, 1), (3, 4)])
def test_step2_polynomial_exactness_and_quadrature_identity(nq, deg):
    d, w = coeffs.gauss_legendre(nq)
    k = nq - 1
    sts = coeffs.step2_linear_stencils(nq)
    cells = list(range(-k, k + 1))
    rng = np.random.default_rng(5)
    for dd in range(deg + 1):
        coef = rng.standard_normal(dd + 1)
        avg = _poly_cell_avgs(coef, cells)
        for m in range(nq):
            assert abs(sts[m] @ avg - _poly_val(coef, d[m])) < 1e-13
    # sum_m w_m Q_m = identity: the face average of the point values is the
    # cell average (the Gauss rule integrates the reconstruction exactly)
    comb = sum(w[m] * sts[m] for m in range(nq))
    e = np.zeros(2 * k + 1)
    e[k] = 1.0
    np.testing.assert_allclose(comb, e, atol=1e-15)


def test_weno_point_functions_exact_on_quadratics():
    # every candidate is exact for degree <= 2 and the weights sum to 1
    rng = np.random.default_rng(11)
    d3, _ = coeffs.gauss_legendre(3)
    for _ in range(5):
        coef = rng.standard_normal(3)
        S = list(_poly_cell_avgs(coef, [-2, -1, 0, 1, 2]))
        v = FA.weno5_step1(*S, eps=1e-6)
        assert abs(v - _poly_val(coef, 0.5)) < 1e-12
        v = FA.weno5_step1(*S[::-1], eps=1e-6)  # "+" side = mirrored stencil
        assert abs(v - _poly_val(coef, -0.5)) < 1e-12
        for m in range(3):
            v = FA.step2_point([np.array(s) for s in S], m, "weno5", 1e-6)
            assert abs(float(v) - _poly_val(coef, d3[m])) < 1e-12


def test_weno_step1_reduces_to_upwind5_on_smooth_data():
    # on a smooth profile sampled ever finer the WENO5 and Upwind5 values agree
    # to higher and higher order (weights -> ideal weights)
    errs = []
    for n in (32, 64, 128):
        x = (np.arange(n) + 0.5) / n
        v = np.sin(2 * np.pi * x)  # point samples serve as stencil data
        S = [np.roll(v, -s) for s in (-2, -1, 0, 1, 2)]
        wv = FA.weno5_step1(*S, eps=(1.0 / n) ** 2)
        st = coeffs.step1_linear(5, "-")
        uv = sum(float(c) * np.roll(v, -s) for s, c in st.items())
        errs.append(np.max(np.abs(wv - uv)))
    assert errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8
