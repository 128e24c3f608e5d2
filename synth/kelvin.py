"""The coastal Kelvin wave of Sec. 5.1: a closed-form solution of the linear
SWE on a domain bounded in x (the coast at x = 0), periodic in y,

    eta = -H A(y + c t) exp(-x / R),   u = 0,   v = c A(y + c t) exp(-x / R),
    A(s) = sum_m eta_m sin(k_m s),   c = sqrt(g H),   R = c / f.

It solves the equations exactly: eta_t + H v_y = 0 (both are H c A'(s)
exp(-x/R) with opposite signs), f v = g eta_x (c f = g H / R), and
v_t + g eta_y = (c^2 - g H) A'(s) exp(-x/R) = 0.  The paper prints both modes
on k^(1); with the second on k^(2) = 2 k^(1) the fields solve the SWE as they
must.  Two modes with eta_2 = 2 eta_1 as in the paper, on the unit square with
g = 9.81, H = 1 and f chosen so that the domain spans five decay lengths
(L / R = 5, as 5e6 m / 1e6 m in the paper); wavelengths 1 and 1/2 in y.
Each term is a damped plane wave (synth/waves.py: sin z = cos(z - pi/2),
omega = -k c), so its cell averages -- on the grid and on ghost cells beyond
x = 0 and x = 1 -- are exact.
"""
import math

KELVIN_DEFAULT = dict(g=9.81, H=1.0, eta=(0.01, 0.02), k=(2 * math.pi, 4 * math.pi), decay_lengths=5.0)


def kelvin_params(**prm):
    P = dict(KELVIN_DEFAULT, **prm)
    c = math.sqrt(P["g"] * P["H"])
    R = 1.0 / P["decay_lengths"]
    return dict(g=P["g"], H=P["H"], f=c / R, lx=1.0, ly=1.0)


def kelvin_waves(**prm):
    P = dict(KELVIN_DEFAULT, **prm)
    g, H = P["g"], P["H"]
    c = math.sqrt(g * H)
    dk = P["decay_lengths"]  # 1 / R on the unit square
    out = []
    for eta, k in zip(P["eta"], P["k"]):
        # eta_m sin(k (y + c t)) = eta_m cos(k y + k c t - pi/2): omega = -k c
        out.append((0, -H * eta, 0.0, k, -k * c, -math.pi / 2, dk))
        out.append((2, c * eta, 0.0, k, -k * c, -math.pi / 2, dk))
    return out
