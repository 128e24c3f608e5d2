"""The barotropic tide of Sec. 5.3: a closed-form solution of the linear SWE
on a domain that is not periodic in x,

    eta = sum_m eta_m cos(k_m x) cos(w_m t),
    u   = sum_m g eta_m w_m k_m / (w_m^2 - f^2) sin(k_m x) sin(w_m t),
    v   = sum_m g eta_m f k_m   / (w_m^2 - f^2) sin(k_m x) cos(w_m t),

with w_m^2 = g H k_m^2 + f^2 (the paper writes the hat-omega of the
inertia-gravity wave in the denominators; with w_m in its place these
fields solve the linear SWE with the Coriolis source exactly).  Two modes
with wavelengths 4L/5 and 4L/9 and eta_2 = 2 eta_1 as in the paper, on the
unit square (L = 1), independent of y, so periodic in y.  Each product of
trigonometric factors is written as plane waves (synth/waves.py) so its cell
averages -- on the grid and on ghost cells beyond x = 0 and x = 1 -- are exact.
"""
import math

TIDE_DEFAULT = dict(g=9.81, H=1.0, f=1.0, eta=(0.01, 0.02), wavelength=(0.8, 4.0 / 9.0))


def tide_waves(**prm):
    P = dict(TIDE_DEFAULT, **prm)
    g, H, f = P["g"], P["H"], P["f"]
    out = []
    for eta, lam in zip(P["eta"], P["wavelength"]):
        k = 2 * math.pi / lam
        w = math.sqrt(g * H * k * k + f * f)
        A = g * eta * w * k / (w * w - f * f)
        B = g * eta * f * k / (w * w - f * f)
        # cos(kx) cos(wt) = [cos(kx - wt) + cos(kx + wt)] / 2
        out += [(0, eta / 2, k, 0.0, w, 0.0), (0, eta / 2, k, 0.0, -w, 0.0)]
        # sin(kx) sin(wt) = [cos(kx - wt) - cos(kx + wt)] / 2
        out += [(1, A / 2, k, 0.0, w, 0.0), (1, -A / 2, k, 0.0, -w, 0.0)]
        # sin(kx) cos(wt) = [sin(kx + wt) + sin(kx - wt)] / 2, sin z = cos(z - pi/2)
        out += [(2, B / 2, k, 0.0, -w, -math.pi / 2), (2, B / 2, k, 0.0, w, -math.pi / 2)]
    return out


def tide_params(**prm):
    P = dict(TIDE_DEFAULT, **prm)
    return dict(g=P["g"], H=P["H"], f=P["f"], lx=1.0, ly=1.0)
