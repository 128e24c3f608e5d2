"""The manufactured solution of the nonlinear SWE (Sec. 5.4) and its forcing.

Problem input, not solver arithmetic: the exact fields
    h = H + eta_hat sin(theta),  hu = h u_hat cos(theta),  hv = 0,
    theta = kx x + ky y - omega t,  omega = sqrt(g H (kx^2 + ky^2)),
and the source that makes them an exact solution of Eq. nonlinear-SWE with
the Coriolis source (0, f hv, -f hu): forcing = dQ/dt + dF/dx + dG/dy - S(Q),
differentiated symbolically (sympy) from the continuous equations and
rewritten as a sum of plane waves amp cos(m kx x + m ky y - m omega t + phase)
(every term is a product of sines and cosines of theta, so m <= 3).

Cell averages and TT cores of plane waves: synth/waves.py.

The paper's amplitudes (eta_hat = 1e-2 m on H = 1000 m, u_hat = 1e-2 m/s on
c = 100 m/s) are 1e-5 H and 1e-4 c, so its case is nearly linear; the
defaults here are 0.1 H and 0.1 so that every nonlinear flux term carries
weight.
"""
import math
from functools import lru_cache

from .waves import waves_cellavg, waves_tt  # noqa: F401  (re-exported)

MMS_DEFAULT = dict(g=9.81, H=1.0, f=1.0, eta_hat=0.1, u_hat=0.1, kx=2 * math.pi, ky=2 * math.pi)


@lru_cache(maxsize=None)
def _symbolic_forcing():
    """[(field, m, kind, coefficient expression)] with kind 'sin' or 'cos' of
    m theta, from sympy."""
    import sympy as sp
    from sympy.simplify.fu import TR8
    x, y, t = sp.symbols("x y t", real=True)
    g, H, f, eh, uh, kx, ky, om = sp.symbols("g H f eta_hat u_hat kx ky omega", positive=True)
    th = kx * x + ky * y - om * t
    h = H + eh * sp.sin(th)
    u = uh * sp.cos(th)
    hu, hv = h * u, sp.Integer(0)
    F = [hu, hu * u + g * h ** 2 / 2, hu * 0]
    G = [hv, hv * u, g * h ** 2 / 2]
    Q = [h, hu, hv]
    S = [0, f * hv, -f * hu]
    out = []
    for c in range(3):
        e = sp.expand(TR8(sp.expand(sp.diff(Q[c], t) + sp.diff(F[c], x) + sp.diff(G[c], y) - S[c])))
        rest = e
        for m in (1, 2, 3):
            for kind, fn in (("sin", sp.sin), ("cos", sp.cos)):
                coef = sp.expand(e).coeff(fn(m * th))
                if coef != 0:
                    out.append((c, m, kind, str(coef)))
                    rest = sp.expand(rest - coef * fn(m * th))
        if sp.simplify(rest) != 0:
            raise AssertionError(f"forcing of field {c} is not a sum of harmonics of theta: {rest}")
    return tuple(out)


def forcing_waves(**prm):
    """The forcing as plane waves: a list of (field, amp, kx, ky, omega,
    phase) meaning amp cos(kx x + ky y - omega t + phase) added to the
    right-hand side of `field`."""
    P = dict(MMS_DEFAULT, **prm)
    om = math.sqrt(P["g"] * P["H"] * (P["kx"] ** 2 + P["ky"] ** 2))
    env = dict(g=P["g"], H=P["H"], f=P["f"], eta_hat=P["eta_hat"], u_hat=P["u_hat"], kx=P["kx"], ky=P["ky"],
               omega=om)
    waves = []
    for c, m, kind, expr in _symbolic_forcing():
        amp = float(eval(expr.replace("^", "**"), {"__builtins__": {}}, env))  # noqa: S307 (own sympy output)
        phase = -math.pi / 2 if kind == "sin" else 0.0
        waves.append((c, amp, m * P["kx"], m * P["ky"], m * om, phase))
    return waves


def exact_waves(**prm):
    """The manufactured fields themselves as plane waves (same form as
    forcing_waves): h = H + eta_hat sin(theta), hu = H u_hat cos(theta) +
    eta_hat u_hat sin(2 theta) / 2, hv = 0."""
    P = dict(MMS_DEFAULT, **prm)
    om = math.sqrt(P["g"] * P["H"] * (P["kx"] ** 2 + P["ky"] ** 2))
    kx, ky = P["kx"], P["ky"]
    return [(0, P["H"], 0.0, 0.0, 0.0, 0.0),
            (0, P["eta_hat"], kx, ky, om, -math.pi / 2),
            (1, P["H"] * P["u_hat"], kx, ky, om, 0.0),
            (1, 0.5 * P["eta_hat"] * P["u_hat"], 2 * kx, 2 * ky, 2 * om, -math.pi / 2)]

