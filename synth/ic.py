"""Seeded synthetic initial conditions in TT form.

A 2-D TT here is a pair (A, B) of float64 arrays, A of shape (nx, r) and B of
shape (ny, r), representing X[i, j] = sum_k A[i, k] B[j, k] (the paper's
G1(i) G2(j) with G2 = B^T).  Every initial field is a short sum of separable
products, so its TT cores are written down directly from exact 1-D cell
averages: no rounding, no cross.

Widths follow the exp(-d^2 / w^2) convention, so w = 0.1 is the "/0.01" of
the linear bump.  Periodic bumps are periodised by summing the images at
shifts -2..2 of the domain length, which keeps them smooth across the
boundary.
"""
import math

import numpy as np

G_DEFAULT = 9.81


def _erf(x):
    return np.vectorize(math.erf, otypes=[float])(x)


def gauss_cellavg_1d(n, length, centre, width, images=2):
    """Exact cell averages of sum_s exp(-(x - centre - s*length)^2 / width^2)
    over the n uniform cells of [0, length]."""
    dx = length / n
    a = np.arange(n) * dx
    b = a + dx
    acc = np.zeros(n)
    for s in range(-images, images + 1):
        c = centre + s * length
        acc += _erf((b - c) / width) - _erf((a - c) / width)
    return acc * (0.5 * math.sqrt(math.pi) * width / dx)


def _gl_cellavg_1d(n, length, fun, npts=8):
    """Cell averages of a smooth 1-D function by npts-point Gauss-Legendre per cell."""
    x, w = np.polynomial.legendre.leggauss(npts)
    dx = length / n
    centres = (np.arange(n) + 0.5) * dx
    pts = centres[:, None] + 0.5 * dx * x[None, :]
    return (fun(pts) * w[None, :]).sum(axis=1) * 0.5


def tt_to_full(A, B):
    return A @ B.T


def _zero_tt(nx, ny):
    return (np.zeros((nx, 1)), np.zeros((ny, 1)))


# ---------------------------------------------------------------------------
# Workloads (the five solver configurations plus small test variants).
# ---------------------------------------------------------------------------

WORKLOADS = {
    # Linear SWE, 64^2, Upwind3, bump 0.01*exp(-r^2/0.01), H=1, CFL 0.4
    "linear64_up3": dict(eqn="linear", scheme="up3", n=64, steps=100, tol=1e-10, cap=8,
                         ic="linear_bump", amp=0.01, width=0.1, cfl=0.4, f=0.0),
    # Nonlinear SWE, 256^2, WENO5 by cross, Taylor reciprocal, 3 seeded bumps
    "nonlinear256_weno5": dict(eqn="nonlinear", scheme="weno5", n=256, steps=500, tol=1e-8,
                               cap=32, ic="bumps", amp=0.1, nbumps=3, seed=1, cfl=0.4, f=0.0),
    # Precision form: nonlinear 1024^2 Upwind5 geostrophic vortex, f=10
    "vortex1024_up5": dict(eqn="nonlinear", scheme="up5", n=1024, steps=200, tol=1e-8, cap=48,
                           ic="vortex", amp=0.05, width2=0.02, cfl=0.4, f=10.0),
    # Learned-pivot form: nonlinear 4096^2 WENO5
    "nonlinear4096_weno5": dict(eqn="nonlinear", scheme="weno5", n=4096, steps=100, tol=1e-8,
                                cap=64, ic="bumps", amp=0.1, nbumps=3, seed=7, cfl=0.4, f=0.0),
}


def workload(name, **over):
    w = dict(WORKLOADS[name])
    w.update(over)
    return w


def _bumps(n, amp, nbumps, seed, width_range=(0.03, 0.1), amp_range=None):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(nbumps, 2))
    widths = rng.uniform(width_range[0], width_range[1], size=nbumps)
    if amp_range is None:
        amps = np.full(nbumps, amp)
    else:
        amps = rng.uniform(amp_range[0], amp_range[1], size=nbumps)
    A = [np.ones((n, 1))]
    B = [np.ones((n, 1))]
    for k in range(nbumps):
        gx = gauss_cellavg_1d(n, 1.0, centres[k, 0], widths[k])
        gy = gauss_cellavg_1d(n, 1.0, centres[k, 1], widths[k])
        A.append(amps[k] * gx[:, None])
        B.append(gy[:, None])
    return (np.hstack(A), np.hstack(B)), dict(centres=centres, widths=widths, amps=amps)


def initial_tt(w):
    """Initial TT cores [(A, B)] * 3 for a workload dict, plus the parameter
    dict of the solver (g, H, f, lx, ly, dt)."""
    n = w["n"]
    g = w.get("g", G_DEFAULT)
    p = dict(g=g, H=w.get("H", 1.0), f=w.get("f", 0.0), lx=1.0, ly=1.0)
    dx = 1.0 / n
    if w["ic"] == "linear_bump":
        gx = gauss_cellavg_1d(n, 1.0, 0.5, w["width"])
        eta = (w["amp"] * gx[:, None], gx[:, None].copy())
        Q = [eta, _zero_tt(n, n), _zero_tt(n, n)]
        p["dt"] = w["cfl"] * dx / math.sqrt(g * p["H"])
        return Q, p
    if w["ic"] == "bumps":
        h, meta = _bumps(n, w["amp"], w["nbumps"], w["seed"],
                         amp_range=w.get("amp_range"))
        Q = [h, _zero_tt(n, n), _zero_tt(n, n)]
        hmax = float(np.max(tt_to_full(*h)))
        p["dt"] = w["cfl"] * dx / math.sqrt(g * hmax)
        return Q, p
    if w["ic"] == "vortex":
        # h = 1 + a exp(-r^2/s), geostrophic u = -(g/f) dh/dy, v = (g/f) dh/dx
        a, s, f = w["amp"], w["width2"], w["f"]
        e = lambda x: np.exp(-((x - 0.5) ** 2) / s)  # noqa: E731
        de = lambda x: -2.0 * (x - 0.5) / s * np.exp(-((x - 0.5) ** 2) / s)  # noqa: E731
        ee = lambda x: e(x) ** 2  # noqa: E731
        ede = lambda x: e(x) * de(x)  # noqa: E731
        one = np.ones((n, 1))
        cx = {k: _gl_cellavg_1d(n, 1.0, fn)[:, None] for k, fn in
              dict(e=e, de=de, ee=ee, ede=ede).items()}
        c = g / f
        h = (np.hstack([one, a * cx["e"]]), np.hstack([one, cx["e"]]))
        # u = -c a e(x) de(y);  hu = u + a e u = -c a [e de] - c a^2 [ee ede]
        hu = (np.hstack([-c * a * cx["e"], -c * a * a * cx["ee"]]),
              np.hstack([cx["de"], cx["ede"]]))
        # v = c a de(x) e(y);  hv = c a [de e] + c a^2 [ede ee]
        hv = (np.hstack([c * a * cx["de"], c * a * a * cx["ede"]]),
              np.hstack([cx["e"], cx["ee"]]))
        Q = [h, hu, hv]
        full = [tt_to_full(*q) for q in Q]
        speed = np.max(np.sqrt(full[1] ** 2 + full[2] ** 2) / full[0] + np.sqrt(g * full[0]))
        p["dt"] = w["cfl"] * dx / speed
        return Q, p
    raise ValueError(w["ic"])


def ensemble(count=256, seed=1000, sizes=(128, 256, 512, 1024), cap_range=(8, 64)):
    """Workload dicts of the batched ensemble: instance k draws its grid size
    (uniform over `sizes`), rank cap (uniform integer in cap_range) and 1-3
    Gaussian bumps of amplitude U[0.01, 0.1] and width U[0.03, 0.1] from
    default_rng(seed + k); the reconstructions are a seeded permutation of
    equal thirds of up3 / up5 / weno5.  Nonlinear SWE, tol 1e-8, CFL 0.4."""
    rng = np.random.default_rng(seed)
    schemes = (["up3", "up5", "weno5"] * ((count + 2) // 3))[:count]
    schemes = [schemes[i] for i in rng.permutation(count)]
    out = []
    for k in range(count):
        rk = np.random.default_rng(seed + k)
        n = int(rk.choice(np.asarray(sizes)))
        cap = int(rk.integers(cap_range[0], cap_range[1] + 1))
        nb = int(rk.integers(1, 4))
        out.append(dict(eqn="nonlinear", scheme=schemes[k], n=n, steps=100, tol=1e-8, cap=cap, ic="bumps",
                        amp=0.1, amp_range=(0.01, 0.1), nbumps=nb, seed=seed + k, cfl=0.4, f=0.0))
    return out


def random_tt(n1, n2, r, seed, decay=None):
    """Seeded random TT cores (A, B) of rank r; with `decay`, column k of A is
    scaled by decay**k so the singular values fall off geometrically."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n1, r))
    B = rng.standard_normal((n2, r))
    if decay is not None:
        A = A * (decay ** np.arange(r))[None, :]
    return A, B


# ---------------------------------------------------------------------------
# Inertia-gravity wave (Sec. 5.2): closed-form linear SWE solution, doubly
# periodic, two modes; exact cell averages by the sinc factor.
# ---------------------------------------------------------------------------

def igw_cellavg(n, t, g=9.81, H=1.0, f=1.0, eta_hat=(0.1, 0.2), kmul=(1, 2)):
    """Cell averages of (eta, u, v) of the two-mode inertia-gravity wave at time
    t on [0,1]^2: eta = eta_hat cos(th), u, v as in Sec. 5.2 with
    omega^2 = g H (kx^2 + ky^2) + f^2 and th = kx x + ky y - omega t."""
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc, indexing="ij")
    out = [np.zeros((n, n)) for _ in range(3)]
    for eh, km in zip(eta_hat, kmul):
        kx = ky = 2.0 * math.pi * km
        om = math.sqrt(g * H * (kx * kx + ky * ky) + f * f)
        th = kx * X + ky * Y - om * t
        sx = math.sin(kx * dx / 2) / (kx * dx / 2)
        sy = math.sin(ky * dx / 2) / (ky * dx / 2)
        c = np.cos(th) * sx * sy
        s = np.sin(th) * sx * sy
        amp = g * eh / (om * om - f * f)
        out[0] += eh * c
        out[1] += amp * (om * kx * c - f * ky * s)
        out[2] += amp * (om * ky * c + f * kx * s)
    return out
