"""Per-field parity measures shared by the GPU tests and the benchmark.

Every comparison is made on reconstructed full tensors, field by field:

* ``field_errors`` -- the relative L2 error of each field against the
  reference's own norm (an absolute error where the reference field is
  identically zero).  This is what the tests and the benchmark report.
* ``field_scales`` -- the scale a truncation-decided bar is measured on.
  A rounding at relative tolerance tol perturbs the rounded tensor by at most
  tol times its own norm (Sec. 3.2).  The forward-Euler round of field c acts
  on u_c + dt L(u)_c (size ||u_c||), but the flux roundings act on the face
  fluxes F_c and G_c (Sec. 4.2), whose errors reach u_c through
  dt (T - 1)/dx, an operator of norm at most 2 dt/dx (Eq. SWE-system-TT).  So
  the truncation error of field c in one stage is bounded by a small multiple
  of tol * S_c with
      S_c = ||u_c|| + 2 dt/dx ||F_c(u)|| + 2 dt/dy ||G_c(u)||.
  For h this is ||h|| up to the small mass-flux term; for hu and hv the
  pressure g h^2/2 inside F_c and G_c dominates, and momentum that starts
  at rest stays far smaller than it.
"""
import numpy as np


def _full(x):
    if isinstance(x, np.ndarray):
        return x
    if hasattr(x, "full"):  # a device TT of the CUDA package
        f = x.full()
        return f.numpy() if hasattr(f, "numpy") else np.asarray(f)
    A, B = x  # an oracle TT (A, B)
    return A @ B.T


def fulls(state):
    return [_full(q) for q in state]


def field_errors(got, ref):
    """Per-field relative L2 error ||got_c - ref_c|| / ||ref_c|| (absolute
    where ||ref_c|| = 0)."""
    g, r = fulls(got), fulls(ref)
    out = []
    for a, b in zip(g, r):
        nb = np.linalg.norm(b)
        e = np.linalg.norm(a - b)
        out.append(float(e / nb) if nb > 0 else float(e))
    return out


def field_scales(ref, eqn, p, dt, d=None):
    """S_c of the module docstring for the reference state ``ref`` (cell
    widths d = (dx, dy); by default the domain of p over ref's shape)."""
    from oracle import fv_full as FA
    r = fulls(ref)
    n1, n2 = r[0].shape
    dx, dy = d if d is not None else (p.get("lx", 1.0) / n1, p.get("ly", 1.0) / n2)
    F = FA.phys_flux(r, "x", eqn, p)
    Gf = FA.phys_flux(r, "y", eqn, p)
    return [float(np.linalg.norm(r[c]) + 2 * dt / dx * np.linalg.norm(F[c]) + 2 * dt / dy * np.linalg.norm(Gf[c]))
            for c in range(3)]


def check_fields(got, ref, bar, scales=None, what=""):
    """Assert ||got_c - ref_c|| <= bar * scale_c for every field (scale_c =
    ||ref_c||, or 1 where that is zero, unless ``scales`` are given) and
    return the per-field relative errors."""
    g, r = fulls(got), fulls(ref)
    errs = field_errors(g, r)
    for c in range(3):
        e = np.linalg.norm(g[c] - r[c])
        s = scales[c] if scales is not None else (np.linalg.norm(r[c]) or 1.0)
        assert e <= bar * s, (what, c, e, bar * s, errs)
    return errs
