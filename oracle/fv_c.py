"""Oracle A in plain C (fv_full.c): the full-tensor finite volume of Sec. 2,
for long runs (hundreds of steps) and large grids.

Oracle code (test infrastructure only): built by ``build()`` with gcc and
OpenMP into oracle/lib/, loaded with ctypes.  The coefficient tables are the
exact ones of coeffs.py, so the C and numpy forms of Oracle A compute the
same discretisation; tests/test_oracle_fv_c.py pins the C form to the numpy
form (itself pinned by convergence, conservation and steady states).
"""
import ctypes
import os
import subprocess

import numpy as np

from . import coeffs

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fv_full.c")
LIB = os.path.join(HERE, "lib", "libfvfull.so")


class FvCoeffs(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int), ("weno", ctypes.c_int), ("lin1", (ctypes.c_double * 5) * 2),
                ("C", ((ctypes.c_double * 3) * 3) * 3), ("gam", (ctypes.c_double * 3) * 3),
                ("split", ctypes.c_int * 3), ("gp", ctypes.c_double * 3), ("gm", ctypes.c_double * 3),
                ("sp", ctypes.c_double), ("sm", ctypes.c_double), ("w", ctypes.c_double * 3)]


class FvGrid(ctypes.Structure):
    _fields_ = [("eqn", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("g", ctypes.c_double), ("H", ctypes.c_double), ("f", ctypes.c_double)]


def build(force=False):
    """Compile fv_full.c into oracle/lib/libfvfull.so (if missing or older than
    the source); returns the library path."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", tmp,
                               "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.fv_ssprk3_steps.argtypes = [ctypes.POINTER(FvGrid), ctypes.POINTER(FvCoeffs)] + \
            [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int]
        lib.fv_ssprk3_steps.restype = ctypes.c_int
        _lib = lib
    return _lib


def make_coeffs(scheme):
    """The tables of coeffs.py for one reconstruction scheme."""
    nq = 2 if scheme == "up3" else 3
    k = nq - 1
    co = FvCoeffs()
    co.nq = nq
    co.weno = 1 if scheme == "weno5" else 0
    if scheme != "weno5":
        order = 3 if scheme == "up3" else 5
        for side, sd in ((0, "-"), (1, "+")):
            st = coeffs.step1_linear(order, sd)
            for s in range(-2, 3):
                co.lin1[side][s + 2] = float(st.get(s, 0))
    Cs = coeffs.step2_C(nq)
    gam = coeffs.step2_gamma(nq)
    for m in range(nq):
        for r in range(k + 1):
            for l in range(k + 1):
                co.C[m][r][l] = float(Cs[m][r, l])
        if gam[m] is None:
            co.split[m] = 1
        else:
            for r in range(k + 1):
                co.gam[m][r] = float(gam[m][r])
    gp, gm, sp, sm = coeffs.step2_split()
    for r in range(3):
        co.gp[r], co.gm[r] = float(gp[r]), float(gm[r])
    co.sp, co.sm = float(sp), float(sm)
    _, w = coeffs.gauss_legendre(nq)
    for m in range(nq):
        co.w[m] = float(w[m])
    return co


def ssprk3_steps(Q, eqn, scheme, p, dt, nsteps):
    """Q (three nx x ny float64 arrays) advanced nsteps SSP-RK3 steps; returns
    new arrays."""
    lib = load()
    out = [np.ascontiguousarray(q, dtype=np.float64).copy() for q in Q]
    nx, ny = out[0].shape
    G = FvGrid(0 if eqn == "linear" else 1, nx, ny, p["lx"] / nx, p["ly"] / ny, p["g"], p.get("H", 1.0),
               p.get("f", 0.0))
    co = make_coeffs(scheme)
    rc = lib.fv_ssprk3_steps(ctypes.byref(G), ctypes.byref(co), *[q.ctypes.data for q in out], float(dt),
                             int(nsteps))
    if rc != 0:
        raise MemoryError("fv_ssprk3_steps: scratch allocation failed")
    return out
