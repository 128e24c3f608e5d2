"""The C form of Oracle A (oracle/fv_full.c) against the numpy form (pinned by
tests/test_oracle_fv.py and tests/test_oracle_flux.py): same discretisation,
so the same states up to round-off, for every scheme, both equations, with
rotation, on non-square grids; and its own pins (IGW convergence order,
mass conservation) so that it stands on its own."""
import math

import numpy as np
import pytest

from oracle import fv_c as FC
from oracle import fv_full as FA
from synth import igw_cellavg, initial_tt, tt_to_full, workload


@pytest.mark.parametrize("scheme", ["up3", "up5", "weno5"])
@pytest.mark.parametrize("eqn", ["linear", "nonlinear"])
def test_c_oracle_matches_numpy_oracle(scheme, eqn):
    rng = np.random.default_rng(7)
    nx, ny = 24, 20
    p = dict(g=9.81, H=1.0, f=2.5, lx=1.2, ly=1.0)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    base = np.exp(-((x[:, None] - 0.4) ** 2 + (y[None, :] - 0.6) ** 2) / 0.05)
    if eqn == "nonlinear":
        Q = [1.0 + 0.1 * base, 0.02 * base + 0.01 * rng.standard_normal((nx, ny)), -0.03 * base]
    else:
        Q = [0.05 * base, 0.01 * rng.standard_normal((nx, ny)), 0.02 * base]
    dt = 1e-3
    a = Q
    for _ in range(3):
        a = FA.ssprk3_step(a, eqn, scheme, p, dt)
    b = FC.ssprk3_steps(Q, eqn, scheme, p, dt, 3)
    for c in range(3):
        assert np.linalg.norm(a[c] - b[c]) <= 1e-13 * max(np.linalg.norm(a[c]), 1e-300), (scheme, eqn, c)


def test_c_oracle_igw_convergence_and_mass():
    # formal order 5 of Upwind5 on the inertia-gravity wave (Sec. 5.2)
    def err(n, T=0.02):
        p = dict(g=9.81, H=1.0, f=1.0, lx=1.0, ly=1.0)
        dx = 1.0 / n
        dt0 = 0.4 * (1.0 / 16) * (16 * dx) ** (5.0 / 3.0) / math.sqrt(9.81)
        nst = int(math.ceil(T / dt0))
        Q = FC.ssprk3_steps(igw_cellavg(n, 0.0), "linear", "up5", p, T / nst, nst)
        ex = igw_cellavg(n, T)
        return np.linalg.norm(Q[0] - ex[0]) / np.linalg.norm(ex[0])
    e = [err(n) for n in (32, 64)]
    assert 4.6 < math.log2(e[0] / e[1]) < 5.5
    w = workload("nonlinear256_weno5", n=48)
    Qt, p = initial_tt(w)
    Q = [tt_to_full(*q) for q in Qt]
    R = FC.ssprk3_steps(Q, "nonlinear", "weno5", p, p["dt"], 4)
    assert abs(R[0].sum() - Q[0].sum()) <= 1e-13 * Q[0].sum()
