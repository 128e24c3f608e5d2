"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests
and the benchmark.

This package holds input generation only: cell-averaged initial conditions in
TT form (exact 1-D cell averages of separable functions), workload
parameters, and the closed-form inertia-gravity wave used by convergence
tests.  It contains none of the solver's arithmetic (no reconstruction, flux,
rounding, cross or reciprocal) and imports neither ``oracle`` nor the CUDA
package.
"""
from .ic import (  # noqa: F401
    WORKLOADS,
    workload,
    initial_tt,
    tt_to_full,
    random_tt,
    ensemble,
    igw_cellavg,
)
