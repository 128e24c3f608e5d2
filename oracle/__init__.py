"""FP64 CPU oracle for the tensor-train finite-volume shallow-water stage.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path and never imports the package
``paper_2408_03483_gb300``.

Two oracles live here (Danis et al., arXiv 2408.03483):

* Oracle A (``fv_full``): the plain full-tensor finite-volume discretisation of
  Sec. 2 -- dimension-by-dimension reconstruction (Sec. 2.3), LLF flux with
  Gauss-Legendre face quadrature (Sec. 2.2, Sec. 2.4), SSP-RK3 (Sec. 4.4).
* Oracle B (``tt``, ``cross``, ``recip``, ``tt_fv``): the paper's TT algorithm
  step by step -- TT rounding (Sec. 3.2), maxvol cross (Sec. 3.3),
  Taylor reciprocal (Algorithm 1), TT reconstruction (Sec. 4.3, Algorithms 2-3),
  TT fluxes (Eq. LLF-TT), TT SSP-RK3 (Eq. tt-ssprk3).

Everything is float64 numpy; library primitives (QR, SVD, solve) serve as
single steps only.

Parity pins: see ``tests/test_oracle_*.py``.  Functions whose result is not
unique (cross pivot sets, exact cross ranks) are "parity unpinned" for those
outputs; their approximation error is pinned instead.
"""
