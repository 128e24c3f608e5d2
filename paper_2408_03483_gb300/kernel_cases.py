"""Representative calls of the library's primitives at the 4096^2 workload's
shapes, for profiling single kernels (small device footprint, ~2 GB):

* factored-route roundings of a 4096 x 12288 TT with R = 49, 68 and 80
  columns (TSQR leaves and merges of both cores, the small SVD, the
  applications), the sizes of the Taylor and flux roundings;
* a Hadamard rounding of two rank-12 faces of that shape (Khatri-Rao cores
  and the range finder through them);
* the Upwind5 reconstruction of a rank-64 4096 x 4096 core pair;
* the split-operand TF32 and BF16 tensor-core contractions of a 4096 x 12288
  face tensor with a 72-column sketch.

    python -m paper_2408_03483_gb300.kernel_cases [repetitions]
"""
import sys

import numpy as np
import torch

from . import api, capi


def run(reps=3, seed=1):
    capi.load()
    rng = np.random.default_rng(seed)
    n1, n2 = 4096, 12288

    def tt(r, decay):
        A = rng.standard_normal((n1, r)) * (decay ** np.arange(r))[None, :]
        B = rng.standard_normal((n2, r))
        return api.DevTT.from_cores(A, B)
    X = tt(49, 0.7)
    X68, X80 = tt(68, 0.75), tt(80, 0.75)
    Z1, Z2 = tt(12, 0.5), tt(12, 0.5)
    C = api.DevTT.from_cores(rng.standard_normal((4096, 64)), rng.standard_normal((4096, 64)))
    W = torch.randn(n1, n2, dtype=torch.float64, device="cuda")
    Om = torch.randn(n2, 72, dtype=torch.float64, device="cuda")
    for _ in range(reps):
        api.tt_round(X, 1e-8, 64)
        api.tt_round(X68, 1e-8, 64)
        api.tt_round(X80, 1e-8, 64)
        api.tt_round_hadamard(Z1, Z2, 1e-8, 64)
        api.tt_recon_linear(C, 0, capi.TT_UP5)
        api.tt_contract(W, Om, precision="tf32", split=True)
        api.tt_contract(W, Om, precision="bf16", split=True)
    torch.cuda.synchronize()
    return torch.cuda.max_memory_allocated()


if __name__ == "__main__":
    peak = run(int(sys.argv[1]) if len(sys.argv) > 1 else 3)
    print(f"kernel cases done, peak device memory {peak / 1e9:.2f} GB")
