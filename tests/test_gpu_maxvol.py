"""Maximum-volume rows (Sec. 3.3, the pivot choice of the cross sweeps)
through tt_maxvol: the rows it returns satisfy the maxvol bound |U U[I]^-1|
<= 1 + delta (checked in FP64 on the host), and the cluster kernel (rows
spread over up to 8 CTAs) makes exactly the choices of the single-CTA kernel
(TT_MAXVOL_CLUSTER=0, run in a child process since the switch is read once).
Several index sets can satisfy the bound, so the test checks validity and
agreement of the two kernels, not one particular set."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

# (n, r, seed): clusters of 8 (12288 x 13, 4096 x 20), 4 (2048 x 12), 1
# (300 x 7), and a shape that only the single-CTA kernel holds (12288 x 40)
CASES = [(12288, 13, 1), (4096, 20, 2), (2048, 12, 3), (300, 7, 4), (12288, 40, 5)]


def _matrix(n, r, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, r))
    # rows of very different scales: partial pivoting alone is then far
    # from maximal volume, so the swap phase has work to do
    U *= np.exp(rng.uniform(-2.0, 2.0, size=(n, 1)))
    return U


def _indices(cases):
    import torch
    from paper_2408_03483_gb300 import api
    out = []
    for n, r, seed in cases:
        U = torch.tensor(_matrix(n, r, seed), dtype=torch.float64, device="cuda")
        out.append(api.tt_maxvol(U, delta=1e-2, max_iter=200).cpu().numpy().tolist())
    return out


def _child(env_value):
    code = ("import json, sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_gpu_maxvol as t; print(json.dumps(t._indices(t.CASES)))"
            % (ROOT, os.path.join(ROOT, "tests")))
    env = dict(os.environ, TT_MAXVOL_CLUSTER=env_value)
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def test_maxvol_bound_holds():
    got = _indices(CASES)
    for (n, r, seed), I in zip(CASES, got):
        I = np.asarray(I)
        assert len(set(I.tolist())) == r and I.min() >= 0 and I.max() < n, (n, r)
        U = _matrix(n, r, seed)
        B = np.linalg.solve(U[I].T, U.T).T  # U U[I]^-1
        # the swaps compare FP32 values against 1 + delta
        assert np.abs(B).max() <= 1.0 + 1e-2 + 1e-4, (n, r, np.abs(B).max())
        assert np.allclose(B[I], np.eye(r), atol=1e-10)


def test_cluster_kernel_matches_single_cta_kernel():
    clustered = _child("1")
    single = _child("0")
    assert clustered == single
