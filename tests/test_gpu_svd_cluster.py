"""The small SVD of the rounding (Sec. 3.2: the SVD of R_A R_B^T) with its
FP64 Jacobi sweeps spread over a thread-block cluster: each CTA takes a
share of every round's column pairs and writes the columns it rotates into
the others' shared memory, so every pair sees the same inputs as in one CTA
and the rounded TT must be bit-identical to the single-CTA kernel's
(TT_SVD_CLUSTER=1), whatever the cluster size (2, 4, 8).  Each size runs in
a child process, since the switch is read once.  The rounded TTs also match
the plain truncated SVD of the full tensor (Eckart-Young) within the
rounding tolerance."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

# (R, decay, seed): R columns of graded scale; 48 and up take the cluster
CASES = [(24, 0.7, 1), (48, 0.7, 2), (64, 0.75, 3), (80, 0.8, 4), (112, 0.85, 5)]
N1, N2 = 700, 1300


def _cores(R, decay, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N1, R)) * (decay ** np.arange(R))[None, :]
    B = rng.standard_normal((N2, R))
    return A, B


def _rounded(cases):
    from paper_2408_03483_gb300 import api
    out = []
    for R, decay, seed in cases:
        A, B = _cores(R, decay, seed)
        y, _ = api.tt_round(api.DevTT.from_cores(A, B), 1e-8, 64)
        a = y.a[:y.rank].cpu().numpy()
        b = y.b[:y.rank].cpu().numpy()
        out.append([y.rank, hashlib.sha256(a.tobytes() + b.tobytes()).hexdigest()])
    return out


def _child(env_value):
    code = ("import json, sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_gpu_svd_cluster as t; print(json.dumps(t._rounded(t.CASES)))"
            % (ROOT, os.path.join(ROOT, "tests")))
    env = dict(os.environ, TT_SVD_CLUSTER=env_value)
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def test_cluster_svd_is_bitwise_the_single_cta_svd():
    single = _child("1")
    for size in ("2", "4", "8"):
        assert _child(size) == single, size


def test_rounding_with_the_cluster_svd_is_a_truncated_svd():
    from paper_2408_03483_gb300 import api
    for R, decay, seed in CASES:
        A, B = _cores(R, decay, seed)
        y, _ = api.tt_round(api.DevTT.from_cores(A, B), 1e-8, 64)
        X = A @ B.T
        s = np.linalg.svd(X, compute_uv=False)
        got = y.full().numpy()
        err = np.linalg.norm(got - X)
        nx = np.linalg.norm(X)
        # the kept rank meets the tolerance (or the cap) and the error is
        # the optimal tail of that rank up to round-off
        assert err <= max(1e-8 * nx, np.sqrt(np.sum(s[y.rank:] ** 2))) * (1 + 1e-6) + 1e-12 * nx, (R, y.rank)
        assert abs(err - np.sqrt(np.sum(s[y.rank:] ** 2))) <= 1e-10 * nx, (R, y.rank)
