"""tt_round_noalloc: rounding for callers that cannot allocate device memory.

Such callers (no cudaMalloc available to them, or a fixed device footprint)
get the same rounding as tt_round, with the scratch taken from an array the
library holds instead of a caller workspace.  Two calls in a row, through the
C ABI, must reproduce tt_round's output within the tolerance the rounding
parity tests use.  This file is collected last so a stop-at-first-failure run
has already run everything else; it also passes alone in a fresh process (the
first call on the device looks up the array's address).
"""
import ctypes

import numpy as np
import pytest

from synth import random_tt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api, capi
    return api, capi, capi.load()


def _noalloc_round(api, capi, lib, X, tol, cap, check_no_alloc=False):
    import torch
    x = api.DevTT.from_cores(X[0], X[1])
    y = api.DevTT(x.n1, x.n2, cap)
    xs, ys = x.struct(), y.struct()
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    err = ctypes.c_double(0.0)
    code = lib.tt_round_noalloc(ctypes.byref(xs), tol, cap, ctypes.byref(ys), ctypes.byref(err),
                                api._stream_ptr(None))
    capi.check("tt_round_noalloc", code)
    torch.cuda.synchronize()
    if check_no_alloc:
        # neither torch's allocator nor the driver saw an allocation
        assert (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]) == before
    y.rank = ys.rank
    return y, err.value


def test_noalloc_round_matches_tt_round_twice(env):
    api, capi, lib = env
    cases = [(random_tt(200, 300, 40, seed=21, decay=0.75), 1e-8, 32),
             (random_tt(256, 768, 24, seed=22, decay=0.7), 1e-10, 20)]
    for k, (X, tol, cap) in enumerate(cases):  # two calls in a row, different shapes
        ref, ref_err = api.tt_round(api.DevTT.from_cores(X[0], X[1]), tol, cap)
        # the first call may look up the array's address; the second is
        # checked to allocate nothing
        got, got_err = _noalloc_round(api, capi, lib, X, tol, cap, check_no_alloc=k > 0)
        assert got.rank == ref.rank
        a, b = got.full().numpy(), ref.full().numpy()
        assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)
        assert abs(got_err - ref_err) <= 1e-12 * np.linalg.norm(b) + 1e-6 * ref_err


def test_noalloc_rejects_oversized_problems(env):
    api, capi, lib = env
    big = api.DevTT(6000, 6000, 120, rank=120)
    y = api.DevTT(6000, 6000, 32)
    xs, ys = big.struct(), y.struct()
    code = lib.tt_round_noalloc(ctypes.byref(xs), 1e-8, 32, ctypes.byref(ys), None, api._stream_ptr(None))
    assert code == capi.TT_ERR_ARG
