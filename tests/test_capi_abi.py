"""The C-ABI library builds, loads without a GPU, and exports every function
include/tt_fv.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared_functions():
    with open(os.path.join(ROOT, "include", "tt_fv.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(tt_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_03483_gb300 import build, capi
    if not os.path.exists(build.lib_path()):
        build.build()
    return capi.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("tt_fv_init", "tt_fv_step", "tt_fv_stage", "tt_round", "tt_cross", "tt_reciprocal"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2408_03483_gb300 import capi
    names = _declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    # the binding covers exactly the header
    assert sorted(capi.SIGNATURES) == names


def test_workspace_queries_without_gpu(lib):
    from paper_2408_03483_gb300 import capi
    assert lib.tt_round_workspace_size(256, 768, 64, 32) > 0
    assert lib.tt_round_workspace_size(0, 768, 64, 32) == 0
    p = capi.tt_fv_params(1, 2, 256, 256, 1.0, 1.0, 9.81, 1.0, 0.0, 4.7e-4, 1e-8, 32, 0, 0, 4, 10, 50, 0)
    assert lib.tt_fv_workspace_size(ctypes.byref(p)) > 0
    bad = capi.tt_fv_params(1, 2, 256, 256, 1.0, 1.0, 9.81, 1.0, 0.0, -1.0, 1e-8, 32, 0, 0, 4, 10, 50, 0)
    assert lib.tt_fv_workspace_size(ctypes.byref(bad)) == 0
    # the precision forms size their FP32 working copies on top of the FP64 cores
    for prec in (capi.TT_FP32, capi.TT_TF32, capi.TT_BF16):
        pp = capi.tt_fv_params(1, 1, 1024, 1024, 1.0, 1.0, 9.81, 1.0, 10.0, 1e-4, 1e-8, 48, prec, 0, 4, 10, 50, 0)
        assert lib.tt_fv_workspace_size(ctypes.byref(pp)) > 0
    pp = capi.tt_fv_params(1, 1, 1024, 1024, 1.0, 1.0, 9.81, 1.0, 10.0, 1e-4, 1e-8, 48, 7, 0, 4, 10, 50, 0)
    assert lib.tt_fv_workspace_size(ctypes.byref(pp)) == 0
    for prec in (capi.TT_FP64, capi.TT_FP32, capi.TT_TF32, capi.TT_BF16):
        for split in (0, 1):
            assert lib.tt_contract_workspace_size(prec, split, 1024, 112, 3072) > 0
    assert lib.tt_contract_workspace_size(9, 1, 1024, 112, 3072) == 0
    assert lib.tt_maxvol_workspace_size(12288, 13) > 0
    assert lib.tt_maxvol_workspace_size(8, 13) == 0 and lib.tt_maxvol_workspace_size(512, 129) == 0
    assert lib.tt_contract_workspace_size(capi.TT_TF32, 1, 0, 112, 3072) == 0


def test_reciprocal_workspace_covers_full_rank_products(lib):
    # Algorithm 1's second iteration multiplies a dy of full rank by x~: the
    # reciprocal's workspace must hold that rounding (the cap x cap product
    # of a stacked 256 x 768 face, which takes the range-finder route), not
    # only the first iteration's rank-1 product
    ws = lib.tt_reciprocal_workspace_size(256, 768, 13, 32)
    assert ws >= lib.tt_round_hadamard_workspace_size(256, 768, 32, 32, 32)
    assert lib.tt_reciprocal_workspace_size(256, 768, 0, 32) == 0


def test_stage_graph_sizing_is_deterministic(lib):
    # the nonlinear stage is sized by a serial dry run of its task graph
    # (every node on an arena of its own, one slice per worker): the same
    # parameters give the same bytes, and WENO5 needs more than Upwind3
    from paper_2408_03483_gb300 import capi
    w5 = capi.tt_fv_params(1, 2, 256, 256, 1.0, 1.0, 9.81, 1.0, 0.0, 4.7e-4, 1e-8, 32, 0, 0, 4, 10, 50, 0)
    u3 = capi.tt_fv_params(1, 0, 256, 256, 1.0, 1.0, 9.81, 1.0, 0.0, 4.7e-4, 1e-8, 32, 0, 0, 4, 10, 50, 0)
    a = lib.tt_fv_workspace_size(ctypes.byref(w5))
    assert a > 0 and a == lib.tt_fv_workspace_size(ctypes.byref(w5))
    assert a > lib.tt_fv_workspace_size(ctypes.byref(u3)) > 0


def test_argument_errors_return_codes(lib):
    from paper_2408_03483_gb300 import capi
    x = capi.tt2(0, 0, 0, 0, None, None)
    y = capi.tt2(0, 0, 0, 0, None, None)
    assert lib.tt_round(ctypes.byref(x), 1e-8, 4, ctypes.byref(y), None, None, 0, None) == capi.TT_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.tt_fv_init(None, None, None, 0, None, ctypes.byref(h)) == capi.TT_ERR_ARG
    assert lib.tt_fv_stage(None, 0) == capi.TT_ERR_ARG


def test_tile_shapes_without_gpu(lib):
    """The TSQR tile shapes the batched form's tuner chooses from: shape 0 is
    the default, and the solver workspace covers every shape (it is sized by
    the largest footprint over them)."""
    n = lib.tt_tile_shapes(None, None, 0)
    assert n >= 2
    lm = (ctypes.c_int32 * n)()
    fi = (ctypes.c_int32 * n)()
    assert lib.tt_tile_shapes(lm, fi, n) == n
    assert (lm[0], fi[0]) == (2, 0)
    assert len({(lm[i], fi[i]) for i in range(n)}) == n
    assert all(1 <= lm[i] <= 8 and (fi[i] == 0 or fi[i] >= 2) for i in range(n))
    assert lib.tt_fv_set_tile_shape(None, 0) != 0
