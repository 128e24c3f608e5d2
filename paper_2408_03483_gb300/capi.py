"""ctypes binding of the C ABI declared in include/tt_fv.h.

Argument marshalling only: every step of the TT finite-volume stage runs in
libttfv.so.  PyTorch supplies device memory (cores, workspaces) and streams.
There is no CPU fallback: importing this module without the built library, or
calling it without a CUDA device, raises.
"""
import ctypes
import os

from . import build as _build

TT_OK, TT_ERR_ARG, TT_ERR_OOM, TT_ERR_CUDA, TT_ERR_NOCONV, TT_ERR_TIMEOUT, TT_ERR_RANKCAP, TT_ERR_NONFINITE = range(8)
TT_LINEAR, TT_NONLINEAR = 0, 1
TT_UP3, TT_UP5, TT_WENO5 = 0, 1, 2
TT_FP64, TT_TF32, TT_BF16, TT_FP32 = 0, 1, 2, 3
TT_PIVOT_MAXVOL, TT_PIVOT_LEARNED = 0, 1
TT_FN_ENTRY, TT_FN_WENO_S1, TT_FN_WENO_S2, TT_FN_LLF_LAMBDA, TT_FN_LLF_FLUX = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "TT_OK", 1: "TT_ERR_ARG", 2: "TT_ERR_OOM", 3: "TT_ERR_CUDA", 4: "TT_ERR_NOCONV",
                5: "TT_ERR_TIMEOUT", 6: "TT_ERR_RANKCAP",
                7: "TT_ERR_NONFINITE"}

SCHEMES = {"up3": TT_UP3, "up5": TT_UP5, "weno5": TT_WENO5}
EQNS = {"linear": TT_LINEAR, "nonlinear": TT_NONLINEAR}
PRECISIONS = {"fp64": TT_FP64, "fp32": TT_FP32, "tf32": TT_TF32, "bf16": TT_BF16}
PIVOTS = {"maxvol": 0, "learned": 1}
EPS_RULES = {"fixed": 0, "adaptive": 1}
FLUXES = {"products": 0, "cross": 1}
BCS = {"periodic": 0, "exact": 1}


class TTError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {STATUS_NAMES.get(code, code)}")
        self.code = code


class tt2(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int32), ("n2", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("cap", ctypes.c_int32), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p)]


class tt_fv_params(ctypes.Structure):
    _fields_ = [("eqn", ctypes.c_int32), ("recon", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("g", ctypes.c_double), ("H", ctypes.c_double), ("f", ctypes.c_double),
                ("dt", ctypes.c_double), ("tol", ctypes.c_double), ("rank_cap", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("pivots", ctypes.c_int32), ("kick", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("seed", ctypes.c_uint32),
                ("eps_rule", ctypes.c_int32), ("c_eps", ctypes.c_double), ("flux", ctypes.c_int32),
                ("forcing_waves", ctypes.c_int32), ("bc_x", ctypes.c_int32), ("boundary_waves", ctypes.c_int32)]


class tt_wave(ctypes.Structure):
    _fields_ = [("field", ctypes.c_int32), ("amp", ctypes.c_double), ("kx", ctypes.c_double),
                ("ky", ctypes.c_double), ("omega", ctypes.c_double), ("phase", ctypes.c_double),
                ("decay", ctypes.c_double)]


class tt_fv_stats(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32 * 3), ("rounds", ctypes.c_int64), ("syncs", ctypes.c_int64),
                ("jacobi_sweeps", ctypes.c_int64), ("cross_calls", ctypes.c_int64),
                ("cross_sweeps", ctypes.c_int64), ("taylor_iters", ctypes.c_int64),
                ("cap_hits", ctypes.c_int64), ("qb_attempts", ctypes.c_int64),
                ("qb_uncertified", ctypes.c_int64), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("device_status", ctypes.c_uint32),
                ("svd_calls", ctypes.c_int64), ("svd_p_sum", ctypes.c_int64), ("svd_pd_sum", ctypes.c_int64),
                ("svd_sweeps_sum", ctypes.c_int64), ("section_ms", ctypes.c_double * 6),
                ("learned_calls", ctypes.c_int64), ("learned_accepted", ctypes.c_int64),
                ("eps_u", ctypes.c_double * 3), ("eps_tt", ctypes.c_double)]


TT_K_NAMES = ["gemm", "form_hadamard", "qr", "qr_apply", "jacobi_svd", "maxvol", "cross_eval", "stencil",
              "other", "qr_merge", "qr_apply_merge"]


class tt_mlp(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]


class tt_kernel_prof(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double),
                ("launches", ctypes.c_int64)]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i32 = ctypes.c_int32
_d = ctypes.c_double

# name -> (restype, argtypes); the list mirrors include/tt_fv.h
SIGNATURES = {
    "tt_fv_version": (ctypes.c_char_p, []),
    "tt_fv_workspace_size": (_sz, [_P(tt_fv_params)]),
    "tt_fv_init": (ctypes.c_int, [_P(tt_fv_params), _P(tt2), _vp, _sz, _vp, _P(_vp)]),
    "tt_fv_step": (ctypes.c_int, [_vp, _i32]),
    "tt_fv_stage": (ctypes.c_int, [_vp, _i32]),
    "tt_fv_get": (ctypes.c_int, [_vp, _P(tt2)]),
    "tt_fv_set": (ctypes.c_int, [_vp, _P(tt2)]),
    "tt_fv_set_forcing": (ctypes.c_int, [_vp, _P(tt_wave), _i32, _d]),
    "tt_fv_set_boundary": (ctypes.c_int, [_vp, _P(tt_wave), _i32, _d]),
    "tt_fv_stats_get": (ctypes.c_int, [_vp, _P(tt_fv_stats)]),
    "tt_fv_destroy": (None, [_vp]),
    "tt_tile_shapes": (_i32, [_P(_i32), _P(_i32), _i32]),
    "tt_fv_set_tile_shape": (ctypes.c_int, [_vp, _i32]),
    "tt_fv_profile": (ctypes.c_int, [_vp, _i32]),
    "tt_fv_kernel_profile": (ctypes.c_int, [_vp, _P(tt_kernel_prof), _i32]),
    "tt_launch_count": (ctypes.c_uint64, []),
    "tt_round_workspace_size": (_sz, [_i32, _i32, _i32, _i32]),
    "tt_round": (ctypes.c_int, [_P(tt2), _d, _i32, _P(tt2), _P(_d), _vp, _sz, _vp]),
    "tt_mlp_workspace_size": (_sz, [_i32, _i32]),
    "tt_mlp_features": (ctypes.c_int, [_P(tt2), _vp, _i32, _vp, _vp, _sz, _vp]),
    "tt_mlp_forward": (ctypes.c_int, [_P(tt_mlp), _vp, _i32, _vp, _vp, _sz, _vp]),
    "tt_mlp_grad": (ctypes.c_int, [_P(tt_mlp), _vp, _vp, _i32, _P(tt_mlp), _vp, _vp, _sz, _vp]),
    "tt_mlp_adam": (ctypes.c_int, [_P(tt_mlp), _P(tt_mlp), _P(tt_mlp), _P(tt_mlp), _i32, ctypes.c_float, _vp]),
    "tt_mlp_topk": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _sz, _vp]),
    "tt_fv_set_pivot_net": (ctypes.c_int, [_vp, _P(tt_mlp)]),
    "tt_fv_record_pivots": (ctypes.c_int, [_vp, _i32]),
    "tt_fv_pivot_rows": (ctypes.c_int64, [_vp]),
    "tt_fv_pivot_take": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64]),
    "tt_fv_batch_workspace_size": (_sz, [_P(tt_fv_params), _i32]),
    "tt_fv_batch_init": (ctypes.c_int, [_P(tt_fv_params), _i32, _P(tt2), _vp, _sz, _vp, _P(_vp)]),
    "tt_fv_batch_configure": (ctypes.c_int, [_vp, _i32, _i32]),
    "tt_fv_batch_step": (ctypes.c_int, [_vp, _i32]),
    "tt_fv_batch_tune": (ctypes.c_int, [_vp, _P(_i32), _i32, _i32, _P(_i32), _P(_i32), _P(_d)]),
    "tt_fv_batch_tune_tiles": (ctypes.c_int, [_vp, _i32, _i32, _P(_i32), _P(_d)]),
    "tt_fv_batch_get": (ctypes.c_int, [_vp, _i32, _P(tt2)]),
    "tt_fv_batch_stats_get": (ctypes.c_int, [_vp, _i32, _P(tt_fv_stats)]),
    "tt_fv_batch_destroy": (None, [_vp]),
    "tt_contract_workspace_size": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "tt_contract": (ctypes.c_int, [_i32, _i32, _i32, _i32, _i32, _d, _vp, ctypes.c_int64, _vp, ctypes.c_int64, _d,
                                   _vp, ctypes.c_int64, _vp, _sz, _vp]),
    "tt_round_noalloc": (ctypes.c_int, [_P(tt2), _d, _i32, _P(tt2), _P(_d), _vp]),
    "tt_round_hadamard_workspace_size": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "tt_round_hadamard": (ctypes.c_int, [_P(tt2), _P(tt2), _d, _i32, _P(tt2), _vp, _sz, _vp]),
    "tt_cross_workspace_size": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "tt_cross": (ctypes.c_int, [_i32, _P(tt2), _i32, _P(tt2), _P(_d), _d, _i32, _i32, _i32, ctypes.c_uint32,
                                _P(tt2), _P(_i32), _vp, _sz, _vp]),
    "tt_maxvol_workspace_size": (_sz, [_i32, _i32]),
    "tt_maxvol": (ctypes.c_int, [_vp, _i32, _i32, _d, _i32, _vp, _vp, _sz, _vp]),
    "tt_reciprocal_workspace_size": (_sz, [_i32, _i32, _i32, _i32]),
    "tt_reciprocal": (ctypes.c_int, [_P(tt2), _d, _i32, _i32, _P(tt2), _P(_i32), _vp, _sz, _vp]),
    "tt_recon_linear": (ctypes.c_int, [_P(tt2), _i32, _i32, _P(tt2), _P(tt2), _vp]),
}

_lib = None


def lib_path():
    return _build.lib_path()


def load(path=None):
    """Load libttfv.so (built by paper_2408_03483_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    import torch  # noqa: F401  (loads the CUDA runtime the library shares)
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(name, code):
    if code != TT_OK:
        raise TTError(name, code)
