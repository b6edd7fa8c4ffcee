"""ctypes declarations of the C ABI in include/krr.h.

Loading fails loudly (ImportError-like RuntimeError) when lib/libkrr.so has not
been built: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libkrr.so")

KRR_MAX_RHS = 16
KRR_MAX_DIM = 64

STATUS = {
    0: "KRR_OK", 1: "KRR_E_INVAL", 2: "KRR_E_CUDA", 3: "KRR_E_NOTSPD", 4: "KRR_E_NOCONV",
    5: "KRR_E_STATE", 6: "KRR_E_NOMEM", 7: "KRR_E_NONFINITE", 8: "KRR_E_TIMEOUT",
}
KRR_OK, KRR_E_INVAL, KRR_E_CUDA, KRR_E_NOTSPD, KRR_E_NOCONV = 0, 1, 2, 3, 4
KRR_E_STATE, KRR_E_NOMEM, KRR_E_NONFINITE, KRR_E_TIMEOUT = 5, 6, 7, 8


class KrrOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("refine_max", C.c_int), ("oversample", C.c_int),
                ("check_every", C.c_int), ("inner_tol", C.c_double), ("anchor_rtol", C.c_double),
                ("precision", C.c_int), ("residual", C.c_int), ("pivot_tol", C.c_double),
                ("escalate", C.c_int), ("sparse_r", C.c_int), ("wait_limit_log2", C.c_int),
                ("test_stall_copies", C.c_int), ("no_precond", C.c_int), ("recurrence", C.c_int),
                ("strong_swaps", C.c_int), ("ex2_correct", C.c_int), ("tc_pv", C.c_int), ("autotune", C.c_int), ("tc_vfold", C.c_int), ("reserved", C.c_int * 1),
                ("strong_f", C.c_double)]


class KrrSolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("sweeps", C.c_int), ("k_eff", C.c_int),
                ("rel_residual", C.c_double * KRR_MAX_RHS), ("build_ms", C.c_double),
                ("solve_ms", C.c_double), ("mvm_count", C.c_int), ("sweep_iters", C.c_int * 8),
                ("sweep_residual", C.c_double * 8), ("product_form", C.c_int),
                ("restarts", C.c_int), ("recurrence64", C.c_int), ("lanczos_steps", C.c_int),
                ("reserved", C.c_int * 2), ("cond_estimate", C.c_double)]


_vp, _i, _ll, _d, _ull = C.c_void_p, C.c_int, C.c_longlong, C.c_double, C.c_ulonglong


class KrrProblem(C.Structure):
    _fields_ = [("X", C.c_void_p), ("n", C.c_longlong), ("d", C.c_int), ("Y", C.c_void_p),
                ("sigma", C.c_double), ("beta", C.c_double), ("k", C.c_int), ("alpha", C.c_void_p)]

# name -> (restype, argtypes)
SIGNATURES = {
    "krr_default_opts": (_i, [C.POINTER(KrrOpts)]),
    "krr_create": (_i, [C.POINTER(_vp), C.POINTER(KrrOpts), _vp]),
    "krr_destroy": (None, [_vp]),
    "krr_last_error": (C.c_char_p, [_vp]),
    "krr_launch_count": (_ll, [_vp]),
    "krr_profile_enable": (_i, [_vp, _i]),
    "krr_profile_read": (_i, [_vp, C.c_char_p, C.POINTER(_d), C.POINTER(_ll)]),
    "krr_peak_probe": (_i, [_i, C.POINTER(_d), _vp]),
    "krr_tc_selftest": (_i, [_i, C.POINTER(_i), C.POINTER(C.c_float), _vp]),
    "krr_exp2_probe": (_i, [_vp, _ll, _i, _vp, _vp]),
    "krr_strong_rrqr": (_i, [_vp, _vp, _ll, _i, _i, _d, _i, _vp, _vp, C.POINTER(_i), C.POINTER(_d)]),
    "krr_anchor_stats": (_i, [_vp, C.POINTER(_i), C.POINTER(_d)]),
    "krr_kmvm": (_i, [_vp, _vp, _ll, _vp, _ll, _i, _d, _d, _vp, _i, _vp]),
    "krr_residual_hp": (_i, [_vp, _vp, _ll, _i, _d, _d, _vp, _vp, _i, _vp]),
    "krr_residual_ff": (_i, [_vp, _vp, _ll, _i, _d, _d, _vp, _vp, _i, _vp]),
    "krr_omega": (_i, [_vp, _ull, _i, _ll, _vp]),
    "krr_sketch": (_i, [_vp, _vp, _ll, _i, _d, _i, _ull, _vp]),
    "krr_qrcp": (_i, [_vp, _vp, _ll, _i, _i, _vp, _vp]),
    "krr_sparse_draw": (_i, [_vp, _ull, _i, _i, _ll, _vp, _vp]),
    "krr_sparse_sketch": (_i, [_vp, _vp, _ll, _i, _d, _i, _i, _ull, _vp]),
    "krr_build_precond": (_i, [_vp, _vp, _ll, _i, _d, _d, _i, _ull]),
    "krr_build_precond_anchors": (_i, [_vp, _vp, _ll, _i, _d, _d, _vp, _i]),
    "krr_get_anchors": (_i, [_vp, _vp, C.POINTER(_i)]),
    "krr_precond_apply": (_i, [_vp, _vp, _i, _vp]),
    "krr_solve": (_i, [_vp, _vp, _vp, _i, _d, _vp, C.POINTER(KrrSolveInfo)]),
    "krr_predict": (_i, [_vp, _vp, _ll, _vp, _i, _vp]),
    "krr_batch_solve": (_i, [C.POINTER(KrrProblem), _i, _i, _d, _ull, C.POINTER(KrrOpts), _i,
                             C.POINTER(KrrSolveInfo), C.POINTER(_i)]),
    "krr_batch_solve_grouped": (_i, [C.POINTER(KrrProblem), _i, _i, _d, _ull, C.POINTER(KrrOpts), _i,
                                     C.POINTER(KrrSolveInfo), C.POINTER(_i)]),
    "krr_autotune": (_i, [_vp, _i, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_d)]),
    "krr_tune_save": (_i, [C.c_char_p]),
    "krr_tune_load": (_i, [C.c_char_p]),
    "krr_tune_get": (_i, [C.c_char_p, C.POINTER(_i), C.POINTER(_i), C.POINTER(_d)]),
    "krr_tune_set": (_i, [C.c_char_p, _i, _i, _d]),
    "krr_tune_clear": (_i, []),
    "krr_kmvm_dsigma": (_i, [_vp, _vp, _ll, _vp, _ll, _i, _d, _vp, _vp]),
    "krr_grad": (_i, [_vp, _vp, _vp, _ll, _vp, _d, C.POINTER(_d), C.POINTER(_d), C.POINTER(_d), _vp]),
    "krr_kmvm_noalloc": (_i, [_vp, _ll, _vp, _ll, _i, _d, _d, _vp, _i, _vp, _vp,
                              C.POINTER(C.c_ulonglong)]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libkrr.so once (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libkrr.so not found at {path}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols(path: str = LIB_PATH) -> list[str]:
    """The entry points this binding declares (all must resolve in the library)."""
    lib = load(path)
    return [n for n in SIGNATURES if hasattr(lib, n)]
