"""ctypes binding of libhelm.so (argument marshalling only).

Every name here mirrors a declaration in include/helm.h.  Loading fails loudly
when the in-tree library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# HELM_LIBRARY=checked loads the bounds-checked variant (built by build(checked=True))
LIB_PATH = os.path.join(HERE, "libhelm_checked.so" if os.environ.get("HELM_LIBRARY") == "checked" else "libhelm.so")

HELM_OK, HELM_BAD_ARG, HELM_NO_DEVICE, HELM_CUDA_ERROR = 0, 1, 2, 3
HELM_NOT_CONVERGED, HELM_DIVERGED, HELM_BREAKDOWN, HELM_SINGULAR_COARSE = 4, 5, 6, 7
HELM_NOT_READY, HELM_OUT_OF_MEMORY, HELM_SCRATCH_TOO_SMALL, HELM_TIMEOUT = 8, 9, 10, 11
STATUS_NAMES = {0: "ok", 1: "bad_arg", 2: "no_device", 3: "cuda_error", 4: "not_converged",
                5: "diverged", 6: "breakdown", 7: "singular_coarse", 8: "not_ready", 9: "out_of_memory",
                10: "scratch_too_small", 11: "timeout"}
HELM_C128, HELM_C64 = 0, 1
HELM_FP64, HELM_MIXED = 0, 1
HELM_RELAX_NONE, HELM_JACOBI, HELM_RBGS, HELM_SOR, HELM_SSOR, HELM_MG = 0, 1, 2, 3, 4, 5
HELM_CORR_NONE, HELM_CORR_TB, HELM_CORR_NONLINEAR = 0, 1, 2
HELM_METHOD_RELAX, HELM_METHOD_FGMRES, HELM_METHOD_BICGSTAB = 0, 1, 2
HELM_ACT_TANH = 0
HELM_ACT_LEAKY_RELU = 1


class SolveOpts(C.Structure):
    _fields_ = [("method", C.c_int), ("relax", C.c_int), ("n_r", C.c_int), ("omega", C.c_double),
                ("correction", C.c_int), ("tol", C.c_double), ("restart", C.c_int),
                ("maxit", C.c_int), ("conj", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("cycles", C.c_int),
                ("precond_applies", C.c_int), ("matvecs", C.c_int), ("rel_res", C.c_double),
                ("ms", C.c_double), ("launches", C.c_longlong), ("n_restrict", C.c_int),
                ("n_prolong", C.c_int), ("restrict_ms", C.c_double), ("prolong_ms", C.c_double),
                ("n_sweep", C.c_int), ("n_apply", C.c_int), ("sweep_ms", C.c_double), ("apply_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


vp, i32, f64, i64 = C.c_void_p, C.c_int, C.c_double, C.c_longlong
H = C.c_void_p

SIGNATURES = {
    "helm_create": (i32, [i32, i32, f64, i32, f64, vp, vp, i32, C.POINTER(H)]),
    "helm_create_bvp": (i32, [i32, i32, f64, vp, vp, i32, C.POINTER(H)]),
    "helm_destroy": (i32, [H]),
    "helm_set_stream": (i32, [H, vp]),
    "helm_last_error": (C.c_char_p, [H]),
    "helm_set_profiling": (i32, [H, i32]),
    "helm_set_wait_limit": (i32, [H, C.c_uint, C.c_uint]),
    "helm_set_reliable": (i32, [H, C.c_double, C.c_double, C.c_double]),
    "helm_checked_status": (i32, [C.POINTER(i32), C.POINTER(C.c_ulonglong)]),
    "helm_mg_setup": (i32, [H, i32]),
    "helm_info": (i32, [H, C.POINTER(i64), C.POINTER(f64)]),
    "helm_layer_k2": (i32, [H, vp, vp]),
    "helm_rhs": (i32, [H, vp, vp, vp]),
    "helm_apply": (i32, [H, vp, vp, i32, i32]),
    "helm_residual": (i32, [H, vp, vp, vp, vp, i32, i32]),
    "helm_relax": (i32, [H, i32, f64, i32, vp, vp, i32, i32]),
    "don_load": (i32, [H, vp, C.POINTER(i32), i32, i32, i32, f64]),
    "don_info": (i32, [H, C.POINTER(i32), C.POINTER(i32)]),
    "don_get_q": (i32, [H, vp]),
    "don_get_ainv": (i32, [H, vp]),
    "don_correct": (i32, [H, i32, vp, vp, i32, i32]),
    "helm_precond": (i32, [H, C.POINTER(SolveOpts), vp, vp]),
    "helm_solve": (i32, [H, C.POINTER(SolveOpts), vp, vp, C.POINTER(Stats), vp, i32]),
    "helm_solve_host": (i32, [H, C.POINTER(SolveOpts), vp, vp, C.POINTER(Stats), vp, i32]),
    "helm_residual_noalloc": (i32, [i32, i32, f64, i32, f64, vp, vp, vp, vp, vp, vp, i32, vp]),
    "helm_receivers_setup": (i32, [H, i32, vp, vp, vp]),
    "helm_receivers_sample": (i32, [H, i32, vp, vp, vp, vp]),
    "helm_receivers_adjoint": (i32, [H, i32, vp, vp, vp, vp]),
    "helm_k2_gradient": (i32, [H, vp, vp, vp]),
    "helm_set_k2": (i32, [H, vp]),
    "don_load_branch": (i32, [H, vp, C.POINTER(i32), i32]),
    "nn_gemm": (i32, [i32, i32, i32, i32, i32, C.c_float, vp, i32, vp, i32, C.c_float, vp, i32, vp]),
    "nn_gemm_bf16": (i32, [i32, i32, i32, i32, i32, C.c_float, vp, i32, vp, i32, C.c_float, vp, i32, vp]),
    "nn_gemm_bf16_status": (i32, [C.POINTER(i32)]),
    "nn_conv3d": (i32, [i32, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp]),
    "nn_conv3d_backward": (i32, [i32, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
    "nn_bias_act": (i32, [i32, i32, vp, vp, i32, vp]),
    "nn_act_backward": (i32, [i64, vp, vp, i32, vp]),
    "nn_bias_grad": (i32, [i32, i32, vp, vp, vp]),
    "nn_adam": (i32, [i64, vp, vp, vp, vp, C.c_float, C.c_float, C.c_float, C.c_float, i32, vp]),
    "nn_rel_l2": (i32, [i32, i32, vp, vp, vp, vp, vp]),
    "nn_gather": (i32, [i32, i32, vp, i64, vp, vp, vp, vp]),
    "helm_batch_create": (i32, [i32, C.POINTER(H), C.POINTER(H)]),
    "helm_batch_destroy": (i32, [H]),
    "helm_batch_set_tile": (i32, [H, i32, i32]),
    "helm_batch_solve": (i32, [H, C.POINTER(SolveOpts), C.POINTER(vp), C.POINTER(vp), C.POINTER(Stats)]),
    "helm_solve_concurrent": (i32, [i32, C.POINTER(H), C.POINTER(SolveOpts), C.POINTER(vp), C.POINTER(vp),
                                    C.POINTER(Stats), i32]),
}

_lib = None


def lib():
    """The loaded libhelm (raises if the in-tree build is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhelm.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib
