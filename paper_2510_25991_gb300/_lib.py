"""ctypes declarations of the C ABI in ``include/ddst.h`` (argument marshalling only).

The library is the in-tree ``_build/libddst.so``; importing this module fails loudly when it
has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libddst.so")

# ddst_status
DDST_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "SINGULAR",
                5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "STATE", 8: "NOT_IMPLEMENTED"}
DDST_FP64 = 0
DDST_MIXED = 1
DDST_AUTO = 2
DDST_MIXED_TF32 = 3


class ddst_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64)]


class ddst_coeffs(C.Structure):
    _fields_ = [("a", C.c_void_p), ("b", C.c_double * 3), ("c", C.c_void_p)]


class ddst_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("gmres_tol", C.c_double), ("gmres_max_iter", C.c_int),
                ("refine_tol", C.c_double), ("refine_max", C.c_int), ("k_max", C.c_int),
                ("oversample", C.c_int), ("leaf_size", C.c_int), ("seed", C.c_uint64),
                ("check_every", C.c_int), ("factor_chunks", C.c_int), ("factor_warmup", C.c_int),
                ("tensor_cores", C.c_int), ("explicit_S", C.c_int),
                ("recompute_factors", C.c_int), ("autotune_cache", C.c_char_p),
                ("interface_solver", C.c_int)]


class ddst_info(C.Structure):
    _fields_ = [("gmres_iters", C.c_int), ("gmres_iters_first", C.c_int),
                ("refine_iters", C.c_int), ("rel_residual", C.c_double),
                ("est_rel_error", C.c_double), ("t_factor", C.c_double),
                ("t_transfer", C.c_double), ("t_compress", C.c_double), ("t_solve", C.c_double),
                ("bytes_factors", C.c_int64), ("bytes_transfer", C.c_int64),
                ("max_rank", C.c_int), ("fail_slab", C.c_int), ("fail_block", C.c_int),
                ("factor_chunks", C.c_int), ("factor_check", C.c_double),
                ("t_direct", C.c_double), ("refine_rho", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ddst_tune_report(C.Structure):
    _fields_ = [("chosen", ddst_options), ("candidates", C.c_int), ("rejected", C.c_int),
                ("default_ms", C.c_double), ("best_ms", C.c_double), ("best_rho", C.c_double),
                ("cache_written", C.c_int)]


_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)

SIGNATURES = {
    "ddst_options_default": (None, [C.POINTER(ddst_options)]),
    "ddst_setup": (C.c_int, [C.POINTER(ddst_grid), C.POINTER(ddst_coeffs), C.c_int,
                             C.POINTER(ddst_options), _P, C.POINTER(_P)]),
    "ddst_setup_batch": (C.c_int, [C.c_int, C.POINTER(ddst_grid), C.POINTER(ddst_coeffs),
                                   C.POINTER(C.c_int), C.POINTER(ddst_options), _P,
                                   C.POINTER(_P)]),
    "ddst_build_transfer": (C.c_int, [_P]),
    "ddst_compress": (C.c_int, [_P, C.c_double]),
    "ddst_compress_hbs": (C.c_int, [_P, C.c_int, C.c_int]),
    "ddst_hbs_create": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int,
                                  C.POINTER(_P)]),
    "ddst_hbs_apply": (C.c_int, [_P, _P, _P, C.c_int]),
    "ddst_hbs_expand": (C.c_int, [_P, _P]),
    "ddst_hbs_stats": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "ddst_hbs_destroy": (None, [_P]),
    "ddst_solve": (C.c_int, [_P, _P, _P, _P, C.POINTER(ddst_info)]),
    "ddst_solve_batch": (C.c_int, [_P, _PP, _PP, _PP, C.POINTER(ddst_info)]),
    "ddst_march": (C.c_int, [_P, C.c_int, C.c_double, _PP, _PP, _PP, C.POINTER(ddst_info)]),
    "ddst_solve_adjoint": (C.c_int, [_P, _P, _P, _P, _P, C.POINTER(ddst_info)]),
    "ddst_solve_adjoint_batch": (C.c_int, [_P, _PP, _PP, _PP, _PP, C.POINTER(ddst_info)]),
    "ddst_interface_trace": (C.c_int, [_P, C.c_int, _P]),
    "ddst_get_transfer": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P]),
    "ddst_apply_interface": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "ddst_time_apply": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_float)]),
    "ddst_solve_interface": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "ddst_query": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64),
                             C.POINTER(C.c_int)]),
    "ddst_get_precision": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "ddst_residual_noalloc": (C.c_int, [C.POINTER(ddst_grid), C.POINTER(ddst_coeffs), _P, _P, _P,
                                        _P, _P, _P]),
    "ddst_kernel_launches": (C.c_int64, []),
    "ddst_autotune": (C.c_int, [C.c_int, C.POINTER(ddst_grid), C.POINTER(ddst_coeffs),
                                C.POINTER(C.c_int), _PP, _PP, C.c_double, C.c_int,
                                C.POINTER(ddst_options), _P, C.POINTER(ddst_tune_report)]),
    "ddst_autotune_key": (C.c_int, [C.c_int, C.POINTER(ddst_grid), C.POINTER(ddst_coeffs),
                                    C.POINTER(C.c_int), C.c_int, C.c_char_p, C.c_size_t]),
    "ddst_autotune_lookup": (C.c_int, [C.c_char_p, C.c_char_p, C.POINTER(ddst_options),
                                       C.POINTER(C.c_int)]),
    "ddst_autotune_store": (C.c_int, [C.c_char_p, C.c_char_p, C.POINTER(ddst_options)]),
    "ddst_get_options": (C.c_int, [_P, C.POINTER(ddst_options)]),
    "ddst_partition": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int),
                                 C.POINTER(C.c_double)]),
    "ddst_last_error": (C.c_char_p, [_P]),
    "ddst_destroy": (None, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library and attach the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
