"""ctypes declarations of the C ABI in include/sgn.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsgn.so")

SGN_OK = 0
STATUS = {0: "SGN_OK", 1: "SGN_ERR_ARG", 2: "SGN_ERR_CUDA", 3: "SGN_ERR_NOT_CONVERGED", 4: "SGN_ERR_BREAKDOWN",
          5: "SGN_ERR_DEFLATION", 6: "SGN_ERR_NONFINITE", 7: "SGN_ERR_TIMEOUT", 8: "SGN_ERR_STATE",
          9: "SGN_ERR_ALLOC"}
PREC_FP64, PREC_MIXED = 0, 1
LINKS_FP32, LINKS_BF16, LINKS_FP16 = 0, 1, 2
APPLY_HOST_BUFFERS, APPLY_ADJOINT, APPLY_NO_A = 1, 2, 4
HW_ADJOINT, HW_PACKED, HW_FLOAT_FLOAT = 1, 2, 4
FORM_A2, FORM_A = 0, 1
METHOD_FOM, METHOD_GMRES = 0, 1

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Report(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("matvecs", C.c_int), ("refine_rounds", C.c_int),
                ("refine_cycles", C.c_int), ("breakdown", C.c_int), ("res_est", C.c_double),
                ("err_est", C.c_double), ("ms", C.c_double),
                ("kernels", C.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes); every symbol include/sgn.h declares
P = C.c_void_p
SIGNATURES = {
    "sgn_create": (C.c_int, [C.POINTER(P), C.POINTER(C.c_int), ALLOC_FN, FREE_FN, P, P]),
    "sgn_destroy": (C.c_int, [P]),
    "sgn_set_stream": (C.c_int, [P, P]),
    "sgn_load_gauge": (C.c_int, [P, P, C.c_int]),
    "sgn_set_mu": (C.c_int, [P, C.c_double]),
    "sgn_set_kernel_mass": (C.c_int, [P, C.c_double]),
    "sgn_set_boundary": (C.c_int, [P, C.POINTER(C.c_int)]),
    "sgn_kenney_laub": (C.c_int, [C.c_int, C.c_double, P, P]),
    "sgn_set_rational": (C.c_int, [P, C.c_int, P, P]),
    "sgn_set_restart": (C.c_int, [P, C.c_int, C.c_double, C.c_int, C.c_int]),
    "sgn_set_precision": (C.c_int, [P, C.c_int, C.c_double, C.c_int]),
    "sgn_set_refinement": (C.c_int, [P, C.c_int, C.c_int]),
    "sgn_set_formulation": (C.c_int, [P, C.c_int]),
    "sgn_set_method": (C.c_int, [P, C.c_int]),
    "sgn_set_deflation": (C.c_int, [P, C.c_int, P, P, P, C.c_int]),
    "sgn_set_deflation_extra": (C.c_int, [P, C.c_int, P, P, P, C.c_int]),
    "sgn_build_deflation": (C.c_int, [P, C.c_int, C.c_int, C.c_double, P]),
    "sgn_get_deflation": (C.c_int, [P, C.POINTER(C.c_int), P, P, P]),
    "sgn_apply": (C.c_int, [P, P, P, C.c_int, C.c_int, C.POINTER(Report)]),
    "sgn_apply_shifts": (C.c_int, [P, P, P, P, C.c_int, C.c_int, C.POINTER(Report)]),
    "sgn_hw_apply": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_int]),
    "sgn_apply_direct": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "sgn_overlap_apply": (C.c_int, [P, P, P, C.c_int]),
    "sgn_overlap_solve": (C.c_int, [P, P, P, C.c_int, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_double)]),
    "sgn_pack_fields": (C.c_int, [P, P, P, C.c_int, C.c_int]),
    "sgn_unpack_fields": (C.c_int, [P, P, P, C.c_int, C.c_int]),
    "sgn_inner_products": (C.c_int, [P, P, C.c_int, P, C.c_int, P]),
    "sgn_inner_products_noalloc": (C.c_int, [P, C.c_int, P, C.c_longlong, C.c_int, P, P]),
    "sgn_dhw_dmu_apply": (C.c_int, [P, P, P, C.c_int]),
    "sgn_grad_mu": (C.c_int, [P, P, P, C.c_int, P]),
    "sgn_get_hessenberg": (C.c_int, [P, C.c_int, P, C.POINTER(C.c_int)]),
    "sgn_set_kernel_timing": (C.c_int, [P, C.c_int]),
    "sgn_get_kernel_timing": (C.c_int, [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_double)]),
    "sgn_last_error": (C.c_char_p, []),
    "sgn_version": (C.c_char_p, []),
}

_LIB = None


class SignError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libsgn.so.  Raises if it has not been built: there is no fallback."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(code: int):
    if code != SGN_OK:
        raise SignError(code, lib().sgn_last_error().decode())
    return code
