"""ctypes declarations of the C ABI in include/omm.h and include/omm_kernels.h.

Loading fails loudly when the in-tree library is missing: there is no CPU
fallback for any step of the path.
"""
from __future__ import annotations

import ctypes as ct
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libomm_gb300.so")

OMM_OK = 0
STATUS_NAMES = {0: "OMM_OK", 1: "OMM_ERR_ARG", 2: "OMM_ERR_NOT_SPD", 3: "OMM_ERR_UNBOUNDED",
                4: "OMM_ERR_NO_CONVERGENCE", 5: "OMM_ERR_NONFINITE", 6: "OMM_ERR_TIMEOUT",
                7: "OMM_ERR_CUDA", 8: "OMM_ERR_OOM", 9: "OMM_ERR_STATE"}
PREC_FP64 = 0
PREC_MIXED = 1


class OmmOpts(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("max_iter", ct.c_int), ("no_precondition", ct.c_int),
                ("check_every", ct.c_int), ("tol_grad", ct.c_double), ("e_tol", ct.c_double),
                ("refine_ratio", ct.c_double), ("profile", ct.c_int),
                ("native_certificate", ct.c_int), ("cholesky", ct.c_int),
                ("precond_slices", ct.c_int), ("debug_expire_wait", ct.c_int)]


class OmmInfo(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iterations", ct.c_int), ("iterations_fp64", ct.c_int),
                ("refinements", ct.c_int), ("E", ct.c_double), ("Etilde", ct.c_double),
                ("gmax", ct.c_double), ("ms_setup", ct.c_double), ("ms_iterate", ct.c_double),
                ("ms_refine", ct.c_double), ("ms_outputs", ct.c_double), ("gemm_flop", ct.c_double),
                ("gemm_flop_tc", ct.c_double), ("kernel_launches", ct.c_double),
                ("ms_main_gemm", ct.c_double), ("main_gemm_launches", ct.c_double),
                ("main_gemm_flop", ct.c_double), ("ms_certify", ct.c_double),
                ("ms_precond", ct.c_double),
                ("tile_width", ct.c_int * 4), ("ms_autotune", ct.c_double),
                ("ms_sliced_gemm", ct.c_double), ("sliced_gemm_flop", ct.c_double),
                ("sliced_gemm_launches", ct.c_double), ("ms_batch", ct.c_double),
                ("ms_transform", ct.c_double), ("ms_gemm_plan", ct.c_double * 4),
                ("flop_gemm_plan", ct.c_double * 4), ("ms_batch_refresh", ct.c_double)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, ct.Array) else v
        return out


class OMMError(RuntimeError):
    def __init__(self, status, where, msg):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


_lib = None

_P = ct.c_void_p
_D = ct.c_double
_I = ct.c_int
_L = ct.c_long

_SIGNATURES = {
    "omm_create": (_I, [_I, _I, _P, _P, _P, _D, _D, ct.POINTER(OmmOpts), _P, ct.POINTER(_P)]),
    "omm_solve": (_I, [_P, _P, _P, ct.POINTER(_D), _P, ct.POINTER(OmmInfo)]),
    "omm_backward": (_I, [_P, _P, _P]),
    "omm_update_H": (_I, [_P, _P]),
    "omm_free": (None, [_P]),
    "omm_status_str": (ct.c_char_p, [_I]),
    "omm_last_error": (ct.c_char_p, []),
    "omm_launch_count": (ct.c_ulonglong, []),
    "omm_create_batched": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, ct.POINTER(OmmOpts), _P, ct.POINTER(_P)]),
    "omm_solve_batched": (_I, [_P, _P, _P, _P, _P]),
    "omm_batch_instance": (_P, [_P, _I]),
    "omm_free_batched": (None, [_P]),
    "omm_create_hermitian": (_I, [_I, _I, _P, _P, _P, _D, _D, ct.POINTER(OmmOpts), _P, ct.POINTER(_P)]),
    "omm_solve_hermitian": (_I, [_P, _P, _P, ct.POINTER(_D), _P, ct.POINTER(OmmInfo)]),
    "omm_backward_hermitian": (_I, [_P, _P, _P]),
    "omm_update_H_hermitian": (_I, [_P, _P]),
    "omm_create_hermitian_batched": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, ct.POINTER(OmmOpts), _P,
                                          ct.POINTER(_P)]),
    "omm_solve_hermitian_batched": (_I, [_P, _P, _P, _P, _P]),
    "omm_kernel_dgemm": (_I, [_I, _I, _I, _I, _I, _D, _P, _L, _P, _L, _D, _P, _L, _P]),
    "omm_kernel_spd_inverse": (_I, [_I, _P, _P, ct.POINTER(_I), _P]),
    "omm_kernel_spd_inverse_sliced": (_I, [_I, _P, _P, ct.POINTER(_I), _P]),
    "omm_kernel_spd_inverse_precond": (_I, [_I, _P, _P, _I, ct.POINTER(_I), _P]),
    "omm_kernel_gemm_tc_tiled": (_I, [_I, _I, _I, _P, _P, ct.c_double, ct.c_double, _P, _I, _I, _P]),
    "omm_kernel_gemm_tc_blocksparse": (_I, [_I, _I, _I, _P, _P, ct.c_double, ct.c_double, _P, _I, _I, _P]),
    "omm_kernel_line_minimum": (_I, [ct.POINTER(_D), ct.POINTER(_D)]),
    "omm_kernel_quartic_coefficients": (_I, [_I, _P, _P, _D, ct.POINTER(_D), _P]),
    "omm_kernel_gemm_tc": (_I, [_I, _I, _I, _P, _P, _D, _D, _P, _I, _P]),
    "omm_kernel_gemm_tc_kn": (_I, [_I, _I, _I, _P, _P, _D, _D, _P, _I, _P]),
    "omm_kernel_gemm_tc_pair": (_I, [_I, _I, _I, _P, _P, _D, _D, _P, _I, _I, _I, _I, _I, _P]),
    "omm_kernel_gemm_emu": (_I, [_I, _I, _I, _P, _P, _D, _D, _P, _I, _P]),
    "omm_kernel_quartic_coefficients_noalloc": (_I, [_I, _P, _P, _D, ct.POINTER(_D), _P]),
}

# entry points declared in include/*.h, for the export check
EXPORTED = list(_SIGNATURES)


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1312_1549_gb300.build` (needs nvcc)")
        L = ct.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, where):
    if status != OMM_OK:
        msg = lib().omm_last_error()
        raise OMMError(status, where, msg.decode() if msg else "")
    return status
