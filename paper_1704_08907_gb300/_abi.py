"""ctypes binding of the C ABI in ``include/aboria_gpu.h`` (names unchanged).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module loads ``_build/libaboria_gpu.so`` and fails
loudly if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libaboria_gpu.so")

AB_OK = 0
AB_ERR_INVALID_ARG = 1
AB_ERR_ALIAS = 2
AB_ERR_STALE = 3
AB_ERR_OOM = 4
AB_ERR_CUDA = 5
AB_ERR_TIMEOUT = 6
AB_ERR_UNSUPPORTED = 7
AB_ERR_CAPACITY = 8

AB_OP_COUNT, AB_OP_GAUSS, AB_OP_LJ, AB_OP_EXPF, AB_OP_SOFT, AB_OP_SPH_DENSITY, AB_OP_SPH_FORCE = range(7)
AB_PREC_FP32, AB_PREC_TF32X3, AB_PREC_BF16X3, AB_PREC_TF32, AB_PREC_BF16 = range(5)

# Every function the headers declare, with its ctypes signature.
P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U64 = ctypes.c_uint64
F32 = ctypes.c_float
ST = ctypes.c_int


class ab_domain(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("periodic", ctypes.c_int32 * 3),
                ("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3),
                ("radius", ctypes.c_float)]


class ab_op_params(ctypes.Structure):
    _fields_ = [("s", ctypes.c_float), ("eps", ctypes.c_float),
                ("sigma", ctypes.c_float), ("c", ctypes.c_float),
                ("k", ctypes.c_float)]


SIGNATURES = {
    "ab_create": (ST, [ctypes.POINTER(P), ctypes.c_int, P]),
    "ab_destroy": (ST, [P]),
    "ab_set_stream": (ST, [P, P]),
    "ab_sync": (ST, [P]),
    "ab_build": (ST, [P, ctypes.POINTER(ab_domain), I64, P]),
    "ab_build_packed": (ST, [P, ctypes.POINTER(ab_domain), I64, P]),
    "ab_cell_shape": (ST, [P, P, P, P]),
    "ab_cell_export": (ST, [P, P, P]),
    "ab_pair_sum": (ST, [P, ctypes.c_int, ctypes.POINTER(ab_op_params), P, P, P]),
    "ab_pair_sum_bwd": (ST, [P, ctypes.c_int, ctypes.POINTER(ab_op_params), P, P, P,
                             P, P]),
    "ab_pair_sum_value_grad": (ST, [P, ctypes.c_int, ctypes.POINTER(ab_op_params), P, P, P,
                                    P, P, P, P]),
    "ab_pair_list": (ST, [P, P, P, I64, P]),
    "ab_kernel_matvec": (ST, [P, I64, I64, P, P, I32, P, F32, ctypes.c_int, P]),
    "ab_kernel_matvec_bwd": (ST, [P, I64, I64, P, P, I32, P, F32, ctypes.c_int, P,
                                  P, P, P, P]),
    "ab_bd_step": (ST, [P, ctypes.POINTER(ab_domain), I64, P, P, F32, F32, U64, U64]),
    "ab_pair_energy_grad": (ST, [P, ctypes.c_int, ctypes.POINTER(ab_op_params), P, P, P]),
    "ab_pair_energy_grad_packed": (ST, [P, ctypes.c_int, ctypes.POINTER(ab_op_params), P, P, P]),
    "ab_md_step": (ST, [P, ctypes.POINTER(ab_domain), I64, P, P, P, F32]),
    "ab_kernel_solve": (ST, [P, I64, P, I32, P, F32, F32, I32, F32, I32, P,
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
    "ab_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ab_last_error": (ctypes.c_char_p, [P]),
    "ab_testing_scan_timeout": (ST, [P, I64, I32, I64]),
    "ab_testing_build_path": (ST, [P, I32]),
    "ab_testing_cell_table": (ST, [P, I32]),
    "ab_testing_build_timeout": (ST, [P, I32, I64]),
    "ab_exclusive_scan_u32_static": (ST, [P, P, I64, P]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library not built: {path} is missing. Run "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc).")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
