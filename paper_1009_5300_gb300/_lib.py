"""ctypes binding of the C ABI declared in include/iobm.h (argument marshalling only).

Every compute step runs inside ``libiobm.so``; this module only converts
arguments.  If the library has not been built the import of the solver fails
loudly -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libiobm.so")

IOBM_OK = 0
IOBM_E_ARG = 1
IOBM_E_THRESHOLD = 2
IOBM_E_PROJ_BOUNDARY = 3
IOBM_E_NOCONV = 4
IOBM_E_BREAKDOWN = 5
IOBM_E_TIMEOUT = 6
IOBM_E_CUDA = 7
IOBM_E_STATE = 8
IOBM_E_UNSUPPORTED = 9

IOBM_FP64 = 0
IOBM_MIXED = 1
IOBM_PRECOND_NONE = 0
IOBM_PRECOND_EQ10 = 1
IOBM_PRECOND_FOURIER = 2
IOBM_PRECOND_EQ10_FOURIER = 3
IOBM_OP_AUTO = 0
IOBM_OP_EXPLICIT = 1
IOBM_SIGMA_FFT = 0
IOBM_SIGMA_DENSE = 1
IOBM_ELEM_C64 = 0
IOBM_ELEM_C32 = 1
IOBM_ELEM_C64_DF = 2


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double), ("nf", C.c_int)]


class Projectors(C.Structure):
    _fields_ = [("nproj", C.c_int), ("row_ptr", C.POINTER(C.c_int64)),
                ("idx", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double)),
                ("coupling", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("alpha", C.c_double), ("use_precond", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("precision", C.c_int), ("refine_delta", C.c_double),
                ("chunk", C.c_int), ("max_iter_mixed", C.c_int), ("op_form", C.c_int),
                ("fp64_modes", C.c_int), ("sigma_form", C.c_int)]


class Report(C.Structure):
    _fields_ = [("energy_index", C.c_int), ("channel", C.c_int), ("side", C.c_int),
                ("status", C.c_int), ("iterations", C.c_int), ("replacements", C.c_int),
                ("residual", C.c_double)]


# every exported symbol with (restype, argtypes)
SIGNATURES = {
    "iobm_default_options": (None, [C.POINTER(Options)]),
    "iobm_status_string": (C.c_char_p, [C.c_int]),
    "iobm_last_error": (C.c_char_p, [C.c_void_p]),
    "iobm_fermi_energy": (C.c_double, [C.c_void_p]),
    "iobm_create": (C.c_int, [C.POINTER(Grid), C.c_void_p, C.POINTER(Projectors), C.c_double,
                              C.POINTER(Options), C.c_void_p, C.POINTER(C.c_void_p)]),
    "iobm_destroy": (None, [C.c_void_p]),
    "iobm_open_channels": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_int), C.c_int,
                                     C.c_void_p, C.c_void_p]),
    "iobm_workspace_size": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]),
    "iobm_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "iobm_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "iobm_num_rhs": (C.c_int, [C.c_void_p]),
    "iobm_max_open": (C.c_int, [C.c_void_p]),
    "iobm_eigenchannels": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "iobm_create_batch": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p,
                                    C.POINTER(C.c_double), C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "iobm_solve_batch": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_int), C.c_int]),
    "iobm_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "iobm_set_tiling": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "iobm_transmission": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "iobm_solution": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "iobm_grad_V": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_int, C.c_void_p]),
    "iobm_apply": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "iobm_apply_precond": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                     C.c_int]),
    "iobm_solve_rhs_count": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                       C.POINTER(C.c_int)]),
    "iobm_set_potential": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "iobm_channels_host": (C.c_int, [C.POINTER(Grid), C.c_double, C.POINTER(C.c_int), C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "iobm_channels_host_bloch": (C.c_int, [C.POINTER(Grid), C.c_double, C.c_double, C.c_double,
                                           C.POINTER(C.c_int), C.c_int, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "iobm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "iobm_set_wait_limit": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int]),
    "iobm_set_bloch": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    "iobm_time_operator": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "iobm_precond_dots_noalloc": (C.c_int, [C.POINTER(Grid), C.c_double, C.c_void_p, C.c_void_p,
                                            C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "iobm_kernel_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "iobm_last_solve_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double),
                                        C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libiobm.so (built by ``paper_1009_5300_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_1009_5300_gb300.build` "
            "(the IOBM solver has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IOBMError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"IOBM error {code}: {message}")
        self.code = code


def check(code: int, handle=None):
    if code == IOBM_OK:
        return
    lib = load()
    msg = lib.iobm_status_string(code).decode()
    if handle:
        detail = lib.iobm_last_error(handle)
        if detail:
            msg += ": " + detail.decode()
    raise IOBMError(code, msg)
