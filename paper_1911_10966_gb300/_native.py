"""ctypes binding of libesdc.so (include/esdc.h).  Argument marshalling only: every step of the
residual, time step and reductions runs in the library's CUDA kernels.  If the shared library is
missing the import of this module fails loudly: there is no fallback implementation."""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libesdc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "esdc.h")

ESDC_OK = 0
ESDC_ERR_ARG = -1
ESDC_ERR_MESH = -2
ESDC_ERR_CUDA = -3
ESDC_ERR_STATE = -4
ESDC_ERR_UNSUPPORTED = -5
FLUX = {"esc": 0, "kg": 1, "dc": 2}
PREC_FP64 = 0
PREC_FP32 = 1


METRICS = {"curl": 0, "optimized": 1}


IC = {"tgv": 0, "vortex": 1, "freestream": 2}


class Setup(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("kx", ctypes.c_int), ("ky", ctypes.c_int), ("kz", ctypes.c_int),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Ma", ctypes.c_double),
                ("Re", ctypes.c_double), ("dissipation", ctypes.c_int), ("precision", ctypes.c_int),
                ("volume_flux", ctypes.c_int), ("ip_coef", ctypes.c_double), ("bounded", ctypes.c_int),
                ("metrics", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("warp_amp", ctypes.c_double), ("warp_seed", ctypes.c_uint64)]


class EsdcError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "esdc_lgl": (I, [I, P, P]),
        "esdc_operators": (I, [I, P, P]),
        "esdc_host_geometry": (I, [ctypes.POINTER(Setup), P, P, P, ctypes.POINTER(D)]),
        "esdc_host_surface_metrics": (I, [ctypes.POINTER(Setup), P, P]),
        "esdc_init_state": (I, [P, I, P, P, P]),
        "esdc_host_coordinates": (I, [ctypes.POINTER(Setup), P]),
        "esdc_create": (I, [ctypes.POINTER(Setup), P, ctypes.POINTER(P)]),
        "esdc_destroy": (I, [P]),
        "esdc_layout": (I, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_int64)]),
        "esdc_geometry": (I, [P, P, P]),
        "esdc_rhs": (I, [P, P, P, P]),
        "esdc_rhs_host": (I, [P, P, P, P]),
        "esdc_workspace_bytes": (I, [P, I, ctypes.POINTER(S)]),
        "esdc_rk_step": (I, [P, P, D, I, P, S, P]),
        "esdc_budgets": (I, [P, P, P, ctypes.POINTER(D), P]),
        "esdc_rk_adaptive": (I, [P, P, D, D, ctypes.POINTER(D), D, D, I, P, S, P, P, I, P]),
        "esdc_budgets_async": (I, [P, P, P, P, P]),
        "esdc_set_exterior": (I, [P, P]),
        "esdc_set_source": (I, [P, P]),
        "esdc_mms_fields": (I, [D, D, D, D, D, P, ctypes.c_int64, P, P, P]),
        "esdc_dt_cfl": (I, [P, P, D, ctypes.POINTER(D), P]),
        "esdc_profile": (I, [P, I]),
        "esdc_device_status": (I, [P, ctypes.POINTER(I), I, P]),
        "esdc_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(ctypes.c_int64)]),
        "esdc_probe_fma": (I, [I, ctypes.POINTER(D), P]),
        "esdc_budgets_noalloc": (I, [I, ctypes.c_int64, D, P, P, P, P, P, P]),
        "esdc_rhs_vjp": (I, [P, P, P, P, ctypes.POINTER(D), P]),
        "esdc_ke_gradient": (I, [P, P, P, P]),
        "esdc_rk_step_ckpt": (I, [P, P, D, I, P, I, P, S, P]),
        "esdc_rk_adjoint_workspace_bytes": (I, [P, ctypes.POINTER(S)]),
        "esdc_rk_step_stages": (I, [P, P, D, I, P, P, S, P]),
        "esdc_rk_adjoint_stages": (I, [P, P, D, I, P, ctypes.POINTER(D), P, S, P]),
        "esdc_rk_adjoint": (I, [P, P, I, D, I, P, ctypes.POINTER(D), P, S, P]),
        "esdc_strerror": (ctypes.c_char_p, [I]),
        "esdc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(code: int, where: str) -> int:
    if code != ESDC_OK:
        msg = lib().esdc_last_error().decode() or lib().esdc_strerror(code).decode()
        raise EsdcError(code, where, msg)
    return code


def header_symbols() -> list[str]:
    """Every function name declared in include/esdc.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(esdc_\w+)\s*\(", txt, flags=re.M)))
