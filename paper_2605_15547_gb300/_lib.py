"""ctypes binding of the C ABI declared in include/crm.h (argument marshalling only).

Every computation happens in libcrm's CUDA kernels; if the shared library is missing or
cannot be loaded this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import platform
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, f"libcrm_{platform.machine()}.so")

FUNCS = [
    "expf", "exp2f", "exp10f", "expm1f", "logf", "log2f", "log10f", "log1pf", "sinf",
    "cosf", "sincosf", "tanf", "asinf", "acosf", "atanf", "sinhf", "coshf", "tanhf",
    "rsqrtf", "exp2", "log", "exp", "log2", "log10", "exp10",
]
FUNC_ID = {n: i for i, n in enumerate(FUNCS)}
F64_FUNCS = {"exp2", "log", "exp", "log2", "log10", "exp10"}
FORMS = {"auto": 0, "plain": 1, "df": 2}
CRM_F32, CRM_F64, CRM_F16, CRM_BF16 = 0, 1, 2, 3
RMODES = {"rn": 0, "rd": 1, "ru": 2, "rz": 3}
NUM_VARIANTS = 13
BATCH_TILE_MIN, BATCH_TILE_MAX = 10, 16


class CrmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib().crm_status_str(status).decode() if _LIB is not None else str(status)
        super().__init__(f"crm status {status} ({msg}){': ' + what if what else ''}")


class crm_desc_t(ctypes.Structure):
    _fields_ = [("func_id", ctypes.c_int32), ("dtype", ctypes.c_int32), ("in_", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class crm_stats_t(ctypes.Structure):
    _fields_ = [("hard_total", ctypes.c_uint64), ("unresolved_total", ctypes.c_uint64),
                ("inline_total", ctypes.c_uint64), ("last_count", ctypes.c_uint64),
                ("timeouts", ctypes.c_uint64), ("fp64_total", ctypes.c_uint64)]


_LIB = None
_LOCK = threading.Lock()


def _lib():
    global _LIB
    if _LIB is None:
        with _LOCK:
            if _LIB is None:
                if not os.path.exists(LIB_PATH):
                    raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                                      "(python -m paper_2605_15547_gb300.build)")
                lib = ctypes.CDLL(LIB_PATH)
                c_int, c_u64, vp = ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
                lib.crm_eval.argtypes = [c_int, c_int, vp, vp, c_u64, vp]
                lib.crm_eval_form.argtypes = [c_int, c_int, c_int, vp, vp, c_u64, vp]
                lib.crm_eval_host.argtypes = [c_int, c_int, c_int, vp, vp, c_u64, vp]
                lib.crm_eval_rm.argtypes = [c_int, c_int, c_int, vp, vp, c_u64, vp]
                lib.crm_eval_complex.argtypes = [c_int, vp, vp, c_u64, vp]
                lib.crm_spectral_dft.argtypes = [vp, c_u64, vp, c_u64, vp, vp]
                lib.crm_eval_batch.argtypes = [ctypes.POINTER(crm_desc_t), c_int, c_int, vp]
                lib.crm_set_form.argtypes = [c_int]
                lib.crm_set_force_slow.argtypes = [c_int]
                lib.crm_set_batch_tile.argtypes = [c_int]
                lib.crm_eval_noalloc.argtypes = [c_int, c_int, c_int, vp, vp, c_u64, vp]
                lib.crm_noalloc_stats.argtypes = [vp, ctypes.POINTER(crm_stats_t)]
                lib.crm_noalloc_stats_reset.argtypes = [vp]
                lib.crm_reserve.argtypes = [c_u64, c_int, vp]
                pi, pf = ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_float)
                lib.crm_variant_info.argtypes = [c_int, pi, pi, pi, pi, pi, pi, pi, pi]
                lib.crm_set_variant.argtypes = [c_int, c_int, c_int]
                lib.crm_get_variant.argtypes = [c_int, c_int, pi]
                lib.crm_autotune.argtypes = [c_int, c_int, c_int, vp, vp, c_u64, c_int, vp, pi, pf]
                lib.crm_autotune_batch.argtypes = [ctypes.POINTER(crm_desc_t), c_int, c_int, c_int, vp, pi, pi, pf]
                lib.crm_set_batch_mode.argtypes = [c_int]
                lib.crm_stats.argtypes = [vp, ctypes.POINTER(crm_stats_t)]
                lib.crm_hard_case_count.argtypes = [vp, ctypes.POINTER(c_u64)]
                lib.crm_stats_reset.argtypes = [vp]
                lib.crm_status_str.argtypes = [c_int]
                lib.crm_status_str.restype = ctypes.c_char_p
                lib.crm_version.restype = ctypes.c_char_p
                lib.crm_shutdown.restype = None
                _LIB = lib
    return _LIB


def lib():
    return _lib()


def check(status: int, what: str = "") -> None:
    if status != 0:
        raise CrmError(status, what)
