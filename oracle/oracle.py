"""Correctly rounded CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python access to ``crm_oracle.c``: a Ziv-loop evaluator over fixed-point big-integer
intervals that returns RN(f(x)) for the paper's one-input functions (Sec. II.A: the 19
binary32 functions; Sec. II.B: binary64 exp2 and log).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
module.  It shares no code with the CUDA library.

The shared library is compiled with the system C compiler on first use (or by
``build()``), so the same source serves x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crm_oracle.c")
_HDR = os.path.join(_HERE, "crm_oracle.h")
_LIB = os.path.join(_HERE, f"liboracle_{platform.machine()}.so")

# Oracle function identifiers (same numbering as the public library by design).
FUNCS = [
    "expf", "exp2f", "exp10f", "expm1f", "logf", "log2f", "log10f", "log1pf",
    "sinf", "cosf", "sincosf", "tanf", "asinf", "acosf", "atanf", "sinhf", "coshf",
    "tanhf", "rsqrtf", "exp2", "log", "exp", "log2", "log10", "exp10",
]
FUNC_ID = {name: i for i, name in enumerate(FUNCS)}
F64_FUNCS = ("exp2", "log", "exp", "log2", "log10", "exp10")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its sources."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.crm_oracle_f32.argtypes = [ctypes.c_int, ctypes.c_uint32, u32p]
            lib.crm_oracle_f64.argtypes = [ctypes.c_int, ctypes.c_uint64, u64p]
            lib.crm_oracle_f32_array.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_uint64, ctypes.c_int]
            for nm in ("crm_oracle_f32_array_rm", "crm_oracle_f64_array_rm"):
                getattr(lib, nm).argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
            lib.crm_oracle_f16_array.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_uint64, ctypes.c_int]
            lib.crm_oracle_f64_array.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_uint64, ctypes.c_int]
            lib.crm_oracle_f64_hardness_array.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                          ctypes.c_uint64, ctypes.c_int]
            lib.crm_oracle_complex_array.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_uint64]
            lib.crm_oracle_constant.argtypes = [ctypes.c_int, ctypes.c_int, u64p, u64p]
            lib.crm_oracle_constant_alt.argtypes = [ctypes.c_int, ctypes.c_int, u64p, u64p]
            lib.crm_oracle_test_divmod.argtypes = [u32p, ctypes.c_int, u32p, ctypes.c_int, u32p]
            lib.crm_oracle_test_isqrt.argtypes = [u64p, ctypes.c_int, u64p]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _fid(func) -> int:
    return FUNC_ID[func] if isinstance(func, str) else int(func)


MODES = {"rn": 0, "rd": 1, "ru": 2, "rz": 3}


def eval_bits(func, xbits: np.ndarray, nthreads: int = 0, mode: str = "rn") -> np.ndarray:
    """Correctly rounded results as bit patterns.  ``xbits`` is uint32 (binary32
    functions) or uint64 (binary64 functions).  For sincosf the result has shape (2, n):
    row 0 is sin, row 1 cos.  ``mode``: rounding direction, "rn" (to nearest, ties to
    even), "rd" (toward -inf), "ru" (toward +inf) or "rz" (toward zero)."""
    lib = _load()
    fid = _fid(func)
    is64 = FUNCS[fid] in F64_FUNCS
    dt = np.uint64 if is64 else np.uint32
    x = np.ascontiguousarray(xbits, dtype=dt).ravel()
    n = x.size
    rows = 2 if FUNCS[fid] == "sincosf" else 1
    out = np.zeros(rows * n, dtype=dt)
    if n:
        fn = lib.crm_oracle_f64_array_rm if is64 else lib.crm_oracle_f32_array_rm
        st = fn(fid, x.ctypes.data, out.ctypes.data, n, nthreads, MODES[mode])
        if st:
            raise OracleError(f"oracle status {st} for {FUNCS[fid]}")
    return out.reshape(2, n) if rows == 2 else out


HALF_FMTS = {"f16": 0, "bf16": 1}


def eval_bits16(func, xbits: np.ndarray, fmt: str = "f16", mode: str = "rn") -> np.ndarray:
    """Correctly rounded results of a binary32 function's formula for 16-bit inputs and
    results (IEEE binary16 "f16" or bfloat16 "bf16"), as uint16 bit patterns; sincosf
    gives shape (2, n)."""
    lib = _load()
    fid = _fid(func)
    x = np.ascontiguousarray(xbits, dtype=np.uint16).ravel()
    n = x.size
    rows = 2 if FUNCS[fid] == "sincosf" else 1
    out = np.zeros(rows * n, dtype=np.uint16)
    if n:
        st = lib.crm_oracle_f16_array(fid, HALF_FMTS[fmt], x.ctypes.data, out.ctypes.data, n, MODES[mode])
        if st:
            raise OracleError(f"oracle status {st} for {FUNCS[fid]} ({fmt})")
    return out.reshape(2, n) if rows == 2 else out


def f64_hardness(func, xbits: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """For binary64 exp2 / log: -log2 of the distance (in ulps of the result) from f(x) to
    the nearest round-to-nearest boundary, per input (float64; capped at 128, <= 1 for
    special inputs and exact results)."""
    lib = _load()
    fid = _fid(func)
    x = np.ascontiguousarray(xbits, dtype=np.uint64).ravel()
    out = np.zeros(x.size, dtype=np.float64)
    if x.size:
        st = lib.crm_oracle_f64_hardness_array(fid, x.ctypes.data, out.ctypes.data, x.size, nthreads)
        if st:
            raise OracleError(f"oracle status {st} for {FUNCS[fid]} hardness")
    return out


COMPLEX = {"cexpf": 0, "clogf": 1, "csinf": 2}


def eval_complex(func, zbits: np.ndarray) -> np.ndarray:
    """Each component of cexp, clog or csin ("cexpf", "clogf", "csinf") of the binary32
    complex numbers zbits (uint32, interleaved re, im), rounded to nearest: uint32 bits,
    interleaved the same way."""
    lib = _load()
    z = np.ascontiguousarray(zbits, dtype=np.uint32).ravel()
    out = np.zeros(z.size, dtype=np.uint32)
    if z.size:
        st = lib.crm_oracle_complex_array(COMPLEX[func], z.ctypes.data, out.ctypes.data, z.size // 2)
        if st:
            raise OracleError(f"oracle status {st} for {func}")
    return out


def eval_f32(func, x: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Float32 convenience wrapper around ``eval_bits``."""
    bits = eval_bits(func, np.asarray(x, dtype=np.float32).view(np.uint32), nthreads)
    return bits.view(np.float32)


def eval_f64(func, x: np.ndarray, nthreads: int = 0) -> np.ndarray:
    bits = eval_bits(func, np.asarray(x, dtype=np.float64).view(np.uint64), nthreads)
    return bits.view(np.float64)


def last_level() -> int:
    return _load().crm_oracle_last_level()


def _limbs_to_int(arr) -> int:
    v = 0
    for i, w in enumerate(arr):
        v |= int(w) << (64 * i)
    return v


def constant(which: int, nlimbs: int, alt: bool = False):
    """(floor, ceil) of c * 2^(64*(nlimbs-1)) for c in {0: ln2, 1: ln10, 2: pi, 3: 2/pi}."""
    lib = _load()
    lo = (ctypes.c_uint64 * nlimbs)()
    hi = (ctypes.c_uint64 * nlimbs)()
    fn = lib.crm_oracle_constant_alt if alt else lib.crm_oracle_constant
    if fn(which, nlimbs, lo, hi):
        raise OracleError("bad constant request")
    return _limbs_to_int(lo), _limbs_to_int(hi)


def test_divmod(u: int, v: int):
    """floor(u/v) and remainder-nonzero flag through the oracle's long division."""
    lib = _load()

    def digits(x):
        d = []
        while x:
            d.append(x & 0xFFFFFFFF)
            x >>= 32
        return d or [0]

    ud, vd = digits(u), digits(v)
    if len(ud) < len(vd):
        return 0, int(u != 0)
    U = (ctypes.c_uint32 * len(ud))(*ud)
    V = (ctypes.c_uint32 * len(vd))(*vd)
    Q = (ctypes.c_uint32 * (len(ud) - len(vd) + 1))()
    nz = lib.crm_oracle_test_divmod(U, len(ud), V, len(vd), Q)
    q = 0
    for i, w in enumerate(Q):
        q |= int(w) << (32 * i)
    return q, nz


def test_isqrt(N: int, nl: int):
    lib = _load()
    arr = (ctypes.c_uint64 * nl)(*[(N >> (64 * i)) & (2**64 - 1) for i in range(nl)])
    out = (ctypes.c_uint64 * nl)()
    inexact = lib.crm_oracle_test_isqrt(arr, nl, out)
    return _limbs_to_int(out), inexact
