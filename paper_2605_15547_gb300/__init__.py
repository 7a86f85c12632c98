"""Correctly rounded array math on GB300 (sm_103a): Python binding of include/crm.h.

    import torch, paper_2605_15547_gb300 as crm
    y = crm.eval("expf", x)            # x: contiguous float32 CUDA tensor
    y = crm.eval("sinf", x, form="df") # force the double-float form

Torch supplies device memory and the current stream; every element is computed by the
library's CUDA kernels (the C ABI), which fail loudly when the library is missing.
"""
from __future__ import annotations

import ctypes

from . import _lib as L
from ._lib import F64_FUNCS, FORMS, FUNC_ID, FUNCS, CrmError, crm_desc_t, crm_stats_t

__all__ = ["eval", "eval_into", "eval_rm", "eval_complex", "spectral_dft", "eval_host", "eval_batch", "stats", "stats_reset",
           "hard_case_count",
           "set_form", "set_force_slow", "set_batch_tile", "reserve", "FUNCS", "FORMS", "CrmError", "version",
           "variant_info", "set_variant", "get_variant", "autotune", "autotune_batch", "set_batch_mode"]


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _fid(func) -> int:
    if isinstance(func, str):
        if func not in FUNC_ID:
            raise ValueError(f"unknown function {func!r}")
        return FUNC_ID[func]
    return int(func)


def _form(form) -> int:
    if form is None:
        return 0
    if isinstance(form, str):
        return FORMS[form]
    return int(form)


def out_shape(func, n: int):
    return (2, n) if FUNCS[_fid(func)] == "sincosf" else (n,)


def _check_tensors(fid: int, x, out) -> None:
    """x and out: contiguous tensors of the function's dtype on the same CUDA device, out
    large enough (2n elements for sincosf).  The C ABI sees only pointers and a length,
    so a strided view or a wrong dtype would otherwise be evaluated as raw memory."""
    import torch
    want = torch.float64 if FUNCS[fid] in F64_FUNCS else torch.float32
    for name, t in (("x", x), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.dtype != want:
            raise TypeError(f"{FUNCS[fid]} takes {want}, got {t.dtype} for {name}")
    if x.device != out.device:
        raise ValueError(f"x is on {x.device}, out on {out.device}")
    need = (2 if FUNCS[fid] == "sincosf" else 1) * x.numel()
    if out.numel() < need:
        raise ValueError(f"out holds {out.numel()} elements, {FUNCS[fid]} needs {need}")


def eval_into(func, x, out, form=None, stream=None) -> None:
    """out <- RN(f(x)) for contiguous CUDA tensors (sincosf: out has 2*n elements)."""
    fid = _fid(func)
    _check_tensors(fid, x, out)
    dtype = L.CRM_F64 if FUNCS[fid] in F64_FUNCS else L.CRM_F32
    n = x.numel()
    L.check(L.lib().crm_eval_form(fid, dtype, _form(form), ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), n, _stream_ptr(stream)),
            FUNCS[fid])


def eval(func, x, out=None, form=None, stream=None):
    """Return RN(f(x)) elementwise (a new tensor unless `out` is given).  For sincosf the
    result has shape (2, *x.shape): sin then cos."""
    import torch
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    fid = _fid(func)
    want = torch.float64 if FUNCS[fid] in F64_FUNCS else torch.float32
    if x.dtype != want:
        raise TypeError(f"{FUNCS[fid]} takes {want}, got {x.dtype}")
    if out is None:
        shape = ((2,) + tuple(x.shape)) if FUNCS[fid] == "sincosf" else x.shape
        out = torch.empty(shape, dtype=want, device=x.device)
    eval_into(fid, x, out, form=form, stream=stream)
    return out


def eval_rm(func, x, mode="rn", out=None, stream=None):
    """f(x) correctly rounded in direction mode ("rn", "rd", "ru", "rz") to x's format:
    float32 or float64 (the function's own), or float16 / bfloat16 for the binary32
    functions (their formula on 16-bit inputs and results).  Returns out (a new tensor
    unless given; sincosf: shape (2, *x.shape))."""
    import torch
    fid = _fid(func)
    kinds = {torch.float32: L.CRM_F32, torch.float64: L.CRM_F64, torch.float16: L.CRM_F16,
             torch.bfloat16: L.CRM_BF16}
    if not isinstance(x, torch.Tensor) or not x.is_cuda or not x.is_contiguous() or x.dtype not in kinds:
        raise ValueError("x must be a contiguous CUDA tensor of float32, float64, float16 or bfloat16")
    rows = 2 if FUNCS[fid] == "sincosf" else 1
    if out is None:
        out = torch.empty(((2,) if rows == 2 else ()) + tuple(x.shape), dtype=x.dtype, device=x.device)
    if not out.is_cuda or not out.is_contiguous() or out.dtype != x.dtype or out.numel() < rows * x.numel() \
            or out.device != x.device:
        raise ValueError("out must be a contiguous CUDA tensor of x's dtype and device, large enough")
    L.check(L.lib().crm_eval_rm(fid, kinds[x.dtype], L.RMODES[mode], ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), x.numel(), _stream_ptr(stream)),
            f"{FUNCS[fid]} {mode}")
    return out


COMPLEX_FUNCS = {"cexpf": 0, "clogf": 1, "csinf": 2}


def eval_complex(func, z, out=None, stream=None):
    """cexpf, clogf or csinf of a contiguous complex64 CUDA tensor (each component within
    2 ulp; see include/crm.h for the valid inputs).  Returns out (new unless given)."""
    import torch
    if not isinstance(z, torch.Tensor) or not z.is_cuda or not z.is_contiguous() or z.dtype != torch.complex64:
        raise ValueError("z must be a contiguous complex64 CUDA tensor")
    if out is None:
        out = torch.empty_like(z)
    if not out.is_contiguous() or out.dtype != torch.complex64 or out.numel() < z.numel() or out.device != z.device:
        raise ValueError("out must be a contiguous complex64 tensor like z")
    L.check(L.lib().crm_eval_complex(COMPLEX_FUNCS[func], ctypes.c_void_p(z.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), z.numel(), _stream_ptr(stream)), func)
    return out


def spectral_dft(x, freq, out=None, stream=None):
    """X(f) = sum_n x[n] exp(-2 pi i f n / N) for each f in freq (float32 CUDA tensors; N =
    x.numel() a power of two), with correctly rounded sines and cosines; returns a complex128
    tensor (out, if given, a float64 tensor of 2 * freq.numel())."""
    import torch
    for name, t in (("x", x), ("freq", freq)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.dtype != torch.float32:
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    m = freq.numel()
    if out is None:
        out = torch.empty(2 * m, dtype=torch.float64, device=x.device)
    if not out.is_contiguous() or out.dtype != torch.float64 or out.numel() < 2 * m:
        raise ValueError("out must be a contiguous float64 tensor of 2 * freq.numel()")
    L.check(L.lib().crm_spectral_dft(ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(freq.data_ptr()),
                                     m, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "spectral_dft")
    return torch.view_as_complex(out[:2 * m].view(m, 2))


def eval_host(func, x_np, out_np=None, form=None, stream=None):
    """Host (numpy) buffers in and out; the library copies, computes and copies back."""
    import numpy as np
    fid = _fid(func)
    f64 = FUNCS[fid] in F64_FUNCS
    x_np = np.ascontiguousarray(x_np, dtype=np.float64 if f64 else np.float32)
    n = x_np.size
    if out_np is None:
        out_np = np.empty((2 * n) if FUNCS[fid] == "sincosf" else n, dtype=x_np.dtype)
    L.check(L.lib().crm_eval_host(fid, L.CRM_F64 if f64 else L.CRM_F32, _form(form),
                                  ctypes.c_void_p(x_np.ctypes.data),
                                  ctypes.c_void_p(out_np.ctypes.data), n,
                                  _stream_ptr(stream)), FUNCS[fid])
    return out_np


def _descs(items):
    descs = (crm_desc_t * len(items))()
    for d, (func, x, out) in zip(descs, items):
        fid = _fid(func)
        _check_tensors(fid, x, out)
        d.func_id = fid
        d.dtype = L.CRM_F64 if FUNCS[fid] in F64_FUNCS else L.CRM_F32
        d.in_ = x.data_ptr()
        d.out = out.data_ptr()
        d.n = x.numel()
    return descs


def eval_batch(items, form=None, stream=None) -> None:
    """items: list of (func, x, out) with contiguous CUDA tensors; one batched launch."""
    L.check(L.lib().crm_eval_batch(_descs(items), len(items), _form(form), _stream_ptr(stream)), "batch")


def stats(stream=None) -> dict:
    s = crm_stats_t()
    L.check(L.lib().crm_stats(_stream_ptr(stream), ctypes.byref(s)))
    return {"hard_total": s.hard_total, "unresolved_total": s.unresolved_total,
            "inline_total": s.inline_total, "last_count": s.last_count, "timeouts": s.timeouts,
            "fp64_total": s.fp64_total}


def hard_case_count(stream=None) -> int:
    """Lanes the last call on the stream queued for the slow path (synchronises)."""
    v = ctypes.c_uint64()
    L.check(L.lib().crm_hard_case_count(_stream_ptr(stream), ctypes.byref(v)))
    return v.value


def stats_reset(stream=None) -> None:
    L.check(L.lib().crm_stats_reset(_stream_ptr(stream)))


def set_form(form) -> None:
    L.check(L.lib().crm_set_form(_form(form)))


def set_batch_tile(log2_elems: int) -> None:
    """Tile size of the batching form: 2^log2_elems elements."""
    L.check(L.lib().crm_set_batch_tile(int(log2_elems)))


def set_force_slow(on) -> None:
    """Test hook: False/0 off; True/1 every lane through every tier of the slow path;
    2 every lane through the slow path, whose first tier decides where it can."""
    L.check(L.lib().crm_set_force_slow(2 if on == 2 else (1 if on else 0)))


def reserve(max_elems: int, max_arrays: int = 0, stream=None) -> None:
    L.check(L.lib().crm_reserve(max_elems, max_arrays, _stream_ptr(stream)))


def variant_info(v: int) -> dict:
    """Launch shape of main-kernel variant v (0 <= v < NUM_VARIANTS)."""
    a = [ctypes.c_int() for _ in range(8)]
    L.check(L.lib().crm_variant_info(int(v), *[ctypes.byref(t) for t in a]))
    return {"unroll": a[0].value, "block": a[1].value, "prefetch": bool(a[2].value),
            "pipelined": bool(a[3].value), "min_blocks": a[4].value, "vec_bytes": a[5].value,
            "reg_table": bool(a[6].value), "easy": bool(a[7].value)}


def set_variant(func, variant: int, form=None) -> None:
    L.check(L.lib().crm_set_variant(_fid(func), _form(form), int(variant)))


def get_variant(func, form=None) -> int:
    v = ctypes.c_int()
    L.check(L.lib().crm_get_variant(_fid(func), _form(form), ctypes.byref(v)))
    return v.value


def autotune(func, x, out=None, form=None, reps: int = 3, stream=None):
    """Time every launch shape of `func` on x (and out, overwritten), keep the fastest for
    later calls; returns (best variant, {variant: ms per call})."""
    import torch
    fid = _fid(func)
    if out is None:
        out = torch.empty(((2,) if FUNCS[fid] == "sincosf" else ()) + tuple(x.shape), dtype=x.dtype,
                          device=x.device)
    best = ctypes.c_int()
    ms = (ctypes.c_float * L.NUM_VARIANTS)()
    dtype = L.CRM_F64 if FUNCS[fid] in F64_FUNCS else L.CRM_F32
    L.check(L.lib().crm_autotune(fid, dtype, _form(form), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), x.numel(), int(reps), _stream_ptr(stream),
                                 ctypes.byref(best), ms), FUNCS[fid])
    return best.value, {v: ms[v] for v in range(L.NUM_VARIANTS) if ms[v] >= 0}


BATCH_MODES = {"mixed": 0, "grouped": 1}


def set_batch_mode(mode) -> None:
    """'mixed': one kernel over all arrays; 'grouped': one kernel per function present."""
    L.check(L.lib().crm_set_batch_mode(BATCH_MODES[mode] if isinstance(mode, str) else int(mode)))


def autotune_batch(items, form=None, reps: int = 2, stream=None):
    """Time the batch modes and tile sizes on this batch and keep the fastest; returns
    (best mode, best log2 tile, {(mode, log2 tile): ms per call})."""
    mode, best = ctypes.c_int(), ctypes.c_int()
    n = L.BATCH_TILE_MAX - L.BATCH_TILE_MIN + 1
    ms = (ctypes.c_float * (2 * n))()
    L.check(L.lib().crm_autotune_batch(_descs(items), len(items), _form(form), int(reps), _stream_ptr(stream),
                                       ctypes.byref(mode), ctypes.byref(best), ms), "batch autotune")
    names = {v: k for k, v in BATCH_MODES.items()}
    return (names[mode.value], best.value,
            {(names[m], L.BATCH_TILE_MIN + i): ms[m * n + i] for m in range(2) for i in range(n)})


def version() -> str:
    return L.lib().crm_version().decode()
