"""CPU checks of the C ABI: the library loads, exports every function include/crm.h
declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2605_15547_gb300 as crm
from paper_2605_15547_gb300 import _lib as L
from paper_2605_15547_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(crm_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "crm_eval" in names and "crm_eval_batch" in names
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (crm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_argument_errors_without_gpu(lib):
    p = ctypes.c_void_p(0x1000)
    assert lib.crm_eval(99, 0, p, p, 10, None) == 1            # CRM_ERR_FUNC
    assert lib.crm_eval(-1, 0, p, p, 10, None) == 1
    assert lib.crm_eval(0, 1, p, p, 10, None) == 2             # expf with F64
    assert lib.crm_eval(19, 0, p, p, 10, None) == 2            # exp2 with F32
    assert lib.crm_eval(0, 7, p, p, 10, None) == 2
    assert lib.crm_eval(0, 0, None, p, 10, None) == 3          # null in
    assert lib.crm_eval(0, 0, p, None, 10, None) == 3
    assert lib.crm_eval(0, 0, None, None, 0, None) == 0        # n == 0: nothing to do
    a = ctypes.c_void_p(0x10000)
    b = ctypes.c_void_p(0x10000 + 8)
    assert lib.crm_eval(0, 0, a, b, 10, None) == 4             # partial overlap
    assert lib.crm_eval_form(0, 0, 5, p, p, 10, None) == 7     # unknown form
    odd = ctypes.c_void_p(0x10002)
    assert lib.crm_eval(0, 0, odd, p, 10, None) == 9           # not element aligned
    assert lib.crm_set_form(3) == 7
    assert lib.crm_set_form(0) == 0


def test_status_strings(lib):
    for s in range(11):
        assert lib.crm_status_str(s)
    assert b"unknown" in lib.crm_status_str(123)


def test_version(lib):
    assert crm.version().startswith("crm")
