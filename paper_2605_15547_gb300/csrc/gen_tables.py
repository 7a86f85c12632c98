#!/usr/bin/env python3
"""Generate ``crm_tables.h``: every table entry and polynomial coefficient that the CUDA
kernels use, computed from mathematics with mpmath at 400 bits and rounded to nearest.

Nothing here is taken from another library: the values are definitions (2^(i/16),
ln 2, Taylor coefficients (ln 2)^k / k!, log(1 + i/16), atan(i/16), bits of 2/pi, ...)
evaluated at high precision and split into float or double words.  The header is
committed; re-running this script must reproduce it bit for bit (a CPU test checks).

Usage: python gen_tables.py [output path]
"""
import os
import sys

import mpmath as mp

mp.mp.prec = 400

OUT = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                        "crm_tables.h")


def rnd(v, bits):
    """Round the mpmath value v to a binary float with `bits` significand bits (nearest)."""
    with mp.workprec(bits):
        return +mp.mpf(v)


def d(v):
    """nearest double (as an exact mpf)"""
    return rnd(v, 53)


def f(v):
    """nearest float (as an exact mpf)"""
    return rnd(v, 24)


def split(v, rounder, parts):
    out = []
    r = mp.mpf(v)
    for _ in range(parts):
        w = rounder(r)
        out.append(w)
        r = r - w
    return out


def split_bits(v, nbits):
    """Leading part of v with at most nbits significant bits (for exact products)."""
    return rnd(v, nbits)


def dlit(v):
    x = float(v)
    assert mp.mpf(x) == v, "not a double"
    return x.hex() if x != 0 else "0x0p+0"


def flit(v):
    x = float(v)
    assert mp.mpf(x) == v, "not exact"
    return (x.hex() if x != 0 else "0x0p+0") + "f"


lines = []


def emit(s=""):
    lines.append(s)


def arr_d(name, vals, comment):
    emit(f"// {comment}")
    emit(f"CRM_TABLE double {name}[{len(vals)}] = {{")
    for i in range(0, len(vals), 2):
        emit("  " + ", ".join(dlit(v) for v in vals[i:i + 2]) + ",")
    emit("};")


def arr_f(name, vals, comment):
    emit(f"// {comment}")
    emit(f"CRM_TABLE float {name}[{len(vals)}] = {{")
    for i in range(0, len(vals), 4):
        emit("  " + ", ".join(flit(v) for v in vals[i:i + 4]) + ",")
    emit("};")


def const_d(name, v, comment=""):
    emit(f"#define {name} {dlit(v)}" + (f"  // {comment}" if comment else ""))


def const_f(name, v, comment=""):
    emit(f"#define {name} {flit(v)}" + (f"  // {comment}" if comment else ""))


emit("// Generated by gen_tables.py -- do not edit.  Values are correctly rounded splits of")
emit("// mathematical constants, table entries and Taylor coefficients (see the generator).")
emit("#pragma once")
emit("#ifndef CRM_TABLE")
emit("#define CRM_TABLE static __device__ const")
emit("#endif")
emit()

LN2 = mp.log(2)
LOG2E = 1 / LN2
LOG2_10 = mp.log(10) / LN2

# ---------------------------------------------------------------- exp family
emit("// ===== exp family: 2^t = 2^k * T[j] * 2^g =====")
# 16-entry double table 2^(i/16)
arr_d("CRM_EXP2_T16_D", [d(mp.power(2, mp.mpf(i) / 16)) for i in range(16)],
      "2^(i/16), nearest double (plain form)")
# 16-entry double-double table
t16dd = []
for i in range(16):
    t16dd += split(mp.power(2, mp.mpf(i) / 16), d, 2)
arr_d("CRM_EXP2_T16_DD", t16dd, "2^(i/16) as (hi, lo) doubles (slow path)")
# 64-entry float-pair table
t64f = []
for i in range(64):
    t64f += split(mp.power(2, mp.mpf(i) / 64), f, 2)
arr_f("CRM_EXP2_T64_DF", t64f, "2^(i/64) as (hi, lo) floats (double-float form)")
emit()
# Taylor coefficients of 2^g = sum (ln2)^k/k! g^k
coef = [LN2 ** k / mp.factorial(k) for k in range(20)]
arr_d("CRM_EXP2_TAYLOR_D", [d(c) for c in coef[:8]], "(ln 2)^k / k!, k = 0..7, nearest double")
ddc = []
for c in coef[:16]:
    ddc += split(c, d, 2)
arr_d("CRM_EXP2_TAYLOR_DD", ddc, "(ln 2)^k / k!, k = 0..15, as (hi, lo) doubles")
a1 = split(coef[1], f, 2)
const_f("CRM_EXP2_A1_HI_F", a1[0], "ln 2 (float hi)")
const_f("CRM_EXP2_A1_LO_F", a1[1], "ln 2 (float lo)")
for k in (2, 3, 4, 5):
    const_f(f"CRM_EXP2_A{k}_F", f(coef[k]), f"(ln 2)^{k}/{k}!")
emit()
# conversion constants t = x * C
for nm, C in (("LOG2E", LOG2E), ("LOG2_10", LOG2_10)):
    p = split(C, d, 3)
    const_d(f"CRM_{nm}_D0", p[0])
    const_d(f"CRM_{nm}_D1", p[1])
    const_d(f"CRM_{nm}_D2", p[2])
    q = split(C, f, 3)
    const_f(f"CRM_{nm}_F0", q[0])
    const_f(f"CRM_{nm}_F1", q[1])
    const_f(f"CRM_{nm}_F2", q[2])
    const_f(f"CRM_{nm}_X16_F", f(16 * C), "16*C rounded: only picks the reduction integer")
    const_f(f"CRM_{nm}_X64_F", f(64 * C), "64*C rounded: only picks the reduction integer")
emit()

emit("// ===== end =====")

text = "\n".join(lines) + "\n"
with open(OUT, "w") as fh:
    fh.write(text)
print(f"wrote {OUT} ({len(lines)} lines)")
