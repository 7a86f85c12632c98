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
# 64-entry float4 table (T hi, T lo, U hi, U lo) with T = 2^(i/64), U = T ln 2
t64u = []
for i in range(64):
    T = mp.power(2, mp.mpf(i) / 64)
    t64u += split(T, f, 2) + split(T * LN2, f, 2)
arr_f("CRM_EXP2_T64U_DF", t64u, "(2^(i/64) hi, lo, 2^(i/64) ln2 hi, lo) floats (double-float form)")
# 16-entry float4 table of the same layout: the register-resident variant (lane l holds
# entry l mod 16, read by warp shuffles)
t16u = []
for i in range(16):
    T = mp.power(2, mp.mpf(i) / 16)
    t16u += split(T, f, 2) + split(T * LN2, f, 2)
arr_f("CRM_EXP2_T16U_DF", t16u, "(2^(i/16) hi, lo, 2^(i/16) ln2 hi, lo) floats (register-table variant)")
emit()


def f32_below(v):
    """largest binary32 value < v (v not representable)"""
    import struct
    x = float(f(v))
    if mp.mpf(x) >= v:
        b = struct.unpack("<i", struct.pack("<f", x))[0]
        b = b - 1 if x > 0 else b + 1
        x = struct.unpack("<f", struct.pack("<i", b))[0]
    assert mp.mpf(x) < v
    return mp.mpf(x)


def f32_above(v):
    import struct
    x = float(f(v))
    if mp.mpf(x) <= v:
        b = struct.unpack("<i", struct.pack("<f", x))[0]
        b = b + 1 if x >= 0 else b - 1
        x = struct.unpack("<f", struct.pack("<i", b))[0]
    assert mp.mpf(x) > v
    return mp.mpf(x)


# Input thresholds of b^x in binary32 (b = e, 2, 10), from the exact rounding boundaries:
#   OVF : largest x with b^x < 2^128 - 2^103 (finite result), larger x give +inf;
#   ZERO: smallest x with b^x > 2^-150 (nonzero result), smaller x give +0;
#   SUB : smallest binary32 x with b^x >= 2^-126 (normal result); x below it and >= ZERO
#         give subnormal results.
OVF_REAL = mp.mpf(2) ** 128 - mp.mpf(2) ** 103
for nm, lnb in (("EXP", mp.mpf(1)), ("EXP2", LN2), ("EXP10", mp.log(10))):
    ovf = f32_below(mp.log(OVF_REAL) / lnb)
    zero = f32_above(mp.log(mp.mpf(2) ** -150) / lnb)
    sub = f32_above(mp.log(mp.mpf(2) ** -126) / lnb)
    const_f(f"CRM_{nm}F_X_OVF", ovf, "largest input with a finite result")
    const_f(f"CRM_{nm}F_X_ZERO", zero, "smallest input with a nonzero result")
    const_f(f"CRM_{nm}F_X_SUB", sub, "smallest input with a normal result")
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
for k in (2, 3, 4, 5, 6):
    const_f(f"CRM_EXP2_A{k}_F", f(coef[k]), f"(ln 2)^{k}/{k}!")
a2 = split(coef[2], f, 2)
const_f("CRM_EXP2_A2_HI_F", a2[0], "(ln 2)^2/2 (float hi)")
const_f("CRM_EXP2_A2_LO_F", a2[1], "(ln 2)^2/2 (float lo)")
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

# ---------------------------------------------------------------- log family
emit("// ===== log family: x = 2^e m with m in [3/4, 3/2) (the paper's Fig. 2 split),      =====")
emit("// ===== c_j = j/128 (j = round(128 m), 96..192), log x = e log 2 + log c_j + log1p(r), =====")
emit("// ===== r = (m - c_j)/c_j, |r| <= 2^-7.58; entry j-96                                  =====")
for kind, base in (("LN", None), ("LOG2", 2), ("LOG10", 10)):
    def lg(v):
        return mp.log(v) if base is None else mp.log(v) / mp.log(base)
    td, tdd = [], []
    for j in range(96, 193):
        c = mp.mpf(j) / 128
        rc = 1 / c
        L = lg(c)
        td += [d(rc), d(L)]
        tdd += split(rc, d, 2) + split(L, d, 2)
    arr_d(f"CRM_{kind}_T97_D", td, f"(1/c_j, {kind.lower()}(c_j)) doubles")
    arr_d(f"CRM_{kind}_T97_DD", tdd, f"(1/c_j, {kind.lower()}(c_j)) as double-double")
# Double-float tier: c_j = j/256 (j = round(256 m), 192..384) and R_j = 1/c_j rounded to 9
# significant bits, so that r = m R_j - 1 is one exact FMA: m R_j is a multiple of 2^-32
# (m has 24 significant bits, R_j 9, and R_j >= 1 exactly when m < 1) and |r| < 2^-8, so r
# is an integer below 2^24 times 2^-32.  L_j = -ln(R_j) is split three ways (log2 and log10
# scale the natural logarithm): L_hi on the grid 2^-17, so that e ln2_hi + L_hi is exact in
# binary32 for every exponent e of a binary32 input (|e| <= 149, ln2_hi = CRM_LN2_F16_HI, a
# multiple of 2^-15: the sum is a multiple of 2^-17 below 2^7); L_mid on the grid 2^-32 with
# |L_mid| <= 2^-18, so that r + L_mid is exact (a multiple of 2^-32 below 2^-8); L_lo the
# nearest float to the rest.  Entry j-192 is (R_j, L_hi, L_mid, L_lo).
emit("// ===== log family, double-float tier: R_j = 1/(j/256) to 9 bits, j = round(256 m) in   =====")
emit("// ===== 192..384, r = m R_j - 1 exact, ln x = e ln 2 - ln R_j + log1p(r); entry j-192 =====")
rmax = mp.mpf(0)
GH, GM = mp.mpf(2) ** -17, mp.mpf(2) ** -32
LN2_F16_HI = rnd(LN2, 16)
assert mp.nint(LN2_F16_HI / 2 ** -15) * 2 ** -15 == LN2_F16_HI and 149 * LN2_F16_HI + 1 < 2 ** 24 * GH
tf, midmax = [], mp.mpf(0)
for j in range(192, 385):
    R = rnd(mp.mpf(256) / j, 9)
    # |r| over m in [(j - 1/2)/256, (j + 1/2)/256] intersected with [3/4, 3/2)
    lo_m = max(mp.mpf(j) - mp.mpf(1) / 2, 192) / 256
    hi_m = min(mp.mpf(j) + mp.mpf(1) / 2, 384) / 256
    rj = max(abs(lo_m * R - 1), abs(hi_m * R - 1))
    rmax = max(rmax, rj)
    L = -mp.log(R)
    Lh = mp.nint(L / GH) * GH
    Lm = mp.nint((L - Lh) / GM) * GM
    Ll = f(L - Lh - Lm)
    assert f(Lh) == Lh and f(Lm) == Lm and abs(Lm) <= GH / 2
    assert abs(L - Lh - Lm - Ll) < mp.mpf(2) ** -57
    midmax = max(midmax, abs(Lm))
    # Fast2Sum(e ln2_hi + L_hi, s) with e = 0 needs |L_hi| >= |s|, s = RN(r + L_mid - r^2/2)
    if j != 256:
        assert abs(Lh) >= (rj + abs(Lm) + rj * rj) * mp.mpf("1.01"), j
    else:
        assert Lh == 0 and Lm == 0 and Ll == 0
    tf += [f(R), Lh, Lm, Ll]
arr_f("CRM_LN_T193M_DF", tf, "(R_j, -ln(R_j) hi (grid 2^-17), mid (grid 2^-32), lo) floats, R_j 9 bits")
assert rmax < mp.mpf(2) ** -8, rmax  # r exact (see above); max |r| = 2^-8.008
assert rmax + midmax < mp.mpf(2) ** -8  # r + L_mid exact
LOG10_2 = mp.log(2) / mp.log(10)
for nm, v in (("LN2", LN2), ("LOG10_2", LOG10_2)):
    hi = rnd(v, 16)
    const_f(f"CRM_{nm}_F16_HI", hi, "16 bits: e * this is exact in binary32")
    const_f(f"CRM_{nm}_F16_LO", f(v - hi))
    hi = rnd(v, 42)
    const_d(f"CRM_{nm}_D42_HI", hi, "42 bits: e * this is exact in binary64")
    const_d(f"CRM_{nm}_D42_LO", d(v - hi))
    dp = split(v, d, 2)
    const_d(f"CRM_{nm}_DD_HI", dp[0])
    const_d(f"CRM_{nm}_DD_LO", dp[1])
for nm, v in (("INV_LN2", 1 / LN2), ("INV_LN10", 1 / mp.log(10))):
    fp = split(v, f, 2)
    const_f(f"CRM_{nm}_F_HI", fp[0])
    const_f(f"CRM_{nm}_F_LO", fp[1])
    dp = split(v, d, 2)
    const_d(f"CRM_{nm}_D_HI", dp[0])
    const_d(f"CRM_{nm}_D_LO", dp[1])
# log1p Taylor coefficients (-1)^(k+1)/k
arr_d("CRM_LOG1P_TAYLOR_D", [d(mp.mpf((-1) ** (k + 1)) / k) for k in range(1, 10)],
      "(-1)^(k+1)/k, k = 1..9, doubles")
l1dd = []
for k in range(1, 18):
    l1dd += split(mp.mpf((-1) ** (k + 1)) / k, d, 2)
arr_d("CRM_LOG1P_TAYLOR_DD", l1dd, "(-1)^(k+1)/k, k = 1..17, double-double")
emit()

# ---------------------------------------------------------------- hyperbolic / expm1
emit("// ===== expm1 / sinh / cosh / tanh =====")
# thresholds: sinh/cosh overflow, tanh rounding to +-1, expm1 rounding to -1
def largest_f32_with(pred, lo, hi):
    """largest binary32 x in [lo, hi] with pred(x) true (pred monotone: true then false)"""
    import struct
    def bits(v):
        return struct.unpack("<i", struct.pack("<f", v))[0]
    def val(b):
        return struct.unpack("<f", struct.pack("<i", b))[0]
    a, b = bits(lo), bits(hi)
    assert pred(mp.mpf(val(a))) and not pred(mp.mpf(val(b)))
    while b - a > 1:
        m = (a + b) // 2
        if pred(mp.mpf(val(m))):
            a = m
        else:
            b = m
    return mp.mpf(val(a))
half_ulp_below_1 = mp.mpf(2) ** -25
const_f("CRM_SINHF_X_OVF", largest_f32_with(lambda v: mp.sinh(v) < OVF_REAL, 80.0, 100.0),
        "largest input with a finite sinh / cosh")
const_f("CRM_TANHF_X_ONE", largest_f32_with(lambda v: 1 - mp.tanh(v) > half_ulp_below_1, 1.0, 20.0),
        "largest input whose tanh does not round to 1")
const_f("CRM_EXPM1F_X_MONE", -largest_f32_with(lambda v: 1 - mp.exp(-v) < 1 - half_ulp_below_1, 1.0, 40.0),
        "inputs below this give exactly -1")
# The next step of the saturation staircases: inputs in (X_NEXT, X_ONE] give tanh = 1 - 2^-24
# exactly, inputs in [X_MONE, X_M2] give expm1 = -1 + 2^-24 (the midpoints next to them
# are 1 - 3 2^-25 and -1 + 3 2^-25, whose preimages are transcendental).
const_f("CRM_TANHF_X_NEXT", f32_below(mp.atanh(1 - 3 * half_ulp_below_1)),
        "largest input whose tanh rounds below 1 - 2^-24")
const_f("CRM_EXPM1F_X_M2", f32_below(mp.log(3 * half_ulp_below_1)),
        "largest input whose expm1 rounds to -1 + 2^-24")
# Taylor coefficients 1/k! (double and double-double)
arr_d("CRM_INVFACT_D", [d(1 / mp.factorial(k)) for k in range(20)], "1/k!, k = 0..19")
ifdd = []
for k in range(28):
    ifdd += split(1 / mp.factorial(k), d, 2)
arr_d("CRM_INVFACT_DD", ifdd, "1/k!, k = 0..27, double-double")
emit()

# ---------------------------------------------------------------- trig
emit("// ===== trig: |x| 64/pi = 128 m + 32 q + j + f (integer reduction), t = f pi/64 =====")
bits_needed = 32 * 14
with mp.workprec(bits_needed + 128):
    v = int(mp.floor(2 / mp.pi * mp.mpf(2) ** bits_needed))
words = [0, 0] + [(v >> (bits_needed - 32 * (i + 1))) & 0xFFFFFFFF for i in range(14)]
emit("// bits of 2/pi after the binary point, 32 per word, preceded by two zero words")
emit(f"CRM_TABLE unsigned int CRM_TWO_OVER_PI_W[{len(words)}] = {{")
for i in range(0, len(words), 4):
    emit("  " + ", ".join(f"0x{w:08X}u" for w in words[i:i + 4]) + ",")
emit("};")
sc_d, sc_f, sc_dd = [], [], []
for j in range(32):
    a = mp.mpf(j) * mp.pi / 64
    S, C = mp.sin(a), mp.cos(a)
    sc_d += [d(S), d(C)]
    sc_f += split(S, f, 2) + split(C, f, 2)
    sc_dd += split(S, d, 2) + split(C, d, 2)
arr_d("CRM_SINCOS_T32_D", sc_d, "(sin, cos)(j pi/64), j = 0..31, doubles")
arr_d("CRM_SINCOS_T32_DD", sc_dd, "(sin, cos)(j pi/64) as double-double")
# Double-float tier: 128 steps per quadrant, a = j pi/256
sc_f, tn_f = [], []
for j in range(128):
    a = mp.mpf(j) * mp.pi / 256
    sc_f += split(mp.sin(a), f, 2) + split(mp.cos(a), f, 2)
    tn_f += split(mp.tan(a), f, 2)
arr_f("CRM_SINCOS_T128_DF", sc_f, "(sin hi, lo, cos hi, lo)(j pi/256), j = 0..127, floats")
arr_f("CRM_TAN_T128_DF", tn_f, "(tan hi, lo)(j pi/256), j = 0..127, floats")
const_f("CRM_TAN_C5_F", f(mp.mpf(2) / 15), "2/15, the t^5 coefficient of tan t")
PIO64 = mp.pi / 64
pp = split(PIO64, d, 2)
const_d("CRM_PIO64_D_HI", pp[0])
const_d("CRM_PIO64_D_LO", pp[1])
PIO256 = mp.pi / 256
pf = split(PIO256, f, 2)
const_f("CRM_PIO256_F_HI", pf[0])
const_f("CRM_PIO256_F_LO", pf[1])
# Cody-Waite split of pi/256 into three floats: CW1 is a multiple of 2^-30, so |x| - k CW1
# is exact after one FMA for the k of |x| < 2^12 (k < 2^18.35); k CW2 is split exactly by an
# FMA, CW3 carries the rest (error < 2^-83)
cw = split(PIO256, f, 3)
assert abs(PIO256 - cw[0] - cw[1] - cw[2]) < mp.mpf(2) ** -83
assert mp.nint(cw[0] * 2 ** 30) == cw[0] * 2 ** 30
const_f("CRM_PIO256_CW1", cw[0], "pi/256 = CW1 + CW2 + CW3 (+ < 2^-83)")
const_f("CRM_PIO256_CW2", cw[1])
const_f("CRM_PIO256_CW3", cw[2])
const_f("CRM_256OPI_F", f(256 / mp.pi), "256/pi, nearest float")
i3 = split(mp.mpf(1) / 3, f, 2)
const_f("CRM_INV3_F_HI", i3[0])
const_f("CRM_INV3_F_LO", i3[1])
i6 = split(mp.mpf(1) / 6, f, 2)
const_f("CRM_INV6_F_HI", i6[0])
const_f("CRM_INV6_F_LO", i6[1])
# (-1)^k / (2k+1)! and (-1)^k/(2k)! as doubles and double-doubles
# FP64-free middle tier of the trigonometric functions: signed Q126 fixed point as
# two's complement 128-bit (low word first)
def q126(v):
    with mp.workprec(400):
        N = int(mp.nint(mp.mpf(v) * mp.mpf(2) ** 126))
    assert -2 ** 127 < N < 2 ** 127
    N &= (1 << 128) - 1
    return [N & 0xFFFFFFFFFFFFFFFF, N >> 64]
def arr_u64(name, vals, comment):
    emit(f"// {comment}")
    emit(f"CRM_TABLE unsigned long long {name}[{len(vals)}] = {{")
    for i in range(0, len(vals), 4):
        emit("  " + ", ".join(f"0x{v:016X}ull" for v in vals[i:i + 4]) + ",")
    emit("};")
tsc = []
for j in range(32):
    a = mp.mpf(j) * mp.pi / 64
    tsc += q126(mp.sin(a)) + q126(mp.cos(a))
arr_u64("CRM_TRIGI_SC", tsc, "(sin, cos)(j pi/64) in Q126, (lo, hi) words, j = 0..31")
arr_u64("CRM_TRIGI_S", sum((q126(mp.mpf((-1) ** k) / mp.factorial(2 * k + 1)) for k in range(1, 7)), []),
        "(-1)^k/(2k+1)! in Q126, k = 1..6")
arr_u64("CRM_TRIGI_C", sum((q126(mp.mpf((-1) ** k) / mp.factorial(2 * k)) for k in range(1, 8)), []),
        "(-1)^k/(2k)! in Q126, k = 1..7")
arr_u64("CRM_TRIGI_PIO64", q126(mp.pi / 64), "pi/64 in Q126")
arr_d("CRM_SIN_TAYLOR_D", [d(mp.mpf((-1) ** k) / mp.factorial(2 * k + 1)) for k in range(10)],
      "(-1)^k/(2k+1)!, k = 0..9")
arr_d("CRM_COS_TAYLOR_D", [d(mp.mpf((-1) ** k) / mp.factorial(2 * k)) for k in range(10)],
      "(-1)^k/(2k)!, k = 0..9")
sdd, cdd = [], []
for k in range(12):
    sdd += split(mp.mpf((-1) ** k) / mp.factorial(2 * k + 1), d, 2)
    cdd += split(mp.mpf((-1) ** k) / mp.factorial(2 * k), d, 2)
arr_d("CRM_SIN_TAYLOR_DD", sdd, "(-1)^k/(2k+1)!, k = 0..11, double-double")
arr_d("CRM_COS_TAYLOR_DD", cdd, "(-1)^k/(2k)!, k = 0..11, double-double")
emit()

# ---------------------------------------------------------------- inverse trig
emit("// ===== atan(a/b) = atan(c_j) + atan(t), c_j = j/16, t = (a - c b)/(b + c a) =====")
at_d, at_f, at_dd = [], [], []
for j in range(17):
    A = mp.atan(mp.mpf(j) / 16)
    at_d.append(d(A))
    at_f += split(A, f, 2)
    at_dd += split(A, d, 2)
arr_u64("CRM_ATANI_T", sum((q126(mp.atan(mp.mpf(j) / 16)) for j in range(17)), []),
        "atan(j/16) in Q126, j = 0..16")
arr_u64("CRM_ATANI_C", sum((q126(mp.mpf((-1) ** k) / (2 * k + 1)) for k in range(1, 12)), []),
        "(-1)^k/(2k+1) in Q126, k = 1..11")
arr_u64("CRM_ATANI_PIO2", q126(mp.pi / 2), "pi/2 in Q126")
arr_u64("CRM_HYPI_E", sum((q126(1 / mp.factorial(k + 1)) for k in range(13)), []),
        "1/(k+1)! in Q126, k = 0..12 (expm1 x = x sum x^k/(k+1)!)")
arr_d("CRM_ATAN_T17_D", at_d + [mp.mpf(0)], "atan(j/16), j = 0..16 (+ padding)")
arr_f("CRM_ATAN_T17_DF", at_f + [mp.mpf(0), mp.mpf(0)], "atan(j/16) (hi, lo) floats")
arr_d("CRM_ATAN_T17_DD", at_dd, "atan(j/16) as double-double")
pio2 = mp.pi / 2
const_d("CRM_PIO2_D_HI", d(pio2))
const_d("CRM_PIO2_D_LO", d(pio2 - d(pio2)))
const_f("CRM_PIO2_F_HI", f(pio2))
const_f("CRM_PIO2_F_LO", f(pio2 - f(pio2)))
const_d("CRM_PI_D_HI", d(mp.pi))
const_d("CRM_PI_D_LO", d(mp.pi - d(mp.pi)))
const_f("CRM_PI_F_HI", f(mp.pi))
const_f("CRM_PI_F_LO", f(mp.pi - f(mp.pi)))
arr_d("CRM_ATAN_TAYLOR_D", [d(mp.mpf((-1) ** k) / (2 * k + 1)) for k in range(8)],
      "(-1)^k/(2k+1), k = 0..7")
atdd = []
for k in range(14):
    atdd += split(mp.mpf((-1) ** k) / (2 * k + 1), d, 2)
arr_d("CRM_ATAN_TAYLOR_DD", atdd, "(-1)^k/(2k+1), k = 0..13, double-double")
emit()

# ---------------------------------------------------------------- binary64 pair
emit("// ===== binary64 exp2: x = k + (256 i1 + 16 i2 + i3)/4096 + R (Sec. II.B) =====")
vals = []
for a, div in ((1, 16), (2, 256), (3, 4096)):
    for i in range(16):
        vals += split(mp.power(2, mp.mpf(i) / div), d, 2)
arr_d("CRM_EXP2D_T", vals, "2^(i/16), 2^(i/256), 2^(i/4096) (i = 0..15) as double-double, one table each")
coefs = []
for k in range(1, 9):
    coefs += split(LN2 ** k / mp.factorial(k), d, 2)
arr_d("CRM_EXP2D_C", coefs, "(ln 2)^k/k!, k = 1..8, double-double")


def limbs192(v, frac_bits):
    """floor(v 2^frac_bits) as three 64-bit limbs (little endian)"""
    with mp.workprec(400):
        N = int(mp.floor(v * mp.mpf(2) ** frac_bits))
    assert 0 <= N < 2 ** 192
    return [(N >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(3)]


def arr_u64(name, vals, comment):
    emit(f"// {comment}")
    emit(f"CRM_TABLE unsigned long long {name}[{len(vals)}] = {{")
    for i in range(0, len(vals), 3):
        emit("  " + ", ".join(f"0x{v:016X}ull" for v in vals[i:i + 3]) + ",")
    emit("};")


emit("// ----- exact (192-bit fixed-point) slow path constants -----")
fx = []
for a, div in ((1, 16), (2, 256), (3, 4096)):
    for i in range(16):
        fx += limbs192(mp.power(2, mp.mpf(i) / div), 190)  # Q2.190
arr_u64("CRM_EXP2_FX_T", fx, "2^(i/16), 2^(i/256), 2^(i/4096) (i = 0..15) as floor(v 2^190), 3 limbs each")
arr_u64("CRM_LN2_FX", limbs192(LN2, 191), "ln 2 as floor(ln2 2^191)")
# constants of the exact tiers of binary64 e^x, 10^x (x log2 b) and log2, log10 (ln x / ln b)
arr_u64("CRM_LOG2E_FX", limbs192(LOG2E, 190), "log2 e as floor(log2(e) 2^190)")
arr_u64("CRM_LOG2_10_FX", limbs192(LOG2_10, 189), "log2 10 as floor(log2(10) 2^189)")
arr_u64("CRM_INV_LN2_FX", limbs192(1 / LN2, 190), "1/ln 2 as floor(2^190 / ln 2)")
arr_u64("CRM_INV_LN10_FX", limbs192(1 / mp.log(10), 190), "1/ln 10 as floor(2^190 / ln 10)")
lfx = []
for j in range(128):
    lfx += limbs192(mp.log(1 + mp.mpf(j) / 128), 191)
arr_u64("CRM_LOG_FX_T", lfx, "log(1 + j/128), j = 0..127, as floor(v 2^191)")
emit("// ===== binary64 log: log x = e ln2 + L_j + log1p(m rcp_j - 1), rcp_j ~ 256/j =====")
rc, Lv = [], []
for j in range(192, 385):
    r = d(mp.mpf(256) / j)
    rc.append(r)
    Lv += split(-mp.log(r), d, 2)
arr_d("CRM_LOGD_RCP", rc, "rcp_j ~ 256/j (j = 192..384), doubles")
arr_d("CRM_LOGD_L", Lv, "-log(rcp_j) as double-double")
lc = []
for k in range(1, 13):
    lc += split(mp.mpf((-1) ** (k + 1)) / k, d, 2)
arr_d("CRM_LOGD_C", lc, "(-1)^(k+1)/k, k = 1..12, double-double")
emit()

emit("// ===== binary64 exp2, FP64-free main path (128-bit fixed point) =====")


def q_round(v, frac_bits, bits):
    """round(v 2^frac_bits) as an integer below 2^bits"""
    with mp.workprec(400):
        N = int(mp.nint(v * mp.mpf(2) ** frac_bits))
    assert 0 <= N < 2 ** bits
    return N


def arr_u64_pairs(name, vals, comment):
    emit(f"// {comment}")
    emit(f"CRM_TABLE unsigned long long {name}[{len(vals)}] = {{")
    for i in range(0, len(vals), 2):
        emit("  " + ", ".join(f"0x{v:016X}ull" for v in vals[i:i + 2]) + ",")
    emit("};")


ti = []
for i in range(1024):
    N = q_round(mp.power(2, mp.mpf(i) / 1024), 124, 128)
    ti += [N & 0xFFFFFFFFFFFFFFFF, N >> 64]
arr_u64_pairs("CRM_EXP2I_T", ti, "2^(i/1024), i = 0..1023, as round(v 2^124): (low, high) 64-bit words")
for k in range(1, 7):
    emit(f"#define CRM_EXP2I_A{k} 0x{q_round(LN2 ** k / mp.factorial(k), 64, 64):016X}ull  // (ln 2)^{k}/{k}! 2^64")
for k in (5, 6):
    emit(f"#define CRM_EXP2I_A{k}_32 0x{q_round(LN2 ** k / mp.factorial(k), 32, 32):08X}u  // (ln 2)^{k}/{k}! 2^32")
emit()

emit("// ===== binary64 log, FP64-free main path (128-bit fixed point) =====")
li, lr = [], []
for j in range(192, 385):
    R = int(mp.nint(mp.mpf(2) ** 9 * 256 / j))
    lr.append(R)
    with mp.workprec(400):
        N = int(mp.nint(-mp.log(mp.mpf(R) / 512) * mp.mpf(2) ** 116))
    N &= (1 << 128) - 1  # two's complement
    li += [N & 0xFFFFFFFFFFFFFFFF, N >> 64]
arr_u64_pairs("CRM_LOGI_L", li, "-log(R_j/2^9), j = 192..384, as round(v 2^116), two's complement (low, high)")
emit("// R_j = round(2^9 256/j), j = 192..384, and a zero pad (whole 32-bit words)")
lr.append(0)
emit(f"CRM_TABLE unsigned short CRM_LOGI_R[{len(lr)}] = {{")
for i in range(0, len(lr), 12):
    emit("  " + ", ".join(str(v) for v in lr[i:i + 12]) + ",")
emit("};")
for n in range(8):
    with mp.workprec(400):
        N = int(mp.nint(mp.mpf((-1) ** n) / (n + 3) * mp.mpf(2) ** 63))
    emit(f"#define CRM_LOGI_C{n} ((int64_t){N}ll)  // (-1)^{n}/{n + 3} 2^63")
for n in range(4, 8):
    with mp.workprec(400):
        N = int(mp.nint(mp.mpf((-1) ** n) / (n + 3) * mp.mpf(2) ** 31))
    emit(f"#define CRM_LOGI_C{n}_32 ((int32_t){N})  // (-1)^{n}/{n + 3} 2^31")
with mp.workprec(400):
    N = int(mp.nint(LN2 * mp.mpf(2) ** 116))
emit(f"#define CRM_LOGI_LN2_LO 0x{N & 0xFFFFFFFFFFFFFFFF:016X}ull  // ln 2 2^116, low word")
emit(f"#define CRM_LOGI_LN2_HI 0x{N >> 64:016X}ull  // high word")
# log2(e) in Q125 and log2(10) in Q124 (both below 2^126), for the binary32 expf / exp10f
# integer tier
for nm, v, q in (("LOG2E_Q125", LOG2E, 125), ("LOG2_10_Q124", LOG2_10, 124)):
    with mp.workprec(400):
        N = int(mp.nint(v * mp.mpf(2) ** q))
    assert N < 2 ** 126
    emit(f"#define CRM_EXPI_{nm}_LO 0x{N & 0xFFFFFFFFFFFFFFFF:016X}ull  // low word")
    emit(f"#define CRM_EXPI_{nm}_HI 0x{N >> 64:016X}ull  // high word")
# 1/ln 2 and 1/ln 10 in Q126 (both below 2), for the binary32 log2f / log10f integer tier
for nm, v in (("INV_LN2", 1 / LN2), ("INV_LN10", 1 / mp.log(10))):
    with mp.workprec(400):
        N = int(mp.nint(v * mp.mpf(2) ** 126))
    assert N < 2 ** 127
    emit(f"#define CRM_LOGI_{nm}_Q126_LO 0x{N & 0xFFFFFFFFFFFFFFFF:016X}ull  // {nm.lower()} 2^126, low word")
    emit(f"#define CRM_LOGI_{nm}_Q126_HI 0x{N >> 64:016X}ull  // high word")
emit()

emit("// ===== end =====")

text = "\n".join(lines) + "\n"
with open(OUT, "w") as fh:
    fh.write(text)
print(f"wrote {OUT} ({len(lines)} lines)")
