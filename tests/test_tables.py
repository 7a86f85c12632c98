"""The kernels' generated tables and constants against the mathematics they stand for.

`csrc/crm_tables.h` is written by the generator beside it; these tests read the header as
text and recompute every checked entry here with mpmath at 200 bits, so that a wrong split,
a shifted index or a stale header fails without a GPU.  The exactness conditions that the
double-float evaluators rely on (which sums and products need no error term) are checked
on the stored values themselves.
"""
from __future__ import annotations

import os
import re

import pytest

mp = pytest.importorskip("mpmath")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2605_15547_gb300", "csrc", "crm_tables.h")


def _literal(tok: str):
    tok = tok.strip()
    if tok.startswith(("0x", "-0x")) and "p" in tok:
        return mp.mpf(float.fromhex(tok.rstrip("f")))
    return int(tok.rstrip("uUlL"), 0)


def _read():
    text = open(HEADER).read()
    tables, consts = {}, {}
    for m in re.finditer(r"CRM_TABLE [a-z ]+ (\w+)\[(\d+)\] = \{(.*?)\};", text, re.S):
        body = re.sub(r"//[^\n]*", "", m.group(3))
        vals = [_literal(t) for t in body.replace("\n", " ").split(",") if t.strip()]
        assert len(vals) == int(m.group(2)), m.group(1)
        tables[m.group(1)] = vals
    for m in re.finditer(r"^#define (CRM_\w+) (-?0x[0-9a-fA-Fp.+-]+f?)\b", text, re.M):
        consts[m.group(1)] = _literal(m.group(2))
    return tables, consts


TABLES, CONSTS = _read()


def rn(v, bits=24):
    """Nearest binary number with `bits` significant bits (ties to even)."""
    with mp.workprec(bits):
        return +mp.mpf(v)


def is_multiple(v, g) -> bool:
    q = mp.mpf(v) / g
    return q == mp.floor(q)


def check_split(hi, lo, v, bits=24):
    """(hi, lo) is the two-word split of v: hi = RN(v), lo = RN(v - hi)."""
    assert hi == rn(v, bits), (hi, v)
    assert lo == rn(v - hi, bits), (lo, v - hi)


@pytest.fixture(autouse=True)
def _precision():
    with mp.workprec(200):
        yield


def test_header_parses():
    for name in ("CRM_LN_T193M_DF", "CRM_EXP2_T64U_DF", "CRM_SINCOS_T128_DF", "CRM_TAN_T128_DF",
                 "CRM_ATAN_T17_DF", "CRM_TWO_OVER_PI_W"):
        assert name in TABLES, name
    for name in ("CRM_LN2_F16_HI", "CRM_LN2_F16_LO", "CRM_PIO256_CW1", "CRM_256OPI_F", "CRM_INV_LN2_F_HI"):
        assert name in CONSTS, name


# ---------------------------------------------------------------- log family (double-float)
def test_log_ln2_split_makes_the_exponent_product_exact():
    kh, kl = CONSTS["CRM_LN2_F16_HI"], CONSTS["CRM_LN2_F16_LO"]
    assert is_multiple(kh, mp.mpf(2) ** -15)
    # e ln2_hi + L_hi is a multiple of 2^-17 below 2^7 for every binary32 exponent e
    assert 149 * kh + mp.mpf("0.3") < 128
    assert abs(mp.log(2) - kh - kl) < mp.mpf(2) ** -42


def test_log_table_entries():
    T = TABLES["CRM_LN_T193M_DF"]
    kh = CONSTS["CRM_LN2_F16_HI"]
    rmax_all = mp.mpf(0)
    for j in range(192, 385):
        R, lh, lm, ll = T[4 * (j - 192): 4 * (j - 192) + 4]
        assert R == rn(mp.mpf(256) / j, 9), j
        L = -mp.log(R)
        assert is_multiple(lh, mp.mpf(2) ** -17) and is_multiple(lm, mp.mpf(2) ** -32), j
        assert abs(lm) <= mp.mpf(2) ** -18, j
        assert abs(lh + lm + ll - L) < mp.mpf(2) ** -57, j
        # every e ln2_hi + L_hi is exact in binary32: a multiple of 2^-17 below 2^7
        assert abs(149 * kh) + abs(lh) < 128
        # r = m R - 1 over the cell of j (m in [3/4, 3/2)): r + L_mid exact (below 2^-8 on
        # the grid 2^-32), and Fast2Sum(L_hi, s) valid at e = 0
        lo_m = max(mp.mpf(j) - mp.mpf(1) / 2, 192) / 256
        hi_m = min(mp.mpf(j) + mp.mpf(1) / 2, 384) / 256
        rj = max(abs(lo_m * R - 1), abs(hi_m * R - 1))
        rmax_all = max(rmax_all, rj)
        assert rj + abs(lm) < mp.mpf(2) ** -8, j
        if j == 256:
            assert lh == lm == ll == 0
        else:
            assert abs(lh) > rj + abs(lm) + rj * rj, j
    assert rmax_all < mp.mpf(2) ** -8


def test_log_scale_constants():
    check_split(CONSTS["CRM_INV_LN2_F_HI"], CONSTS["CRM_INV_LN2_F_LO"], 1 / mp.log(2))
    check_split(CONSTS["CRM_INV_LN10_F_HI"], CONSTS["CRM_INV_LN10_F_LO"], 1 / mp.log(10))


# ---------------------------------------------------------------- exp family (double-float)
def test_exp_table_entries():
    T = TABLES["CRM_EXP2_T64U_DF"]
    for i in range(64):
        v = mp.power(2, mp.mpf(i) / 64)
        check_split(T[4 * i], T[4 * i + 1], v)
        check_split(T[4 * i + 2], T[4 * i + 3], v * mp.log(2))
    T16 = TABLES["CRM_EXP2_T16U_DF"]
    for i in range(16):
        v = mp.power(2, mp.mpf(i) / 16)
        check_split(T16[4 * i], T16[4 * i + 1], v)
        check_split(T16[4 * i + 2], T16[4 * i + 3], v * mp.log(2))


# ---------------------------------------------------------------- trigonometric (double-float)
def test_sincos_and_tan_tables():
    SC, TT = TABLES["CRM_SINCOS_T128_DF"], TABLES["CRM_TAN_T128_DF"]
    for j in range(128):
        a = mp.mpf(j) * mp.pi / 256
        check_split(SC[4 * j], SC[4 * j + 1], mp.sin(a))
        check_split(SC[4 * j + 2], SC[4 * j + 3], mp.cos(a))
        check_split(TT[2 * j], TT[2 * j + 1], mp.tan(a))


def test_cody_waite_split_of_pi_over_256():
    c1, c2, c3 = CONSTS["CRM_PIO256_CW1"], CONSTS["CRM_PIO256_CW2"], CONSTS["CRM_PIO256_CW3"]
    assert abs(mp.pi / 256 - c1 - c2 - c3) < mp.mpf(2) ** -83
    # |x| - k C1 exact by one FMA: C1 and |x| >= 2^-7 are multiples of 2^-30 and the
    # reduced |x| - k C1 is below 2^-7, so it has at most 23 significant bits
    assert is_multiple(c1, mp.mpf(2) ** -30)
    k_max = mp.floor(mp.mpf(2) ** 12 * CONSTS["CRM_256OPI_F"]) + 1
    assert k_max < mp.mpf(2) ** 18.36
    # |k C2| < 2^-13 (its FMA split's low word at most 2^-38) and |k C3| < 2^-37.7 for k
    # below k_max: the bounds behind the reduction's error budget
    assert k_max * abs(c2) < mp.mpf(2) ** -13 and k_max * abs(c3) < mp.mpf(2) ** -37.7
    assert k_max * abs(mp.pi / 256 - c1) < mp.mpf(2) ** -12.6  # so |x| - k C1 stays below 2^-7
    assert CONSTS["CRM_256OPI_F"] == rn(256 / mp.pi)
    # |x| RN(256/pi) within 2^-6 of |x| 256/pi for |x| < 2^12
    assert abs(CONSTS["CRM_256OPI_F"] - 256 / mp.pi) * mp.mpf(2) ** 12 < mp.mpf(2) ** -6
    check_split(CONSTS["CRM_PIO256_F_HI"], CONSTS["CRM_PIO256_F_LO"], mp.pi / 256)


def test_two_over_pi_words():
    W = TABLES["CRM_TWO_OVER_PI_W"]
    assert W[0] == W[1] == 0  # two zero words ahead of the fraction bits
    bits = 32 * (len(W) - 2)
    v = 0
    for w in W[2:]:
        v = (v << 32) | w
    with mp.workprec(bits + 64):
        exact = int(mp.floor(2 / mp.pi * mp.mpf(2) ** bits))
    assert v == exact


def test_trig_series_constants():
    check_split(CONSTS["CRM_INV6_F_HI"], CONSTS["CRM_INV6_F_LO"], mp.mpf(1) / 6)
    check_split(CONSTS["CRM_INV3_F_HI"], CONSTS["CRM_INV3_F_LO"], mp.mpf(1) / 3)
    assert CONSTS["CRM_TAN_C5_F"] == rn(mp.mpf(2) / 15)


# ---------------------------------------------------------------- inverse trigonometric
def test_atan_table_and_pi_constants():
    A = TABLES["CRM_ATAN_T17_DF"]
    for j in range(17):
        check_split(A[2 * j], A[2 * j + 1], mp.atan(mp.mpf(j) / 16))
    assert A[34] == A[35] == 0
    check_split(CONSTS["CRM_PIO2_F_HI"], CONSTS["CRM_PIO2_F_LO"], mp.pi / 2)
    check_split(CONSTS["CRM_PI_F_HI"], CONSTS["CRM_PI_F_LO"], mp.pi)
