"""Directed rounding in the oracle (IEEE 754 Sec. 4.3: toward -inf, +inf, zero), pinned
without the oracle's own arithmetic: the round-to-nearest results (pinned elsewhere) and
mpmath at 200 bits fix both neighbours of every value, exact results are listed by hand,
and the overflow / underflow / saturation cases follow the standard's definitions.  The
library itself rounds to nearest only (Sec. III.C); these modes extend the oracle for the
directed-rounding kernels."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

mp.mp.prec = 500  # tiny |x|: f(x) - x can be 2^-300 of x
F32 = [f for f in W.F32_FUNCS if f != "sincosf"]
MPF = {"expf": mp.exp, "exp2f": lambda v: mp.power(2, v), "exp10f": lambda v: mp.power(10, v),
       "expm1f": mp.expm1, "logf": mp.log, "log2f": lambda v: mp.log(v, 2), "log10f": mp.log10,
       "log1pf": mp.log1p, "sinf": mp.sin, "cosf": mp.cos, "tanf": mp.tan, "asinf": mp.asin,
       "acosf": mp.acos, "atanf": mp.atan, "sinhf": mp.sinh, "coshf": mp.cosh, "tanhf": mp.tanh,
       "rsqrtf": lambda v: 1 / mp.sqrt(v)}
MAXF = 0x7F7FFFFF


def f32(bits):
    return np.asarray(bits, dtype=np.uint32).view(np.float32)


def neighbours(rn_bits, v):
    """(RD, RU) bit patterns of the real v from its round-to-nearest rn_bits (finite,
    nonzero): RN is one of the two floats around v, or v itself."""
    r = f32([rn_bits])[0]
    rv = mp.mpf(float(r))
    if rv == v:
        return rn_bits, rn_bits
    up = np.nextafter(r, np.float32(np.inf)).view(np.uint32)
    dn = np.nextafter(r, np.float32(-np.inf)).view(np.uint32)
    return (rn_bits, int(up)) if v > rv else (int(dn), rn_bits)


@pytest.mark.parametrize("func", F32)
def test_directed_against_mpmath(func):
    rng = W.rng_for(3, func, salt=21)
    x = W.domain_bits(func, 400, rng, special_frac=0.0)
    rn = O.eval_bits(func, x)
    got = {m: O.eval_bits(func, x, mode=m) for m in ("rd", "ru", "rz")}
    checked = 0
    for i in range(x.size):
        r = f32([rn[i]])[0]
        if not np.isfinite(r) or r == 0 or abs(r) < 2.0**-126 or (int(rn[i]) & 0x7FFFFFFF) == MAXF:
            continue
        v = MPF[func](mp.mpf(float(f32([x[i]])[0])))
        rd, ru = neighbours(int(rn[i]), v)
        rz = rd if v > 0 else ru
        assert (int(got["rd"][i]), int(got["ru"][i]), int(got["rz"][i])) == (rd, ru, rz), (func, hex(int(x[i])))
        checked += 1
    assert checked > 300


@pytest.mark.parametrize("func", ["exp2", "log"])
def test_directed_binary64_brackets(func):
    rng = W.rng_for(3, func, salt=22)
    x = (W.f64_uniform(-20, 20, 200, rng) if func == "exp2" else W.f64_uniform(0.125, 8.0, 200, rng)).view(np.uint64)
    rn, rd, ru, rz = (O.eval_bits(func, x, mode=m) for m in ("rn", "rd", "ru", "rz"))
    for i in range(x.size):
        xv = mp.mpf(float(x[i:i + 1].view(np.float64)[0]))
        v = mp.power(2, xv) if func == "exp2" else mp.log(xv)
        r = rn[i:i + 1].view(np.float64)[0]
        if mp.mpf(float(r)) == v:
            exp = (rn[i], rn[i])
        else:
            up = np.nextafter(r, np.inf).view(np.uint64)
            dn = np.nextafter(r, -np.inf).view(np.uint64)
            exp = (rn[i], up) if v > mp.mpf(float(r)) else (dn, rn[i])
        assert (rd[i], ru[i]) == exp
        assert rz[i] == (rd[i] if v > 0 else ru[i])


def exact_cases():
    c = []
    c += [("exp2f", np.float32(2.0**n), np.float32(n)) for n in range(-149, 128)]
    c += [("exp10f", np.float32(10.0**k), np.float32(k)) for k in range(0, 11)]
    c += [("log2f", np.float32(n), np.float32(2.0**n)) for n in range(-149, 128)]
    c += [("log10f", np.float32(k), np.float32(10.0**k)) for k in range(1, 11)]
    c += [("rsqrtf", np.float32(2.0**-j), np.float32(4.0**j)) for j in range(-74, 64)]
    return c


def test_exact_results_in_every_mode():
    """exp2 of integers, 10^k, log2 of powers of two, log10 of powers of ten and rsqrt of
    powers of four are exact: every mode returns the value itself."""
    for func, y, x in exact_cases():
        xb = np.array([x], dtype=np.float32).view(np.uint32)
        want = int(np.array([y], dtype=np.float32).view(np.uint32)[0])
        for m in ("rn", "rd", "ru", "rz"):
            assert int(O.eval_bits(func, xb, mode=m)[0]) == want, (func, float(x), m)
    for n in (-1074, -1022, -1, 0, 1, 52, 1023):
        xb = np.array([float(n)]).view(np.uint64)
        want = int(np.array([2.0**n]).view(np.uint64)[0])
        assert all(int(O.eval_bits("exp2", xb, mode=m)[0]) == want for m in ("rd", "ru", "rz"))


def one(func, x, m):
    return int(O.eval_bits(func, np.array([x], dtype=np.float32).view(np.uint32), mode=m)[0])


def test_overflow_underflow_and_saturation():
    INF, ONE, BELOW1, SB = 0x7F800000, 0x3F800000, 0x3F7FFFFF, 0x80000000
    for x in (88.8, 200.0, 1000.0):  # e^x beyond the largest float
        assert (one("expf", x, "rn"), one("expf", x, "rd"), one("expf", x, "ru"), one("expf", x, "rz")) == (INF, MAXF, INF, MAXF)
    for x in (-104.0, -200.0):  # 0 < e^x < 2^-150
        assert (one("expf", x, "rn"), one("expf", x, "rd"), one("expf", x, "ru"), one("expf", x, "rz")) == (0, 0, 1, 0)
    assert (one("sinhf", -200.0, "rd"), one("sinhf", -200.0, "ru"), one("sinhf", -200.0, "rz")) == (SB | INF, SB | MAXF, SB | MAXF)
    assert (one("coshf", 200.0, "rd"), one("coshf", 200.0, "ru")) == (MAXF, INF)
    # tanh x < 1 for finite x; expm1 x > -1
    assert (one("tanhf", 50.0, "rn"), one("tanhf", 50.0, "rd"), one("tanhf", 50.0, "ru"), one("tanhf", 50.0, "rz")) == (ONE, BELOW1, ONE, BELOW1)
    assert (one("tanhf", -50.0, "rd"), one("tanhf", -50.0, "ru"), one("tanhf", -50.0, "rz")) == (SB | ONE, SB | BELOW1, SB | BELOW1)
    assert (one("tanhf", np.inf, "rd"), one("tanhf", -np.inf, "ru")) == (ONE, SB | ONE)
    assert (one("expm1f", -50.0, "rn"), one("expm1f", -50.0, "rd"), one("expm1f", -50.0, "ru"), one("expm1f", -50.0, "rz")) == (SB | ONE, SB | ONE, SB | BELOW1, SB | BELOW1)
    assert one("expm1f", -np.inf, "ru") == SB | ONE  # exactly -1


@pytest.mark.parametrize("func", ["sinf", "tanf", "atanf", "asinf", "sinhf", "tanhf", "expm1f", "log1pf"])
def test_directed_modes_order_and_symmetry(func):
    rng = W.rng_for(3, func, salt=23)
    x = W.domain_bits(func, 300, rng, special_frac=0.0)
    rd, ru, rn, rz = (O.eval_bits(func, x, mode=m).view(np.float32) for m in ("rd", "ru", "rn", "rz"))
    ok = np.isfinite(rd) & np.isfinite(ru)
    assert np.all(rd[ok] <= rn[ok]) and np.all(rn[ok] <= ru[ok])
    step = ru[ok] == rd[ok]
    nxt = np.nextafter(rd[ok], np.float32(np.inf))
    assert np.all(step | (ru[ok] == nxt))
    assert np.array_equal(rz, np.where(rn >= 0, rd, ru))
    if func in ("sinf", "tanf", "atanf", "asinf", "sinhf", "tanhf"):  # odd: RD(f(-x)) = -RU(f(x))
        neg = O.eval_bits(func, x ^ np.uint32(0x80000000), mode="rd").view(np.float32)
        assert np.array_equal(neg.view(np.uint32), (-ru).view(np.uint32))
