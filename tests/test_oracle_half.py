"""The oracle's 16-bit formats (IEEE binary16 and bfloat16), pinned against mpmath at 400
bits rounded by an independent rounding routine written here from the formats'
definitions (precision p, minimum exponent emin, gradual underflow, overflow by the
rounding direction, IEEE 754 Sec. 4.3).  Sampled inputs for every binary32 function's
formula, all four rounding directions, all 2^16 binary16 inputs of expf and logf to
nearest, and all 2^16 bfloat16 inputs of expf, exp2f and exp10f."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

mp.mp.prec = 400
FMT = {"f16": (11, -14, 15), "bf16": (8, -126, 127)}
MPF = {"expf": mp.exp, "exp2f": lambda v: mp.power(2, v), "exp10f": lambda v: mp.power(10, v),
       "expm1f": mp.expm1, "logf": mp.log, "log2f": lambda v: mp.log(v, 2), "log10f": mp.log10,
       "log1pf": mp.log1p, "sinf": mp.sin, "cosf": mp.cos, "tanf": mp.tan, "asinf": mp.asin,
       "acosf": mp.acos, "atanf": mp.atan, "sinhf": mp.sinh, "coshf": mp.cosh, "tanhf": mp.tanh,
       "rsqrtf": lambda v: 1 / mp.sqrt(v)}
DOMAIN = {"logf": (0, None), "log2f": (0, None), "log10f": (0, None), "rsqrtf": (0, None),
          "log1pf": (-1, None), "asinf": (-1, 1), "acosf": (-1, 1),
          # beyond these, -1 + e^x and tanh x lie within 2^-400 of +-1, below mpmath's
          # working precision here (the saturated ranges are pinned in the directed tests)
          "expm1f": (-40, None), "tanhf": (-40, 40)}


def decode(b, fmt):
    p, emin, emax = FMT[fmt]
    ew = 16 - p
    s, e, m = b >> 15, (b >> (p - 1)) & ((1 << ew) - 1), b & ((1 << (p - 1)) - 1)
    if e == (1 << ew) - 1:
        return None
    v = mp.mpf(m) * mp.mpf(2) ** (emin - p + 1) if e == 0 else \
        mp.mpf(m + (1 << (p - 1))) * mp.mpf(2) ** (e - (1 << (ew - 1)) + 1 - p + 1)
    return -v if s else v


def encode(v, fmt, mode):
    """v (an mpf) rounded to the format in the direction mode, as a 16-bit pattern."""
    p, emin, emax = FMT[fmt]
    bias = (1 << (15 - p)) - 1
    s = 0x8000 if v < 0 else 0
    a = abs(v)
    if a == 0:
        return s
    away = (mode == "ru" and not s) or (mode == "rd" and s)
    e = int(mp.floor(mp.log(a, 2)))
    while mp.mpf(2) ** e > a:
        e -= 1
    while mp.mpf(2) ** (e + 1) <= a:
        e += 1
    q = max(e, emin) - (p - 1)
    sc = a / mp.mpf(2) ** q
    n = int(mp.floor(sc))
    fr = sc - n
    if mode == "rn":
        n += 1 if (fr > 0.5 or (fr == 0.5 and n % 2 == 1)) else 0
    elif away and fr > 0:
        n += 1
    inf = ((2 * bias + 1) << (p - 1))
    if n == 0:
        return s
    val_e = q + n.bit_length() - 1  # exponent of the rounded value
    if val_e > emax:
        return s | (inf if (mode == "rn" or away) else inf - 1)
    if n < (1 << (p - 1)):
        return s | n  # subnormal
    if n == (1 << p):  # carried into the next binade
        n >>= 1
        q += 1
    return s | (((q + p - 1 + bias) << (p - 1)) + n - (1 << (p - 1)))


def sample(func, fmt, k, seed):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 1 << 16, 6 * k).astype(np.uint16)
    keep = []
    lo, hi = DOMAIN.get(func, (None, None))
    for b in bits:
        v = decode(int(b), fmt)
        if v is None or v == 0 or (lo is not None and v <= lo) or (hi is not None and v >= hi):
            continue
        keep.append(int(b))
        if len(keep) == k:
            break
    return np.array(keep, dtype=np.uint16)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("func", sorted(MPF))
def test_half_formats_against_mpmath(func, fmt):
    x = sample(func, fmt, 60, hash((func, fmt)) & 0xFFFF)
    for mode in ("rn", "rd", "ru", "rz"):
        got = O.eval_bits16(func, x, fmt, mode)
        for i, b in enumerate(x):
            want = encode(MPF[func](decode(int(b), fmt)), fmt, mode)
            assert int(got[i]) == want, (func, fmt, mode, hex(int(b)), hex(int(got[i])), hex(want))


@pytest.mark.parametrize("func", ["expf", "logf"])
def test_all_binary16_inputs_to_nearest(func):
    x = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    got = O.eval_bits16(func, x, "f16")
    for b in range(1 << 16):
        v = decode(b, "f16")
        if v is None or v == 0 or (func == "logf" and v < 0):
            continue
        assert int(got[b]) == encode(MPF[func](v), "f16", "rn"), (func, hex(b))


@pytest.mark.parametrize("func", ["expf", "exp2f", "exp10f"])
def test_all_bfloat16_inputs_of_the_exp_family(func):
    """bfloat16 has binary32's exponent range, so its saturation cut-offs (overflow to inf,
    underflow to +0, the band of subnormal results) are those of the format's own range,
    not binary64's; every input, to nearest and toward -inf."""
    x = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    for mode in ("rn", "rd"):
        got = O.eval_bits16(func, x, "bf16", mode)
        for b in range(1 << 16):
            v = decode(b, "bf16")
            if v is None:
                continue
            assert int(got[b]) == encode(MPF[func](v), "bf16", mode), (func, mode, hex(b))


def test_half_specials_and_sincos():
    x = np.array([0x0000, 0x8000, 0x7C00, 0xFC00, 0x7E00], dtype=np.uint16)  # +-0, +-inf, NaN
    assert [hex(v) for v in O.eval_bits16("expf", x)] == ["0x3c00", "0x3c00", "0x7c00", "0x0", "0x7e00"]
    assert [hex(v) for v in O.eval_bits16("logf", x)] == ["0xfc00", "0xfc00", "0x7c00", "0x7e00", "0x7e00"]
    xs = sample("sinf", "bf16", 40, 7)
    sc = O.eval_bits16("sincosf", xs, "bf16")
    assert np.array_equal(sc[0], O.eval_bits16("sinf", xs, "bf16"))
    assert np.array_equal(sc[1], O.eval_bits16("cosf", xs, "bf16"))
