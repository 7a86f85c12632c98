"""Pins of the oracle's complex components (cexp, clog, csin; the paper's application of
Sec. III.A) against mpmath at 320 bits, each component rounded to nearest binary32 by the
independent integer rounding of test_oracle.rn_bits, on seeded inputs over [-40, 40]^2,
near |z| = 1 (clog's cancellation), near multiples of pi/2, with tiny and zero parts."""
import numpy as np
import pytest

from oracle import oracle as O

mpmath = pytest.importorskip("mpmath")
from test_oracle import F32, rn_bits  # noqa: E402


def inputs(func, seed):
    rng = np.random.default_rng(seed)
    z = [rng.uniform(-40, 40, (300, 2))]
    z.append(np.stack([rng.uniform(-2, 2, 100), rng.uniform(-2, 2, 100)], axis=1))
    if func == "clogf":  # |z| = 1 up to a few ulps: log|z| cancels
        t = rng.uniform(0, 2 * np.pi, 100)
        r = 1.0 + rng.integers(-4, 5, 100) * 2.0 ** -24
        z.append(np.stack([r * np.cos(t), r * np.sin(t)], axis=1))
        z.append(np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0], [-3.0, 1e-30], [-3.0, -1e-30],
                           [1e-30, 40.0], [40.0, 1e-38], [-40.0, 2e-45]]))
    else:
        k = rng.integers(-25, 26, 60)
        near = (k * np.pi / 2).astype(np.float32).astype(np.float64)
        z.append(np.stack([rng.uniform(-40, 40, 60), near], axis=1))
        z.append(np.stack([near, rng.uniform(-40, 40, 60)], axis=1))
        z.append(np.array([[0.0, 0.0], [0.0, 3.0], [3.0, 0.0], [-0.0, -1e-30], [1e-30, 2e-45], [-40.0, 40.0]]))
    return np.concatenate(z).astype(np.float32)


def ref_bits(func, z):
    out = []
    with mpmath.workprec(320):
        for x, y in z.astype(np.float64):
            x, y = mpmath.mpf(float(x)), mpmath.mpf(float(y))
            if func == "cexpf":
                re, im = mpmath.exp(x) * mpmath.cos(y), mpmath.exp(x) * mpmath.sin(y)
            elif func == "csinf":
                re, im = mpmath.sin(x) * mpmath.cosh(y), mpmath.cos(x) * mpmath.sinh(y)
            else:
                re, im = mpmath.log(x * x + y * y) / 2, mpmath.atan2(y, x)
            out += [rn_bits(re, F32) & 0x7FFFFFFF if re == 0 else rn_bits(re, F32),
                    rn_bits(im, F32) & 0x7FFFFFFF if im == 0 else rn_bits(im, F32)]
    return np.array(out, dtype=np.uint32)


@pytest.mark.parametrize("func", ["cexpf", "clogf", "csinf"])
def test_complex_components_match_mpmath(func):
    z = inputs(func, 5 + len(func))
    got = O.eval_complex(func, z.view(np.uint32))
    ref = ref_bits(func, z)
    zero = (got & 0x7FFFFFFF) == 0  # the sign of an exact zero part is not specified
    bad = np.nonzero((got != ref) & ~(zero & ((ref & 0x7FFFFFFF) == 0)))[0]
    assert bad.size == 0, [(z.reshape(-1)[2 * (i // 2):2 * (i // 2) + 2].tolist(), i % 2, hex(int(got[i])),
                            hex(int(ref[i]))) for i in bad[:5]]


def test_complex_identities():
    rng = np.random.default_rng(4)
    z = rng.uniform(-40, 40, (200, 2)).astype(np.float32)
    zc = z.copy()
    zc[:, 1] = -zc[:, 1]
    for func in ("cexpf", "csinf", "clogf"):  # f(conj z) = conj f(z)
        a = O.eval_complex(func, z.view(np.uint32)).view(np.float32).reshape(-1, 2)
        b = O.eval_complex(func, zc.view(np.uint32)).view(np.float32).reshape(-1, 2)
        assert np.array_equal(a[:, 0], b[:, 0]) and np.array_equal(a[:, 1], -b[:, 1]), func
    # cexp(x + 0i) = RN(e^x), clog(x + 0i) = RN(log x) for x > 0: the real functions' results
    x = rng.uniform(0.01, 40, 100).astype(np.float32)
    zr = np.stack([x, np.zeros_like(x)], axis=1)
    assert np.array_equal(O.eval_complex("cexpf", zr.view(np.uint32)).reshape(-1, 2)[:, 0],
                          O.eval_bits("expf", x.view(np.uint32)))
    assert np.array_equal(O.eval_complex("clogf", zr.view(np.uint32)).reshape(-1, 2)[:, 0],
                          O.eval_bits("logf", x.view(np.uint32)))
