"""The paper's applications built on the library (Sec. III.A), on the GPU through the C ABI:

* complex expf, logf, sinf: every component within one float of the oracle's correctly rounded
  component (so within 1.5 ulp of the exact value, inside the paper's 2 ulp), on seeded inputs
  over [-40, 40]^2 and on the hard regions (near |z| = 1 for clog, near multiples of pi/2, tiny
  and zero parts);
* spectral interpolation by a brute-force DFT: the sum of x[n] cos and x[n] sin of the phases
  theta_n (formed the same way on the host), with sin and cos taken from the oracle, summed
  exactly (math.fsum); the device's sums must agree within 2^-40 of sum |x[n]| -- far below one
  ulp of any single term, so a single misrounded sine or cosine would show.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    yield


def complex_inputs(func, seed, n=60000):
    rng = np.random.default_rng(seed)
    z = [rng.uniform(-40, 40, (n, 2))]
    if func == "clogf":
        t = rng.uniform(0, 2 * np.pi, 4000)
        r = 1.0 + rng.integers(-8, 9, 4000) * 2.0 ** -24
        z += [np.stack([r * np.cos(t), r * np.sin(t)], axis=1),
              np.stack([rng.uniform(-1, 1, 2000) * 2.0 ** rng.uniform(-58, 0, 2000),
                        rng.uniform(-1, 1, 2000) * 2.0 ** rng.uniform(-140, 5, 2000)], axis=1),
              np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0], [-3.0, 0.0], [-3.0, -0.0], [40.0, 2e-45]])]
    else:
        k = rng.integers(-25, 26, 4000)
        near = (k * np.pi / 2).astype(np.float32).astype(np.float64)
        z += [np.stack([rng.uniform(-40, 40, 4000), near], axis=1),
              np.stack([near, rng.uniform(-40, 40, 4000)], axis=1),
              np.stack([rng.uniform(-40, 40, 2000), rng.uniform(-1, 1, 2000) * 2.0 ** rng.uniform(-149, -20, 2000)],
                       axis=1),
              np.array([[0.0, 0.0], [0.0, 3.0], [3.0, 0.0], [-0.0, -1e-30], [-40.0, 40.0], [40.0, -40.0]])]
    return np.concatenate(z).astype(np.float32)


def float_distance(a, b):
    """number of binary32 values between a and b (uint32 patterns; +0 and -0 coincide)"""
    def key(u):
        u = u.astype(np.int64)
        return np.where(u >= 0x80000000, 0x80000000 - u, u)
    return np.abs(key(a) - key(b))


@pytest.mark.parametrize("func", ["cexpf", "clogf", "csinf"])
def test_complex_within_one_float_of_correct_rounding(func):
    z = complex_inputs(func, 17 + len(func))
    zt = torch.from_numpy(z.reshape(-1)).cuda().view(torch.complex64)
    got = crm.eval_complex(func, zt).view(torch.float32).cpu().numpy().view(np.uint32)
    ref = O.eval_complex(func, z.view(np.uint32).reshape(-1))
    d = float_distance(got, ref)
    bad = np.nonzero(d > 1)[0]
    assert bad.size == 0, [(z.reshape(-1)[2 * (i // 2):2 * (i // 2) + 2].tolist(), i % 2, hex(int(got[i])),
                            hex(int(ref[i]))) for i in bad[:5]]
    # and mostly the correctly rounded value itself
    assert (d == 0).mean() > 0.99, (d == 0).mean()


def dft_phase_host(f, n, lg):
    """theta_n = RN(RN(u) 2^-w RN(2 pi)), u 2^-w = frac(f n / 2^lg), as in the library"""
    fb = np.float32(f).view(np.uint32)
    if fb & 0x7FFFFFFF == 0:
        return np.zeros(n.size, dtype=np.float32)
    mf = np.uint64((int(fb) & 0x007FFFFF) | 0x00800000)
    w = lg - ((int(fb) >> 23) - 150)
    if w <= 0:
        return np.zeros(n.size, dtype=np.float32)
    u = mf * n.astype(np.uint64)
    if w < 64:
        u &= np.uint64((1 << w) - 1)
    p = u.astype(np.float32) * np.float32(2.0 ** -w)
    return p * np.float32(float.fromhex("0x1.921fb6p+2"))


@pytest.mark.parametrize("lg", [10, 14])
def test_spectral_dft_matches_exact_sums(lg):
    N = 1 << lg
    rng = np.random.default_rng(lg)
    t = np.arange(N)
    x = (np.sin(2 * np.pi * 37.3 * t / N) + 0.5 * np.cos(2 * np.pi * 101.7 * t / N) +
         0.1 * rng.standard_normal(N)).astype(np.float32)
    freq = np.concatenate([rng.uniform(0, N, 40), [0.0, 37.3, 101.7, 0.5, N - 0.25, 2.0 ** -10, 3.0]]).astype(np.float32)
    got = crm.spectral_dft(torch.from_numpy(x).cuda(), torch.from_numpy(freq).cuda()).cpu().numpy()
    nidx = np.arange(N, dtype=np.uint64)
    tol = 2.0 ** -40 * float(np.abs(x.astype(np.float64)).sum())
    for m, f in enumerate(freq):
        th = dft_phase_host(f, nidx, lg)
        sc = O.eval_bits("sincosf", th.view(np.uint32)).view(np.float32)
        xs = x.astype(np.float64)
        re = math.fsum(xs * sc[1].astype(np.float64))
        im = math.fsum(-xs * sc[0].astype(np.float64))
        assert abs(got[m].real - re) <= tol and abs(got[m].imag - im) <= tol, (f, got[m], re, im, tol)


def test_spectral_dft_rejects_bad_sizes():
    x = torch.ones(1000, device="cuda")
    f = torch.ones(3, device="cuda")
    with pytest.raises(crm.CrmError):
        crm.spectral_dft(x, f)
