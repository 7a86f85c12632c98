"""The host-buffer entry point (crm_eval_host) against the device entry point and the
oracle, bit for bit, on both of its paths: pageable numpy buffers (chunked copies through
the library's staging area; sizes that cross the 2^22-element chunk boundary with a ragged
tail) and page-locked buffers the device addresses directly (evaluated in place), with
misaligned starts for the head and tail handling.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

CHUNK = 1 << 22  # the staging path's chunk (elements)


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    yield


def inputs(func, n, seed):
    rng = W.rng_for(seed, func)
    if func in W.F32_FUNCS:
        return W.domain_bits(func, n, rng).view(np.float32)
    return W.f64_uniform(-20, 20, n, rng) if func == "exp2" else W.f64_uniform(0.125, 8.0, n, rng)


def device_result(func, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = crm.eval(func, xd)
    torch.cuda.synchronize()
    return y.reshape(-1).cpu().numpy()


def bits(a):
    return a.view(np.uint64 if a.dtype == np.float64 else np.uint32)


def check_sample(func, x, got, k=4096, seed=0):
    """a sample of the outputs against the oracle (both rows for sincosf)"""
    n = x.size
    idx = np.unique(np.concatenate([np.arange(min(n, 64)), np.arange(max(0, n - 64), n),
                                    np.random.default_rng(seed).integers(0, n, k)]))
    ref = O.eval_bits(func, bits(x[idx]))
    g = bits(got).reshape(2, n)[:, idx] if func == "sincosf" else bits(got)[idx]
    assert np.array_equal(g, ref), f"{func}: host-buffer results differ from the oracle"


@pytest.mark.parametrize("func,n", [("expf", CHUNK + 4099), ("sincosf", CHUNK + 17), ("tanhf", 3 * CHUNK + 1),
                                    ("exp2", 100003), ("log", CHUNK + 5)])
def test_pageable_buffers_staged(func, n):
    x = inputs(func, n, 11)
    got = crm.eval_host(func, x)
    assert np.array_equal(bits(got), bits(device_result(func, x)))
    check_sample(func, x, got)


@pytest.mark.parametrize("func,n,off", [("expf", CHUNK + 4099, 1), ("sincosf", 100003, 3), ("logf", 1 << 20, 0),
                                        ("acosf", 77777, 2), ("exp2", 65537, 1), ("log", 4097, 0)])
def test_page_locked_buffers_in_place(func, n, off):
    x = inputs(func, n, 12)
    tdt = torch.float64 if x.dtype == np.float64 else torch.float32
    rows = 2 if func == "sincosf" else 1
    hin = torch.empty(n + off, dtype=tdt).pin_memory()
    hout = torch.empty(rows * n + off, dtype=tdt).pin_memory()
    hin[off:] = torch.from_numpy(x)
    xin = hin[off:].numpy()
    yout = hout[off:].numpy()
    crm.eval_host(func, xin, yout)
    assert np.array_equal(bits(yout), bits(device_result(func, x)))
    check_sample(func, x, yout)


def test_empty_host_call():
    x = np.zeros(0, dtype=np.float32)
    assert crm.eval_host("expf", x).size == 0
