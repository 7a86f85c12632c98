"""GPU parity for the binary64 pair (exp2, log): the FP64-free fixed-point main path
(the default form), the double-double main path (the plain form) and the exact 192-bit
integer slow path, each checked bit for bit against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    crm.set_force_slow(False)
    yield
    crm.set_force_slow(False)


def run64(func, x, off=0, form=None):
    xb = np.ascontiguousarray(x, dtype=np.float64)
    buf = torch.zeros(xb.size + off + 2, dtype=torch.float64, device="cuda")
    buf[off:off + xb.size] = torch.from_numpy(xb).cuda()
    out = torch.full((xb.size + 2,), float("nan"), dtype=torch.float64, device="cuda")
    crm.eval_into(func, buf[off:off + xb.size], out[:xb.size], form=form)
    torch.cuda.synchronize()
    return out[:xb.size].cpu().numpy().view(np.uint64)


def inputs(func, rng):
    if func == "exp2":
        parts = [W.f64_uniform(-1075, 1024, 40000, rng), W.f64_uniform(-20, 20, 40000, rng),
                 W.f64_uniform(-1080, -1020, 5000, rng), np.arange(-1080, 1030, dtype=np.float64),
                 rng.uniform(-1, 1, 5000) * np.exp2(rng.uniform(-1070, -5, 5000)),
                 np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1023.999, -1074.5, -1075.0, -1074.999]),
                 rng.uniform(-1, 1, 5000) * np.exp2(rng.uniform(-80, -40, 5000)),
                 np.nextafter(np.arange(-1075, 1024, dtype=np.float64), np.inf),
                 np.nextafter(np.arange(-1075, 1024, dtype=np.float64), -np.inf)]
    else:
        parts = [W.f64_positive_bits(40000, rng), W.f64_uniform(0.125, 8.0, 40000, rng),
                 1.0 + rng.uniform(-1, 1, 5000) * np.exp2(rng.uniform(-52, -3, 5000)),
                 np.exp2(rng.uniform(-1074, -1022, 3000)),
                 1.0 + np.arange(-3000, 3000) * 2.0 ** -52, np.exp2(np.arange(-1074, 1024, dtype=np.float64)),
                 rng.integers(1, 1 << 52, 3000, dtype=np.uint64).view(np.float64),
                 np.array([1.0, 0.0, -0.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, 1.7976931348623157e308,
                           2.2250738585072014e-308])]
    return np.concatenate(parts)


@pytest.mark.parametrize("form", ["plain", "df"])
@pytest.mark.parametrize("func", ["exp2", "log"])
def test_f64_parity(func, form):
    x = inputs(func, W.rng_for(5, func))
    got = run64(func, x, form=form)
    ref = O.eval_bits(func, x.view(np.uint64))
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, [(x[i], hex(int(got[i])), hex(int(ref[i]))) for i in bad[:6]]


@pytest.mark.parametrize("func", ["exp2", "log"])
def test_f64_forced_exact_path(func):
    """every lane through the 192-bit integer slow path"""
    x = inputs(func, W.rng_for(5, func, salt=2))[::3]
    crm.stats_reset()
    crm.set_force_slow(True)
    try:
        got = run64(func, x, off=1)
    finally:
        crm.set_force_slow(False)
    ref = O.eval_bits(func, x.view(np.uint64))
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, [(x[i], hex(int(got[i])), hex(int(ref[i]))) for i in bad[:6]]
    assert crm.stats()["unresolved_total"] == 0
