"""More binary64 functions (e^x, log2, log10, 10^x) on the fixed-point cores: GPU against the
oracle, bit for bit, in every rounding direction, on seeded domain samples, bands, exact cases
(10^k, log2 of powers of two, log10 of 10^k, log(1); 10^23 is a binary64 midpoint), specials
and the near-midpoint sets of tests/golden/f64_hard (make_f64_hard.py), with the fast path and
with every lane forced through the exact 192-bit slow path."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "f64_hard")
MORE = ["exp", "log2", "log10", "exp10"]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    crm.set_force_slow(False)
    yield
    crm.set_force_slow(False)


def inputs(func):
    rng = W.rng_for(5, func, salt=3)
    if func in ("exp", "exp10"):
        hi, lo = (709.8, -745.2) if func == "exp" else (308.3, -323.7)
        parts = [rng.uniform(lo, hi, 30000), rng.uniform(-20, 20, 20000),
                 rng.uniform(-1, 1, 5000) * np.exp2(rng.uniform(-80, -1, 5000)),
                 rng.uniform(hi - 2, hi + 2, 3000), rng.uniform(lo - 2, lo + 2, 3000),
                 np.arange(-330, 330, dtype=np.float64), np.arange(0, 31, dtype=np.float64),
                 np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-300, -1e-300, 1024.0, -1024.0, 5e-324])]
    else:
        parts = [W.f64_positive_bits(30000, rng), W.f64_uniform(0.125, 8.0, 20000, rng),
                 1.0 + rng.uniform(-1, 1, 5000) * np.exp2(rng.uniform(-52, -3, 5000)),
                 np.exp2(np.arange(-1074, 1024, dtype=np.float64)), 10.0 ** np.arange(0, 40, dtype=np.float64),
                 1.0 + np.arange(-1000, 1000) * 2.0 ** -52,
                 np.array([1.0, 0.0, -0.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, 1.7976931348623157e308])]
    x = np.concatenate(parts).view(np.uint64)
    path = os.path.join(GOLDEN, func + ".txt")
    if os.path.exists(path):
        hard = [int(line.split()[0], 16) for line in open(path) if line.strip() and not line.startswith("#")]
        x = np.concatenate([x, np.array(hard, dtype=np.uint64)])
    return x


def run(func, xb, mode="rn", force=0):
    x = torch.from_numpy(xb.view(np.float64).copy()).cuda()
    crm.set_force_slow(force)
    try:
        crm.stats_reset()
        y = crm.eval(func, x) if mode == "rn" else crm.eval_rm(func, x, mode)
        torch.cuda.synchronize()
        st = crm.stats()
    finally:
        crm.set_force_slow(False)
    return y.cpu().numpy().view(np.uint64), st


@pytest.mark.parametrize("force", [0, 1])
@pytest.mark.parametrize("mode", ["rn", "rd", "ru", "rz"])
@pytest.mark.parametrize("func", MORE)
def test_f64_more_against_oracle(func, mode, force):
    xb = inputs(func)
    got, st = run(func, xb, mode, force)
    ref = O.eval_bits(func, xb, mode=mode)
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, (bad.size, [(xb.view(np.float64)[i], hex(int(got[i])), hex(int(ref[i]))) for i in bad[:6]])
    assert st["unresolved_total"] == 0


def test_f64_more_only_the_fixed_point_form():
    x = torch.ones(8, dtype=torch.float64, device="cuda")
    with pytest.raises(crm.CrmError):
        crm.eval("exp", x, form="plain")
    assert torch.equal(crm.eval("exp", x), torch.full_like(x, float(np.exp(1.0))))
