"""Binary64 exp2 and log where correct rounding is decided: inputs whose exact results lie
closest to a rounding midpoint, and every element of the binary64 workload arrays.

* tests/golden/f64_hard/<func>.txt: the 10^4 inputs (of about 10^7 seeded candidates) whose
  results the oracle finds nearest to a binary64 midpoint (make_f64_hard.py).  Each form,
  and the slow path forced on every lane (all tiers, or its first tier deciding), must give
  the oracle's bits on every one of them; the fast path must send the closest ones (within
  its own error bound of a midpoint) to the slow path.
* tests/golden/f64_full/<label>.txt: digests of the oracle's results on all 2^26 inputs of
  each binary64 workload array (make_f64_digests.py), compared chunk by chunk with the
  device's results in each form the function has.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import exhaustive_hash as EH  # noqa: E402
import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    crm.set_force_slow(False)
    yield
    crm.set_force_slow(False)


def hard_set(func):
    xb, h = [], []
    with open(os.path.join(GOLDEN, "f64_hard", func + ".txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            a, b = line.split()
            xb.append(int(a, 16))
            h.append(float(b))
    return np.array(xb, dtype=np.uint64), np.array(h)


def run(func, xb, form, force=0):
    x = torch.from_numpy(xb.view(np.float64).copy()).cuda()
    y = torch.full_like(x, float("nan"))
    crm.set_force_slow(force)
    try:
        crm.stats_reset()
        crm.eval_into(func, x, y, form=form)
        torch.cuda.synchronize()
        st = crm.stats()
    finally:
        crm.set_force_slow(False)
    return y.cpu().numpy().view(np.uint64), st


@pytest.mark.parametrize("force", [0, 1, 2])
@pytest.mark.parametrize("form", ["df", "plain"])
@pytest.mark.parametrize("func", ["exp2", "log"])
def test_near_midpoint_inputs(func, form, force):
    xb, h = hard_set(func)
    assert xb.size == 10000
    ref = O.eval_bits(func, xb)
    got, st = run(func, xb, form, force)
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, [(hex(int(xb[i])), h[i], hex(int(got[i])), hex(int(ref[i]))) for i in bad[:6]]
    assert st["unresolved_total"] == 0
    if force:
        assert st["hard_total"] == xb.size


# Error bounds of the fast paths, in ulps of the result: the fixed-point exp2 core is good
# to 2^54 units of a Q124 value rounded at bit 72 (2^-18 ulp); the double-double main paths
# to 2^-100 (exp2) and 2^-98 (log) relative, at most 2^-46 ulp.  Results nearer a midpoint
# than a quarter of these bounds can only be decided by a slower tier.
QUEUED_BEYOND = {("exp2", "df"): 20.0, ("exp2", "plain"): 50.0, ("log", "plain"): 50.0}


@pytest.mark.parametrize("func,form", sorted(QUEUED_BEYOND))
def test_fast_path_queues_the_closest(func, form):
    xb, h = hard_set(func)
    sel = h > QUEUED_BEYOND[(func, form)]
    assert sel.sum() > 0
    got, st = run(func, xb[sel], form)
    assert np.array_equal(got, O.eval_bits(func, xb[sel]))
    assert st["hard_total"] == int(sel.sum()), (st["hard_total"], int(sel.sum()))


F64_FULL = [("exp2:domain", "exp2"), ("exp2:u20", "exp2"), ("log:bits", "log"), ("log:u0.125_8", "log"),
            ("exp:edomain", "exp"), ("exp10:tdomain", "exp10"), ("log2:bits", "log2"), ("log10:bits", "log10")]


# exp, exp10, log2 and log10 have the fixed-point form only
F64_FULL_CASES = [(lab, f, form) for lab, f in F64_FULL for form in ("df", "plain")
                  if form == "df" or f in ("exp2", "log")]


@pytest.mark.parametrize("label,func,form", F64_FULL_CASES)
def test_workload_arrays_every_element(label, func, form):
    path = os.path.join(GOLDEN, "f64_full", label.replace(":", "_") + ".txt")
    ref = EH.read_fixture(path)
    n = 1 << 26
    assert len(ref) == 2 * n // EH.CHUNK
    x = torch.from_numpy(W.bench_input_host("f64", label, func, n)).cuda()
    y = torch.empty_like(x)
    crm.stats_reset()
    crm.eval_into(func, x, y, form=form)
    words = y.view(torch.int32)
    w1, w2 = (torch.from_numpy(w).cuda() for w in EH.weights())
    bad = [c for c in sorted(ref)
           if EH.digest_torch(words[c * EH.CHUNK:(c + 1) * EH.CHUNK], w1, w2) != ref[c]]
    assert not bad, f"{label} ({form}): chunks {bad} differ from the oracle"
    assert crm.stats()["unresolved_total"] == 0
