"""Exhaustive binary32 sweeps on the GPU: all 2^32 input bit patterns per function.

* Against the oracle: the device results of every chunk of 2^24 consecutive patterns are
  digested (tests/exhaustive_hash.py) and compared with the digests the oracle's results
  gave (tests/golden/exhaustive/<func>.txt, written by tests/golden/make_exhaustive.py).
  A function whose file lists all 256 chunks is checked over its whole input space.
* No FP64 in the default form: the slow path's FP64-free tier decides every queued lane
  (crm_stats fp64_total stays 0 over all 2^32 inputs).
* Between the forms: the double-float form and the plain FP64 form (two independent
  evaluations with their own rounding tests) give the same bits on all 2^32 inputs, and
  sincosf gives (sinf, cosf) bit for bit.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import exhaustive_hash as EH  # noqa: E402
import paper_2605_15547_gb300 as crm  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "exhaustive")
SINGLE = [f for f in W.F32_FUNCS if f != "sincosf"]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    crm.set_force_slow(False)
    yield


@pytest.fixture(scope="module")
def weights():
    w1, w2 = EH.weights()
    return torch.from_numpy(w1).cuda(), torch.from_numpy(w2).cuda()


def chunk_input(c):
    base = c << EH.CHUNK_LOG2
    bits = torch.arange(base, base + EH.CHUNK, dtype=torch.int64, device="cuda")
    bits = torch.remainder(bits + 2**31, 2**32) - 2**31  # the uint32 pattern as int32
    return bits.to(torch.int32).view(torch.float32)


@pytest.mark.parametrize("func", SINGLE)
def test_exhaustive_against_oracle_digests(func, weights):
    path = os.path.join(GOLDEN, func + ".txt")
    ref = EH.read_fixture(path)
    assert len(ref) == EH.NCHUNKS, f"{func}: the oracle digests cover {len(ref)} of {EH.NCHUNKS} chunks"
    w1, w2 = weights
    y = torch.empty(EH.CHUNK, dtype=torch.float32, device="cuda")
    bad = []
    crm.stats_reset()
    for c in sorted(ref):
        crm.eval_into(func, chunk_input(c), y)
        got = EH.digest_torch(y.view(torch.int32), w1, w2)
        if got != ref[c]:
            bad.append(c)
    assert not bad, f"{func}: chunks {bad[:8]} differ from the oracle ({len(bad)} of {len(ref)})"
    st = crm.stats()
    assert st["unresolved_total"] == 0
    # the FP64-free middle tier decides every lane the fast path queues: over all 2^32
    # inputs no lane goes on to the FP64 (double-double) tier
    assert st["fp64_total"] == 0, f"{func}: {st['fp64_total']} lanes ran the FP64 tier"


@pytest.mark.parametrize("func", ["expf", "exp2f", "exp10f"])
def test_exhaustive_register_table_variant(func, weights):
    """the exp family's 16-entry register-table evaluator (warp shuffles instead of the
    64-entry shared-memory table) against the oracle on all 2^32 inputs"""
    ref = EH.read_fixture(os.path.join(GOLDEN, func + ".txt"))
    w1, w2 = weights
    y = torch.empty(EH.CHUNK, dtype=torch.float32, device="cuda")
    v = next(i for i in range(crm._lib.NUM_VARIANTS) if crm.variant_info(i)["reg_table"])
    crm.set_variant(func, v, form="df")
    try:
        bad = [c for c in sorted(ref)
               if (crm.eval_into(func, chunk_input(c), y, form="df") or
                   EH.digest_torch(y.view(torch.int32), w1, w2)) != ref[c]]
    finally:
        crm.set_variant(func, 1, form="df")
    assert not bad, f"{func} (register table): chunks {bad[:8]} differ from the oracle"


@pytest.mark.parametrize("func", SINGLE)
def test_exhaustive_forms_agree(func):
    a = torch.empty(EH.CHUNK, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    for c in range(EH.NCHUNKS):
        x = chunk_input(c)
        crm.eval_into(func, x, a, form="df")
        crm.eval_into(func, x, b, form="plain")
        if not torch.equal(a.view(torch.int32), b.view(torch.int32)):
            d = torch.nonzero(a.view(torch.int32) != b.view(torch.int32))[:4].flatten().tolist()
            pytest.fail(f"{func}: forms differ in chunk {c} at offsets {d}")


def test_exhaustive_sincosf_is_sinf_cosf():
    s = torch.empty(EH.CHUNK, dtype=torch.float32, device="cuda")
    co = torch.empty_like(s)
    sc = torch.empty(2 * EH.CHUNK, dtype=torch.float32, device="cuda")
    for c in range(EH.NCHUNKS):
        x = chunk_input(c)
        crm.eval_into("sinf", x, s)
        crm.eval_into("cosf", x, co)
        crm.eval_into("sincosf", x, sc)
        ok = torch.equal(sc[:EH.CHUNK].view(torch.int32), s.view(torch.int32)) and \
            torch.equal(sc[EH.CHUNK:].view(torch.int32), co.view(torch.int32))
        assert ok, f"sincosf differs from (sinf, cosf) in chunk {c}"


EASY = [f for f in SINGLE if f not in ("logf", "log2f", "log10f", "rsqrtf")]


@pytest.mark.parametrize("func", EASY)
def test_exhaustive_packing_shape(func, weights):
    """The packing launch shape (tiny arguments resolved without the evaluator, the rest
    packed across the warp) against the oracle on all 2^32 inputs: a warp's vector of
    consecutive bit patterns is all easy, none or a mix, so every easy() bound is checked
    on every input below and around it."""
    ref = EH.read_fixture(os.path.join(GOLDEN, func + ".txt"))
    w1, w2 = weights
    y = torch.empty(EH.CHUNK, dtype=torch.float32, device="cuda")
    v = next(i for i in range(crm._lib.NUM_VARIANTS) if crm.variant_info(i)["easy"])
    crm.set_variant(func, v, form="df")
    crm.stats_reset()
    try:
        bad = [c for c in sorted(ref)
               if (crm.eval_into(func, chunk_input(c), y, form="df") or
                   EH.digest_torch(y.view(torch.int32), w1, w2)) != ref[c]]
    finally:
        crm.set_variant(func, 1, form="df")
    assert not bad, f"{func} (packing): chunks {bad[:8]} differ from the oracle"
    assert crm.stats()["unresolved_total"] == 0


def test_exhaustive_sincosf_packing_is_sinf_cosf():
    v = next(i for i in range(crm._lib.NUM_VARIANTS) if crm.variant_info(i)["easy"])
    s = torch.empty(EH.CHUNK, dtype=torch.float32, device="cuda")
    co = torch.empty_like(s)
    sc = torch.empty(2 * EH.CHUNK, dtype=torch.float32, device="cuda")
    crm.set_variant("sincosf", v, form="df")
    try:
        for c in range(EH.NCHUNKS):
            x = chunk_input(c)
            crm.eval_into("sinf", x, s)
            crm.eval_into("cosf", x, co)
            crm.eval_into("sincosf", x, sc)
            ok = torch.equal(sc[:EH.CHUNK].view(torch.int32), s.view(torch.int32)) and \
                torch.equal(sc[EH.CHUNK:].view(torch.int32), co.view(torch.int32))
            assert ok, f"sincosf (packing) differs from (sinf, cosf) in chunk {c}"
    finally:
        crm.set_variant("sincosf", 1, form="df")
