"""GPU tests of the launch shapes and the autotuner: every variant of the main kernel
computes the same bits (checked against the oracle), and the autotuner keeps one of the
variants it timed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402
from paper_2605_15547_gb300._lib import NUM_VARIANTS  # noqa: E402

pytestmark = pytest.mark.gpu

FUNCS = ["expf", "log1pf", "sinf", "sincosf", "atanf", "tanhf", "rsqrtf", "acosf"]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    crm.set_force_slow(False)
    yield
    for f in W.F32_FUNCS + ["exp2", "log"]:
        crm.set_variant(f, 1, form="df")


REGTAB_FUNCS = ("expf", "exp2f", "exp10f")
# the functions with easy arguments (the packing shapes)
EASY_FUNCS = tuple(f for f in W.F32_FUNCS if f not in ("logf", "log2f", "log10f", "rsqrtf"))


@pytest.mark.parametrize("func", FUNCS)
def test_every_variant_gives_the_oracle_bits(func):
    rng = W.rng_for(7, func)
    n = (1 << 17) + 13
    xb = W.domain_bits(func, n, rng)
    ref = O.eval_bits(func, xb).reshape(-1)
    buf = torch.from_numpy(np.concatenate([np.zeros(1, np.uint32), xb]).view(np.float32)).cuda()
    x = buf[1:]  # 4-byte aligned, not 16: exercises the scalar head as well
    for v in range(NUM_VARIANTS):
        info = crm.variant_info(v)
        if (info["reg_table"] and func not in REGTAB_FUNCS) or (info["easy"] and func not in EASY_FUNCS):
            with pytest.raises(crm.CrmError):  # shapes the function does not provide
                crm.set_variant(func, v, form="df")
            continue
        crm.set_variant(func, v, form="df")
        y = crm.eval(func, x, form="df")
        got = y.cpu().numpy().view(np.uint32).reshape(-1)
        assert np.array_equal(got, ref), f"{func} variant {v} ({crm.variant_info(v)})"
    crm.set_variant(func, 1, form="df")


@pytest.mark.parametrize("func", ["expf", "sincosf", "tanhf", "exp2", "log"])
@pytest.mark.parametrize("off", [0, 3])
def test_every_variant_with_congruent_arrays(func, off):
    """in and out at the same offset modulo 32 bytes, so that the 32-byte shapes run their
    vector loop (with a scalar head when off > 0) and a ragged tail"""
    rng = W.rng_for(7, func, salt=3)
    n = (1 << 16) + 29
    f64 = func in ("exp2", "log")
    if f64:
        xh = W.f64_uniform(-30, 30, n, rng) if func == "exp2" else W.f64_positive_bits(n, rng)
        xb, bits, dt = xh.view(np.uint64), np.uint64, torch.float64
    else:
        xb, bits, dt = W.domain_bits(func, n, rng), np.uint32, torch.float32
        xh = xb.view(np.float32)
    ref = O.eval_bits(func, xb).reshape(-1)
    rows = 2 if func == "sincosf" else 1
    xbuf = torch.zeros(n + 64, dtype=dt, device="cuda")
    ybuf = torch.zeros(rows * n + 64, dtype=dt, device="cuda")
    x = xbuf[off:off + n]
    x.copy_(torch.from_numpy(xh))
    y = ybuf[off:off + rows * n]
    guard = torch.full_like(ybuf, 12345.0)
    for v in range(NUM_VARIANTS):
        try:
            crm.set_variant(func, v, form="df")
        except crm.CrmError:
            continue
        ybuf.copy_(guard)
        crm.eval_into(func, x, y, form="df")
        got = y.cpu().numpy().view(bits)
        assert np.array_equal(got, ref), f"{func} variant {v} ({crm.variant_info(v)}) off {off}"
        # nothing written outside the output
        assert torch.equal(ybuf[:off], guard[:off]) and torch.equal(ybuf[off + rows * n:], guard[off + rows * n:]), \
            f"{func} variant {v}: a write outside the output array"
    crm.set_variant(func, 1, form="df")


@pytest.mark.parametrize("func", ["asinf", "sincosf", "expf", "tanf"])
def test_packing_shapes_on_ragged_sizes(func):
    """The packing shapes on arrays whose last vectors leave lanes or whole warps idle
    (mostly easy arguments, so that packing runs): the oracle's bits, and no write outside
    the output (guard words on both sides)."""
    rng = W.rng_for(7, func, salt=5)
    rows = 2 if func == "sincosf" else 1
    for v in (11, 12):
        crm.set_variant(func, v, form="df")
        for n in (1, 7, 31, 33, 100, 257, 1000, 4099, 65537, 300001):
            xb = W.domain_bits(func, n, rng)
            ref = O.eval_bits(func, xb).reshape(-1)
            x = torch.from_numpy(xb.view(np.float32)).cuda()
            ybuf = torch.full((rows * n + 128,), 12345.0, device="cuda")
            y = ybuf[64:64 + rows * n]
            crm.eval_into(func, x, y, form="df")
            got = y.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref), f"{func} variant {v} n {n}"
            assert bool((ybuf[:64] == 12345.0).all()) and bool((ybuf[64 + rows * n:] == 12345.0).all()), \
                f"{func} variant {v} n {n}: a write outside the output array"
    crm.set_variant(func, 1, form="df")


def test_plain_form_has_only_the_default_shape():
    with pytest.raises(crm.CrmError):
        crm.set_variant("expf", 4, form="plain")
    crm.set_variant("expf", 1, form="plain")
    assert crm.get_variant("expf", form="plain") == 1


def test_autotune_keeps_a_timed_variant():
    x = torch.from_numpy(W.domain_bits("logf", 1 << 22, W.rng_for(8, "logf")).view(np.float32)).cuda()
    best, ms = crm.autotune("logf", x, form="df", reps=2)
    # every shape but the register table and the packing ones (log has no easy arguments)
    assert best in ms and len(ms) == NUM_VARIANTS - 3
    assert all(t > 0 for t in ms.values())
    assert crm.get_variant("logf", form="df") == best
    y = crm.eval("logf", x[:4099], form="df")
    ref = O.eval_bits("logf", x[:4099].cpu().numpy().view(np.uint32))
    assert np.array_equal(y.cpu().numpy().view(np.uint32), ref)


def test_autotune_batch_picks_a_tile():
    rng = np.random.default_rng(3)
    items = []
    for i in range(40):
        f = W.F32_FUNCS[i % 19]
        n = int(rng.integers(1, 1 << 15))
        x = torch.from_numpy(W.domain_bits(f, n, rng).view(np.float32)).cuda()
        items.append((f, x, torch.empty((2 * n,) if f == "sincosf" else (n,), device="cuda")))
    mode, best, ms = crm.autotune_batch(items, reps=1)
    assert 10 <= best <= 16 and (mode, best) in ms and mode in ("mixed", "grouped")
    assert len(ms) == 14 and all(t > 0 for t in ms.values())
    crm.set_batch_tile(14)
    crm.set_batch_mode("grouped")
