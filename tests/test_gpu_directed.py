"""GPU parity in every rounding direction and in the 16-bit formats (crm_eval_rm) against
the oracle, bit for bit.

* binary32, toward -inf, +inf and zero: every function on a domain sample, specials, the
  function's own focus sets and its exact results (2^k, 10^k, log2 of powers of two, log10
  of powers of ten, rsqrt of powers of four, ...), also with every lane forced through the
  slow path; expf and logf over all 2^32 inputs against the oracle's digests;
* binary64 exp2 and log in every direction on the near-midpoint set, random inputs,
  integers and specials;
* IEEE binary16 and bfloat16: all 2^16 inputs of every binary32 function in all four
  directions.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import exhaustive_hash as EH  # noqa: E402
import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402
from test_gpu_parity import focus_inputs  # noqa: E402

pytestmark = pytest.mark.gpu

DIRECTED = ["rd", "ru", "rz"]
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


def run_rm(func, xbits, mode, fmt="f32"):
    """crm.eval_rm on the bit patterns xbits (uint32 for binary32, uint64 for binary64,
    uint16 for fmt f16 / bf16); returns result bit patterns ((2, n) for sincosf)."""
    n = xbits.size
    if fmt in ("f16", "bf16"):
        x = torch.from_numpy(xbits.astype(np.int16)).cuda().view(torch.float16 if fmt == "f16" else torch.bfloat16)
        bits = np.uint16
    elif xbits.dtype == np.uint64:
        x = torch.from_numpy(xbits.view(np.float64)).cuda()
        bits = np.uint64
    else:
        x = torch.from_numpy(xbits.view(np.float32)).cuda()
        bits = np.uint32
    y = crm.eval_rm(func, x, mode)
    torch.cuda.synchronize()
    out = y.cpu().view(torch.int16 if bits == np.uint16 else (torch.int64 if bits == np.uint64 else torch.int32))
    out = out.numpy().view(bits).reshape(-1)
    return out.reshape(2, n) if func == "sincosf" else out


def exact_inputs(func):
    """inputs whose results are binary32 numbers (the cases a directed rounding must not
    move), and their neighbours"""
    ints = np.arange(-160, 131, dtype=np.float32)
    if func == "exp2f":
        base = ints
    elif func == "exp10f":
        base = np.arange(-50, 46, dtype=np.float32)
    elif func in ("logf", "log2f", "log10f", "log1pf"):
        p2 = np.ldexp(np.float32(1), np.arange(-149, 128)).astype(np.float32)
        base = np.concatenate([p2, np.float32(10.0) ** np.arange(0, 11, dtype=np.float32),
                               np.array([1.0, 2.0, 0.5], np.float32)])
    elif func == "rsqrtf":
        base = np.ldexp(np.float32(1), np.arange(-148, 128, 2)).astype(np.float32)
    else:
        base = np.array([0.0, 1.0, -1.0, 0.5, 2.0], dtype=np.float32)
    b = base.view(np.uint32).astype(np.int64)
    near = np.concatenate([b + d for d in (-1, 0, 1)])
    near = near[(near > 0) & (near < 0x7F800000)]
    return np.concatenate([near, near | 0x80000000]).astype(np.uint32)


def directed_inputs(func, seed):
    rng = W.rng_for(9, func, salt=seed)
    parts = [W.domain_bits(func, (1 << 15) + 37, rng), W.specials_f32(func, rng).view(np.uint32),
             focus_inputs(func, rng)[::2], exact_inputs(func)]
    return np.concatenate([p.astype(np.uint32) for p in parts])


def assert_same(what, xbits, got, ref):
    bad = np.nonzero(got.reshape(-1) != ref.reshape(-1))[0]
    n = xbits.size
    assert bad.size == 0, (what, bad.size, [(hex(int(xbits[i % n])), hex(int(got.reshape(-1)[i])),
                                             hex(int(ref.reshape(-1)[i]))) for i in bad[:6]])


@pytest.mark.parametrize("mode", DIRECTED)
@pytest.mark.parametrize("func", W.F32_FUNCS)
def test_binary32_directed(func, mode):
    xb = directed_inputs(func, 1)
    crm.stats_reset()
    got = run_rm(func, xb, mode)
    assert_same(f"{func} {mode}", xb, got, O.eval_bits(func, xb, mode=mode))
    assert crm.stats()["unresolved_total"] == 0


@pytest.mark.parametrize("force", [1, 2])
@pytest.mark.parametrize("mode", DIRECTED)
@pytest.mark.parametrize("func", W.F32_FUNCS)
def test_binary32_directed_slow_path(func, mode, force):
    """every lane through the slow path (force 1: every tier; 2: the first tier decides)"""
    xb = directed_inputs(func, 2)[::4]
    crm.set_force_slow(force)
    try:
        crm.stats_reset()
        got = run_rm(func, xb, mode)
        st = crm.stats()
    finally:
        crm.set_force_slow(False)
    assert_same(f"{func} {mode} forced {force}", xb, got, O.eval_bits(func, xb, mode=mode))
    assert st["unresolved_total"] == 0


def test_rn_is_crm_eval():
    xb = W.domain_bits("expf", 4099, W.rng_for(9, "expf"))
    got = run_rm("expf", xb, "rn")
    assert np.array_equal(got, O.eval_bits("expf", xb))


def f64_inputs(func):
    rng = W.rng_for(9, func)
    hard = []
    with open(os.path.join(GOLDEN, "f64_hard", func + ".txt")) as fh:
        for line in fh:
            if not line.startswith("#") and line.strip():
                hard.append(int(line.split()[0], 16))
    if func == "exp2":
        parts = [W.f64_uniform(-1075, 1024, 20000, rng), W.f64_uniform(-20, 20, 20000, rng),
                 np.arange(-1080, 1030, dtype=np.float64), W.f64_uniform(-1080, -1020, 4000, rng),
                 rng.uniform(-1, 1, 4000) * np.exp2(rng.uniform(-80, -40, 4000)),
                 np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -1075.0, 1024.0, 1023.999])]
    else:
        parts = [W.f64_positive_bits(20000, rng), W.f64_uniform(0.125, 8.0, 20000, rng),
                 np.exp2(np.arange(-1074, 1024, dtype=np.float64)),
                 1.0 + np.arange(-2000, 2000) * 2.0 ** -52,
                 np.array([1.0, 0.0, -0.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, 1.7976931348623157e308])]
    x = np.concatenate(parts).view(np.uint64)
    return np.concatenate([x, np.array(hard, dtype=np.uint64)])


@pytest.mark.parametrize("mode", DIRECTED)
@pytest.mark.parametrize("func", ["exp2", "log"])
def test_binary64_directed(func, mode):
    xb = f64_inputs(func)
    for force in (0, 1):
        crm.set_force_slow(force)
        try:
            got = run_rm(func, xb, mode)
        finally:
            crm.set_force_slow(False)
        assert_same(f"{func} {mode} force {force}", xb, got, O.eval_bits(func, xb, mode=mode))


ALL16 = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("func", W.F32_FUNCS)
def test_16bit_formats_all_inputs(func, fmt):
    for mode in ("rn", "rd", "ru", "rz"):
        got = run_rm(func, ALL16, mode, fmt)
        ref = O.eval_bits16(func, ALL16, fmt, mode)
        assert_same(f"{func} {fmt} {mode}", ALL16, got, ref)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("func", ["expf", "logf", "sincosf", "tanhf", "rsqrtf", "acosf"])
def test_16bit_formats_slow_path(func, fmt):
    crm.set_force_slow(1)
    try:
        for mode in ("rn", "rz"):
            got = run_rm(func, ALL16, mode, fmt)
            assert_same(f"{func} {fmt} {mode} forced", ALL16, got, O.eval_bits16(func, ALL16, fmt, mode))
    finally:
        crm.set_force_slow(False)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("func", ["expf", "sincosf", "atanf"])
def test_16bit_ragged_and_misaligned(func, fmt):
    """The 16-bit path's 16-byte vectors between a scalar head and tail: every start offset
    modulo 8 halves and ragged lengths, in place or not, with guard halves around the
    output that must stay untouched."""
    rng = np.random.default_rng(5)
    rows = 2 if func == "sincosf" else 1
    dt = torch.float16 if fmt == "f16" else torch.bfloat16
    for n in (1, 7, 8, 9, 63, 1000, 4101):
        xb = rng.integers(0, 1 << 16, n).astype(np.uint16)
        ref = O.eval_bits16(func, xb, fmt, "rd").reshape(-1)
        for off in range(0, 8, 3):
            xbuf = torch.zeros(n + 16, dtype=torch.int16, device="cuda")
            xbuf[off:off + n] = torch.from_numpy(xb.astype(np.int16)).cuda()
            x = xbuf[off:off + n].view(dt)
            for oo in (off, (off + 5) % 8):
                ybuf = torch.full((rows * n + 32,), 0x5A5A, dtype=torch.int16, device="cuda")
                y = ybuf[oo + 8:oo + 8 + rows * n].view(dt)
                crm.eval_rm(func, x, "rd", out=y)
                got = y.view(torch.int16).cpu().numpy().view(np.uint16)
                assert np.array_equal(got, ref), f"{func} {fmt} n {n} offsets {off} {oo}"
                assert bool((ybuf[:oo + 8] == 0x5A5A).all()) and bool((ybuf[oo + 8 + rows * n:] == 0x5A5A).all()), \
                    f"{func} {fmt} n {n}: a write outside the output"


@pytest.mark.parametrize("func", ["asinf", "sincosf", "expf", "atanf"])
def test_binary32_directed_ragged_with_guards(func):
    """The directed kernel's vectors (and their packing of easy arguments) on ragged sizes
    and a misaligned start, with guard words around the output."""
    rng = W.rng_for(9, func)
    rows = 2 if func == "sincosf" else 1
    for mode in ("rd", "rz"):
        for n in (1, 33, 1000, 4101, 65537):
            xb = W.domain_bits(func, n, rng)
            ref = O.eval_bits(func, xb, mode=mode).reshape(-1)
            for off in (0, 1):
                xbuf = torch.zeros(n + 8, dtype=torch.float32, device="cuda")
                xbuf[off:off + n] = torch.from_numpy(xb.view(np.float32)).cuda()
                ybuf = torch.full((rows * n + 64,), 12345.0, device="cuda")
                y = ybuf[32 + off:32 + off + rows * n]
                crm.eval_rm(func, xbuf[off:off + n], mode, out=y)
                got = y.cpu().numpy().view(np.uint32)
                assert np.array_equal(got, ref), f"{func} {mode} n {n} off {off}"
                assert bool((ybuf[:32 + off] == 12345.0).all()) and bool((ybuf[32 + off + rows * n:] == 12345.0).all()), \
                    f"{func} {mode} n {n}: a write outside the output"


def chunk_input(c):
    base = c << EH.CHUNK_LOG2
    bits = torch.arange(base, base + EH.CHUNK, dtype=torch.int64, device="cuda")
    bits = torch.remainder(bits + 2**31, 2**32) - 2**31
    return bits.to(torch.int32).view(torch.float32)


@pytest.mark.parametrize("mode", DIRECTED)
@pytest.mark.parametrize("func", ["expf", "logf"])
def test_exhaustive_directed_against_oracle_digests(func, mode):
    path = os.path.join(GOLDEN, "exhaustive_" + mode, func + ".txt")
    if not os.path.exists(path):
        pytest.skip(f"no oracle digests for {func} {mode}")
    ref = EH.read_fixture(path)
    assert len(ref) == EH.NCHUNKS, f"{func} {mode}: the oracle digests cover {len(ref)} of {EH.NCHUNKS} chunks"
    w1, w2 = (torch.from_numpy(w).cuda() for w in EH.weights())
    y = torch.empty(EH.CHUNK, dtype=torch.float32, device="cuda")
    crm.stats_reset()
    bad = []
    for c in sorted(ref):
        crm.eval_rm(func, chunk_input(c), mode, out=y)
        if EH.digest_torch(y.view(torch.int32), w1, w2) != ref[c]:
            bad.append(c)
    assert not bad, f"{func} {mode}: chunks {bad[:8]} differ from the oracle ({len(bad)} of {len(ref)})"
    assert crm.stats()["unresolved_total"] == 0
