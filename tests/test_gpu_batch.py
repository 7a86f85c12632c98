"""GPU tests of the batching form (crm_eval_batch): many arrays of mixed functions and
uneven lengths in one persistent launch must give exactly the per-array results, which
the parity suite ties to the oracle; a sample is also checked against the oracle here.
"""
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


def make_batch(count, max_log2, seed, misalign=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    items = []
    for i in range(count):
        f = W.F32_FUNCS[int(rng.integers(0, len(W.F32_FUNCS)))]
        n = int(round(2 ** rng.uniform(0, max_log2)))
        off = int(rng.integers(0, 4)) if misalign else 0
        x = W.domain_bits(f, n, rng).view(np.float32)
        buf = torch.zeros(n + off + 4, dtype=torch.float32, device="cuda")
        buf[off:off + n] = torch.from_numpy(x).cuda()
        rows = 2 if f == "sincosf" else 1
        oo = int(rng.integers(0, 4)) if misalign else 0
        obuf = torch.full((rows * n + oo + 4,), float("nan"), device="cuda")
        items.append((f, buf[off:off + n], obuf[oo:oo + rows * n], x))
    return items


@pytest.mark.parametrize("mode", ["mixed", "grouped"])
@pytest.mark.parametrize("form", ["plain", "df"])
@pytest.mark.parametrize("tile", [10, 14])
def test_batch_matches_single_calls(form, tile, mode):
    items = make_batch(300, 15, seed=100 + tile)
    crm.set_batch_tile(tile)
    crm.set_batch_mode(mode)
    try:
        crm.eval_batch([(f, x, y) for f, x, y, _ in items], form=form)
    finally:
        crm.set_batch_tile(14)
        crm.set_batch_mode("grouped")
    torch.cuda.synchronize()
    for f, x, y, _ in items:
        ref = torch.empty_like(y)
        crm.eval_into(f, x, ref, form=form)
        torch.cuda.synchronize()
        a = y.cpu().numpy().view(np.uint32)
        b = ref.cpu().numpy().view(np.uint32)
        assert np.array_equal(a, b), f"{f}: {int(np.count_nonzero(a != b))} differ"


@pytest.mark.parametrize("shape", [11, 12])
def test_grouped_batch_packs_like_the_packing_shapes(shape):
    """With a packing launch shape chosen for every function that has one, the grouped
    batch packs those functions' elements too: the results must equal the oracle's."""
    easy = [f for f in W.F32_FUNCS if crm.variant_info(shape)["easy"]]
    items = make_batch(150, 13, seed=300 + shape, misalign=False)
    chosen = []
    for f in easy:
        try:
            crm.set_variant(f, shape, form="df")
            chosen.append(f)
        except crm.CrmError:  # no easy arguments: the function keeps its shape
            pass
    assert len(chosen) == 15
    try:
        crm.set_batch_mode("grouped")
        crm.eval_batch([(f, x, y) for f, x, y, _ in items], form="df")
        torch.cuda.synchronize()
    finally:
        for f in chosen:
            crm.set_variant(f, 1, form="df")
    for f, x, y, xh in items:
        got = y.cpu().numpy().view(np.uint32)
        ref = O.eval_bits(f, xh.view(np.uint32)).reshape(-1)
        assert np.array_equal(got, ref), f
        tail = y._base[y.storage_offset() + y.numel():]  # the output buffer's guard words
        assert bool(torch.isnan(tail).all()), f"{f}: a write past the end of the output"


def test_batch_against_oracle_sample():
    items = make_batch(120, 12, seed=7)
    crm.eval_batch([(f, x, y) for f, x, y, _ in items])
    torch.cuda.synchronize()
    for f, x, y, xh in items:
        got = y.cpu().numpy().view(np.uint32)
        ref = O.eval_bits(f, xh.view(np.uint32)).reshape(-1)
        assert np.array_equal(got, ref), f
    assert crm.stats()["unresolved_total"] == 0


@pytest.mark.parametrize("mode", ["mixed", "grouped"])
def test_batch_forced_slow_path(mode):
    items = make_batch(100, 12, seed=9)
    crm.set_force_slow(True)
    crm.set_batch_mode(mode)
    try:
        crm.eval_batch([(f, x, y) for f, x, y, _ in items])
        torch.cuda.synchronize()
    finally:
        crm.set_force_slow(False)
        crm.set_batch_mode("grouped")
    for f, x, y, xh in items:
        got = y.cpu().numpy().view(np.uint32)
        ref = O.eval_bits(f, xh.view(np.uint32)).reshape(-1)
        assert np.array_equal(got, ref), f


def test_batch_graph_capture_and_replay():
    items = make_batch(64, 14, seed=11, misalign=False)
    s = torch.cuda.Stream()
    crm.reserve(1 << 24, 4096, stream=s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        crm.eval_batch([(f, x, y) for f, x, y, _ in items], stream=s)  # warm-up
    s.synchronize()
    for _, _, y, _ in items:
        y.fill_(float("nan"))
    with torch.cuda.graph(g, stream=s):
        crm.eval_batch([(f, x, y) for f, x, y, _ in items], stream=s)
    for rep in range(3):
        for _, _, y, _ in items:
            y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for f, x, y, xh in items:
            got = y.cpu().numpy().view(np.uint32)
            ref = O.eval_bits(f, xh.view(np.uint32)).reshape(-1)
            assert np.array_equal(got, ref), (rep, f)


def test_batch_graphs_keep_their_arrays():
    """A captured batch owns its staged descriptors: a later batch call on the stream with
    other arrays, and a second capture, leave the first graph evaluating its own arrays."""
    a = make_batch(40, 12, seed=31, misalign=False)
    b = make_batch(70, 12, seed=32, misalign=False)
    s = torch.cuda.Stream()
    crm.reserve(1 << 24, 4096, stream=s)
    with torch.cuda.stream(s):
        crm.eval_batch([(f, x, y) for f, x, y, _ in a], stream=s)
    s.synchronize()
    ga, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(ga, stream=s):
        crm.eval_batch([(f, x, y) for f, x, y, _ in a], stream=s)
    with torch.cuda.stream(s):  # outside capture: stages b's descriptors in new buffers
        crm.eval_batch([(f, x, y) for f, x, y, _ in b], stream=s)
    s.synchronize()
    with torch.cuda.graph(gb, stream=s):
        crm.eval_batch([(f, x, y) for f, x, y, _ in b], stream=s)
    for rep in range(2):
        for items, g in ((a, ga), (b, gb)):
            for _, _, y, _ in a + b:
                y.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            for f, x, y, xh in items:
                ref = O.eval_bits(f, xh.view(np.uint32)).reshape(-1)
                assert np.array_equal(y.cpu().numpy().view(np.uint32), ref), (rep, f)
            other = b if items is a else a
            assert all(torch.isnan(y).all() for _, _, y, _ in other)  # untouched


def test_single_call_graph_capture():
    x = torch.from_numpy(W.domain_bits("logf", 1 << 20, W.rng_for(2, "logf")).view(np.float32)).cuda()
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    crm.reserve(1 << 24, 0, stream=s)
    with torch.cuda.stream(s):
        crm.eval_into("logf", x, y, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        crm.eval_into("logf", x, y, stream=s)
    y.fill_(0)
    g.replay()
    torch.cuda.synchronize()
    ref = O.eval_bits("logf", x.cpu().numpy().view(np.uint32))
    assert np.array_equal(y.cpu().numpy().view(np.uint32), ref)


def test_batch_with_binary64_arrays():
    """binary64 arrays mixed into a batch (the grouped mode runs them) against the oracle"""
    rng = np.random.default_rng(21)
    items = []
    for i in range(60):
        f = ["expf", "exp2", "logf", "log", "sincosf"][i % 5]
        n = int(rng.integers(1, 5000))
        if f == "exp2":
            x = W.f64_uniform(-1080, 1030, n, rng)
        elif f == "log":
            x = W.f64_positive_bits(n, rng)
        else:
            x = W.domain_bits(f, n, rng).view(np.float32)
        xt = torch.from_numpy(x).cuda()
        rows = 2 if f == "sincosf" else 1
        items.append((f, xt, torch.empty(rows * n, dtype=xt.dtype, device="cuda"), x))
    for mode in ("mixed", "grouped"):  # mixed falls back to grouped for binary64
        crm.set_batch_mode(mode)
        try:
            crm.eval_batch([(f, x, y) for f, x, y, _ in items])
            torch.cuda.synchronize()
        finally:
            crm.set_batch_mode("grouped")
        for f, x, y, xh in items:
            bits = np.uint64 if xh.dtype == np.float64 else np.uint32
            got = y.cpu().numpy().view(bits)
            ref = O.eval_bits(f, xh.view(bits)).reshape(-1)
            assert np.array_equal(got, ref), (mode, f)
