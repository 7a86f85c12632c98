"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (the
autotuner's choice of launch shape or batch tile): the bench's own seeded inputs are
evaluated once and a sample of the outputs (random positions plus both ends of every
array) is compared with the oracle bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2605_15547_gb300 as crm  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
SAMPLE = 4096


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    crm.set_force_slow(False)
    yield
    for f in W.F32_FUNCS + ["exp2", "log"]:
        crm.set_variant(f, 1, form="auto")
    crm.set_batch_tile(14)


def sample_idx(n, rng):
    ends = np.r_[np.arange(min(64, n)), np.arange(max(0, n - 64), n)]
    return np.unique(np.r_[ends, rng.integers(0, n, SAMPLE)])


def check_sampled(func, x, y, rng):
    n = x.numel()
    idx = sample_idx(n, rng)
    it = torch.from_numpy(idx).to(x.device)
    bits = np.uint64 if x.dtype == torch.float64 else np.uint32
    xs = x[it].cpu().numpy().view(bits)
    ref = O.eval_bits(func, xs)
    if func == "sincosf":
        got = np.stack([y[0][it].cpu().numpy().view(bits), y[1][it].cpu().numpy().view(bits)])
    else:
        got = y[it].cpu().numpy().view(bits)
    bad = np.nonzero((got != ref).reshape(-1))[0]
    assert bad.size == 0, f"{func}: {bad.size} of {idx.size} sampled outputs differ"


@pytest.mark.parametrize("workload", ["all19", "precision", "trig", "f64"])
def test_bench_workload_sampled(workload):
    arrays, _ = W.bench_arrays(workload)
    rng = np.random.default_rng(11)
    crm.stats_reset()
    for label, func, n in arrays:
        x = W.bench_input_device(workload, label, func, n)
        y = torch.empty(((2,) if func == "sincosf" else ()) + (n,), dtype=x.dtype, device="cuda")
        crm.autotune(func, x, y, reps=1)
        crm.eval_into(func, x, y)
        check_sampled(func, x, y, rng)
        del x, y
    assert crm.stats()["unresolved_total"] == 0


def test_batch_workload_sampled():
    rng = np.random.Generator(np.random.PCG64(W.seed_for(4, 0)))
    lens, funcs = W.batch_lengths(10000, rng)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(W.seed_for(4, 0))
    items = []
    for f, n in zip(funcs, lens):
        x = W.domain_bits_device(f, int(n), gen)
        items.append((f, x, torch.empty((2 * int(n),) if f == "sincosf" else (int(n),), device="cuda")))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        crm.reserve(1 << 24, len(items), stream=s)
        crm.autotune_batch(items, reps=1, stream=s)
        crm.eval_batch(items, stream=s)
    s.synchronize()
    pick = np.random.default_rng(5).choice(len(items), 60, replace=False)
    srng = np.random.default_rng(6)
    for i in pick:
        f, x, y = items[i]
        yy = y.view(2, -1) if f == "sincosf" else y
        check_sampled(f, x, yy, srng)


def test_array_beyond_2p33_elements():
    """The vector loop works in segments of 2^31 vectors (2^33 binary32 elements): an
    array one segment plus a ragged tail long (64 GiB in and out on the device), checked
    on both sides of the segment boundary, at both ends and at random positions."""
    n = (1 << 33) + 4101
    free, _ = torch.cuda.mem_get_info()
    if free < 2 * 4 * n + (4 << 30):
        pytest.skip("not enough device memory for a 2^33-element array pair")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(W.seed_for(9, 0))
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    x.uniform_(-87.0, 88.0, generator=gen)
    y = torch.empty_like(x)
    crm.eval_into("expf", x, y)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    b = 1 << 33
    idx = np.unique(np.r_[np.arange(b - 300, b + 300), np.arange(n - 64, n), np.arange(64),
                          rng.integers(0, n, SAMPLE)])
    it = torch.from_numpy(idx).cuda()
    xs = x[it].cpu().numpy().view(np.uint32)
    got = y[it].cpu().numpy().view(np.uint32)
    del x, y
    torch.cuda.empty_cache()
    assert np.array_equal(got, O.eval_bits("expf", xs))
