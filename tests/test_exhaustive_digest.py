"""Host checks of the exhaustive-sweep digests: the numpy and torch forms agree, the
digest notices single-ulp and multiple-of-P changes, and the stored files are well formed.
"""
import os

import numpy as np
import pytest

import exhaustive_hash as EH

torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "exhaustive")


@pytest.fixture(scope="module")
def weights():
    return EH.weights()


def test_numpy_and_torch_digests_agree(weights):
    w1, w2 = weights
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.integers(0, 2**32, EH.CHUNK, dtype=np.uint64).astype(np.uint32)
        a = EH.digest_np(v, w1, w2)
        b = EH.digest_torch(torch.from_numpy(v.view(np.int32)), torch.from_numpy(w1), torch.from_numpy(w2))
        assert a == b


def test_digest_detects_small_changes(weights):
    w1, w2 = weights
    v = EH.chunk_bits(77)  # any vector
    base = EH.digest_np(v, w1, w2)
    for i, delta in [(0, 1), (EH.CHUNK - 1, -1), (12345, EH.P), (999, 2 * EH.P)]:
        u = v.astype(np.int64)
        u[i] = (u[i] + delta) % 2**32
        assert EH.digest_np(u.astype(np.uint32), w1, w2) != base
    # two compensating 1-ulp changes still move the weighted sums
    u = v.copy()
    u[10] += 1
    u[20] -= 1
    d = EH.digest_np(u, w1, w2)
    assert d[0] == base[0] and d[1:] != base[1:]


def test_chunks_cover_the_space():
    assert EH.CHUNK * EH.NCHUNKS == 2**32
    assert EH.chunk_bits(0)[0] == 0 and EH.chunk_bits(EH.NCHUNKS - 1)[-1] == 0xFFFFFFFF


def test_stored_digest_files_are_well_formed():
    if not os.path.isdir(GOLDEN):
        pytest.skip("no digest files")
    for name in sorted(os.listdir(GOLDEN)):
        d = EH.read_fixture(os.path.join(GOLDEN, name))
        assert all(0 <= c < EH.NCHUNKS for c in d), name
        for s, h1, h2 in d.values():
            assert 0 <= s < 2**56 and 0 <= h1 < EH.P and 0 <= h2 < EH.P, name


def test_every_single_output_function_has_complete_digests():
    """All 2^32 inputs of the 18 single-output binary32 functions are covered (sincosf is
    checked on the GPU through its equality with sinf and cosf)."""
    funcs = ["expf", "exp2f", "exp10f", "expm1f", "logf", "log2f", "log10f", "log1pf", "sinf", "cosf",
             "tanf", "asinf", "acosf", "atanf", "sinhf", "coshf", "tanhf", "rsqrtf"]
    for f in funcs:
        d = EH.read_fixture(os.path.join(GOLDEN, f + ".txt"))
        assert sorted(d) == list(range(EH.NCHUNKS)), f
