"""Chunk digests for the exhaustive binary32 sweeps (test infrastructure).

The 2^32 input bit patterns of a one-input binary32 function are cut into 256 chunks of
2^24 consecutive patterns; chunk c holds the patterns c * 2^24 + i, i = 0 .. 2^24 - 1.
The outputs v_i (uint32 bit patterns) of a chunk are summarised by three integers:

    s  = sum_i v_i                                   (exact, < 2^56)
    h1 = sum_i ((v_i mod P) * w1_i mod P) mod P
    h2 = sum_i ((v_i mod P) * w2_i mod P) mod P      with P = 2^31 - 1,

where w1, w2 are fixed pseudo-random weights in [1, P) (numpy PCG64, seed WEIGHT_SEED).
For a fixed nonzero difference between two output vectors, each weighted sum collides
with probability about 1/P over the weights, and a difference that is a multiple of P in
every position still moves s.  The same arithmetic is written once for numpy (the oracle
side, on the host) and once for torch (the device side): all values stay below 2^63.
"""
from __future__ import annotations

import numpy as np

CHUNK_LOG2 = 24
CHUNK = 1 << CHUNK_LOG2
NCHUNKS = 1 << (32 - CHUNK_LOG2)
P = (1 << 31) - 1
WEIGHT_SEED = 0x5EEDE4A5


def weights() -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.Generator(np.random.PCG64(WEIGHT_SEED))
    w1 = rng.integers(1, P, CHUNK, dtype=np.int64)
    w2 = rng.integers(1, P, CHUNK, dtype=np.int64)
    return w1, w2


def chunk_bits(c: int) -> np.ndarray:
    return (np.arange(CHUNK, dtype=np.uint64) + (c << CHUNK_LOG2)).astype(np.uint32)


def digest_np(v: np.ndarray, w1: np.ndarray, w2: np.ndarray) -> tuple[int, int, int]:
    x = v.astype(np.uint32).astype(np.int64)
    xm = x % P
    s = int(x.sum())
    h1 = int(((xm * w1) % P).sum() % P)
    h2 = int(((xm * w2) % P).sum() % P)
    return s, h1, h2


def digest_torch(v, w1, w2) -> tuple[int, int, int]:
    """v: int32 tensor of output bit patterns (any device); w1, w2: int64 on that device."""
    import torch

    x = v.to(torch.int64) & 0xFFFFFFFF
    xm = torch.remainder(x, P)
    s = int(x.sum().item())
    h1 = int(torch.remainder(torch.remainder(xm * w1, P).sum(), P).item())
    h2 = int(torch.remainder(torch.remainder(xm * w2, P).sum(), P).item())
    return s, h1, h2


def read_fixture(path: str) -> dict[int, tuple[int, int, int]]:
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            c, s, h1, h2 = (int(t) for t in line.split())
            out[c] = (s, h1, h2)
    return out
