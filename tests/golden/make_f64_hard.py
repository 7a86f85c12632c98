"""Writes tests/golden/f64_hard/<func>.txt: binary64 inputs of exp2, log (and of exp, log2,
log10, exp10) whose results
lie closest to a rounding boundary (a midpoint between two binary64 numbers), selected by
the oracle alone.

The fast paths decide a result only when no midpoint lies within their error bound of the
approximation; inputs whose exact result is within 2^-h ulp of a midpoint, for h beyond
those bounds, are the ones that exercise the rounding tests and the slow paths (the
hard-to-round cases of Sec. II.B; the published hard-case sets are not available here, so
this search stands in for them).  About 10^7 candidates per function are drawn from seeded
families (below) and the oracle's distance diagnostic (oracle.f64_hardness) ranks them;
the 10^4 closest are kept.

Candidate families (numpy PCG64, seed 0xC0DE0500 + function id):
  exp2: x whose 2^x sits near 1 + (j + 1/2) 2^-52 or 1 - (j + 1/2) 2^-53 (x ~ (j + 1/2)
        2^-52 / ln 2 and neighbours: 2^x = 1 + x ln 2 + ..., hardness up to ~55 bits);
        x near integers (k + i ulp(k)); x near the subnormal and overflow ends; uniform
        over the domain and over the paper's [-20, 20]; tiny |x|.
  log:  x = 1 + 2^a o 2^-52 and 1 - 2^a o 2^-53 (o odd: log x = t - t^2/2 + ..., whose
        second term lands on a half-ulp when a is o's bit length less one, or o's bit length
        for x < 1); x near 1; near powers of two; subnormal; near
        the largest double; uniform positive bit patterns and the paper's [0.125, 8].

    python tests/golden/make_f64_hard.py [--keep 10000] [--threads T]
"""
from __future__ import annotations

import argparse
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

OUT_DIR = os.path.join(HERE, "f64_hard")
LN2 = math.log(2.0)


def _bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)


def neighbours(x, r, rng, count):
    """count doubles within r ulps of each x (the bit patterns of positive finite x)."""
    b = np.repeat(_bits(np.abs(x)), count)
    off = rng.integers(-r, r + 1, b.size, dtype=np.int64)
    nb = (b.astype(np.int64) + off).astype(np.uint64)
    sign = np.repeat(np.signbit(x), count)
    return nb.view(np.float64) * np.where(sign, -1.0, 1.0)


def exp2_candidates(rng):
    parts = []
    # near 1 + (j + 1/2) 2^-52 and 1 - (j + 1/2) 2^-53: j log-uniform in [0, 2^24)
    j = np.floor(np.exp2(rng.uniform(0, 24, 40000))) - 1
    j = np.concatenate([np.arange(0, 512), j])
    xp = (j + 0.5) * 2.0 ** -52 / LN2
    xn = -(j + 0.5) * 2.0 ** -53 / LN2
    parts += [neighbours(xp, 64, rng, 40), neighbours(xn, 64, rng, 40)]
    # near integers, in every binade of the result
    k = rng.integers(-1074, 1024, 1_500_000).astype(np.float64)
    ulp = np.spacing(np.maximum(np.abs(k), 1.0))
    i = np.round(rng.uniform(-1, 1, k.size) * np.exp2(rng.uniform(0, 30, k.size)))
    parts.append(np.where(k == 0, i * 2.0 ** -80, k + i * ulp))
    parts += [rng.uniform(-1075.0, 1024.0, 1_500_000), rng.uniform(-20.0, 20.0, 1_500_000),
              rng.uniform(-1076.0, -1020.0, 1_000_000), rng.uniform(1016.0, 1024.0, 500_000),
              np.where(rng.integers(0, 2, 1_000_000) == 1, 1.0, -1.0) * np.exp2(rng.uniform(-80, -1, 1_000_000))]
    return np.concatenate(parts)


def log_candidates(rng):
    parts = []
    # 1 + 2^a o 2^-52 and 1 - 2^a o 2^-53, o odd
    a = rng.integers(0, 44, 1_000_000)
    o = 2 * np.floor(np.exp2(rng.uniform(0, 14, a.size))) + 1
    m = np.exp2(a) * o
    m = m[m < 2.0 ** 50]
    parts += [1.0 + m * 2.0 ** -52, 1.0 - m * 2.0 ** -53]
    # the same with the second term exactly on a half-ulp, so that the distance is the third
    # term's: x = 1 + 2^(B-1) o 2^-52 and 1 - 2^B o 2^-53 with B the bit length of o
    # (t^2/2 = o^2/2 ulps, o odd), h about 54.6 - 4B
    o = np.arange(1, 1 << 16, 2, dtype=np.float64)
    B = np.floor(np.log2(o)) + 1
    parts += [1.0 + np.exp2(B - 1) * o * 2.0 ** -52, 1.0 - np.exp2(B) * o * 2.0 ** -53]
    # near 1, near powers of two, subnormal, near the largest double
    parts.append(1.0 + rng.uniform(-1, 1, 1_500_000) * np.exp2(rng.uniform(-52, -4, 1_500_000)))
    e = rng.integers(-1074, 1024, 1_500_000).astype(np.float64)
    parts.append(np.exp2(e) * (1.0 + rng.uniform(-1, 1, e.size) * np.exp2(rng.uniform(-52, -2, e.size))))
    parts.append(rng.integers(1, 1 << 52, 700_000, dtype=np.uint64).view(np.float64))
    big = (np.uint64(0x7FEFFFFFFFFFFFFF) - rng.integers(0, 1 << 44, 300_000, dtype=np.uint64))
    parts.append(big.view(np.float64))
    bits = rng.integers(1, 0x7FF0000000000000, 1_500_000, dtype=np.uint64)
    parts += [bits.view(np.float64), rng.uniform(0.125, 8.0, 1_500_000)]
    x = np.concatenate(parts)
    return x[np.isfinite(x) & (x > 0)]


def exp_candidates(rng, hi, lo, lnb):
    """b^x: near 0, where b^x = 1 + x ln b + ... sits next to the midpoints 1 + (j + 1/2) 2^-52
    and 1 - (j + 1/2) 2^-53 for x ~ (j + 1/2) 2^-52 / ln b (and neighbours); near the range
    ends, uniform, near integers"""
    j = np.floor(np.exp2(rng.uniform(0, 24, 40000))) - 1
    j = np.concatenate([np.arange(0, 512), j])
    parts = [neighbours((j + 0.5) * 2.0 ** -52 / lnb, 64, rng, 40), neighbours(-(j + 0.5) * 2.0 ** -53 / lnb, 64, rng, 40)]
    parts += [rng.uniform(lo, hi, 2_000_000), rng.uniform(-20.0, 20.0, 1_500_000),
             np.where(rng.integers(0, 2, 1_000_000) == 1, 1.0, -1.0) * np.exp2(rng.uniform(-80, -1, 1_000_000)),
             rng.uniform(hi - 8.0, hi, 500_000), rng.uniform(lo, lo + 30.0, 500_000)]
    k = rng.integers(int(lo), int(hi), 1_000_000).astype(np.float64)
    i = np.round(rng.uniform(-1, 1, k.size) * np.exp2(rng.uniform(0, 30, k.size)))
    parts.append(k + i * np.spacing(np.maximum(np.abs(k), 1.0)))
    return np.concatenate(parts)


def logb_candidates(rng):
    """log2, log10: the log families (near 1, near powers of two, bit patterns)"""
    return log_candidates(rng)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--keep", type=int, default=10000)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--funcs", default="", help="comma list (default: all)")
    args = ap.parse_args()
    os.makedirs(OUT_DIR, exist_ok=True)
    gens = (("exp2", exp2_candidates), ("log", log_candidates),
            ("exp", lambda r: exp_candidates(r, 709.7, -745.0, 1.0)), ("log2", logb_candidates),
            ("log10", logb_candidates), ("exp10", lambda r: exp_candidates(r, 308.2, -323.5, math.log(10.0))))
    for func, gen in gens:
        if args.funcs and func not in args.funcs.split(","):
            continue
        seed = 0xC0DE0500 + O.FUNC_ID[func]
        rng = np.random.Generator(np.random.PCG64(seed))
        xb = np.unique(_bits(gen(rng)))
        h = O.f64_hardness(func, xb, args.threads)
        order = np.lexsort((xb, -h))[:args.keep]
        with open(os.path.join(OUT_DIR, func + ".txt"), "w") as fh:
            fh.write(f"# {func}: the {args.keep} inputs (of {xb.size} seeded candidates, seed {seed:#x}) whose\n"
                     "# results lie closest to a binary64 rounding midpoint; columns: input bit pattern (hex),\n"
                     "# h = -log2(distance to the midpoint in ulps), from the oracle (f64_hardness)\n"
                     "# written by: python tests/golden/make_f64_hard.py\n")
            for b, hv in zip(xb[order], h[order]):
                fh.write(f"{int(b):016x} {hv:.3f}\n")
        hk = h[order]
        print(f"{func}: {xb.size} candidates, kept {hk.size}: h from {hk.min():.1f} to {hk.max():.1f}, "
              f"{int((h > 30).sum())} candidates beyond 30 bits", flush=True)


if __name__ == "__main__":
    main()
