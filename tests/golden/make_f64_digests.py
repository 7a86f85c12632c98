"""Writes tests/golden/f64_full/<label>.txt: digests of the oracle's results on every
element of the eight binary64 workload arrays (2^26 inputs each: exp2 uniform on
(-1075, 1024) and on the paper's [-20, 20]; log on uniform positive finite bit patterns and
on the paper's [0.125, 8]; exp on (-745, 710), exp10 on (-324, 309), log2 and log10 on
positive finite bit patterns), generated on the host by the seeded recipe of
paper_2605_15547_gb300/workloads.py (bench_input_host).

The 2^26 uint64 results are read as 2^27 uint32 words (little-endian halves), cut into 8
chunks of 2^24 words and digested like the exhaustive binary32 sweeps
(tests/exhaustive_hash.py).  Calls only the oracle.

    python tests/golden/make_f64_digests.py [--threads T] [label ...]
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import exhaustive_hash as EH  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2605_15547_gb300 import workloads as W  # noqa: E402

OUT_DIR = os.path.join(HERE, "f64_full")
N = 1 << 26
ARRAYS = [("exp2:domain", "exp2"), ("exp2:u20", "exp2"), ("log:bits", "log"), ("log:u0.125_8", "log"),
          ("exp:edomain", "exp"), ("exp10:tdomain", "exp10"), ("log2:bits", "log2"), ("log10:bits", "log10")]


def fname(label: str) -> str:
    return label.replace(":", "_") + ".txt"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("labels", nargs="*", help="arrays to write (default: all)")
    args = ap.parse_args()
    os.makedirs(OUT_DIR, exist_ok=True)
    w1, w2 = EH.weights()
    for label, func in ARRAYS:
        if args.labels and label not in args.labels:
            continue
        x = W.bench_input_host("f64", label, func, N).view(np.uint64)
        y = O.eval_bits(func, x, args.threads).view(np.uint32)
        with open(os.path.join(OUT_DIR, fname(label)), "w") as fh:
            fh.write(f"# {label}: oracle results of {func} on the 2^26 inputs of "
                     f"workloads.bench_input_host('f64', '{label}', '{func}', 2^26)\n")
            fh.write("# the uint64 results as 2^27 uint32 words, 8 chunks of 2^24; columns: chunk s h1 h2 "
                     "(tests/exhaustive_hash.py)\n")
            fh.write("# written by: python tests/golden/make_f64_digests.py\n")
            for c in range(y.size // EH.CHUNK):
                s, h1, h2 = EH.digest_np(y[c * EH.CHUNK:(c + 1) * EH.CHUNK], w1, w2)
                fh.write(f"{c} {s} {h1} {h2}\n")
        print(label, "done", flush=True)


if __name__ == "__main__":
    main()
