"""Writes tests/golden/exhaustive/<func>.txt: the chunk digests of the oracle's results
over all 2^32 binary32 inputs (digest definition in tests/exhaustive_hash.py).

Calls only the oracle.  Resumable: chunks already present in a file are skipped, and each
chunk is appended as soon as it is done, so a partial file lists the chunks covered so far.

    python tests/golden/make_exhaustive.py [--threads T] [--out-dir D] [--mode M] func [func ...]

--mode rd|ru|rz digests the results rounded toward -inf, +inf or zero instead (files under
exhaustive_<mode>/ by default).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import exhaustive_hash as EH  # noqa: E402
from oracle import oracle as O  # noqa: E402

OUT_DIR = os.path.join(HERE, "exhaustive")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("funcs", nargs="+")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out-dir", default=None, help="where the files go (default: next to this script)")
    ap.add_argument("--mode", default="rn", choices=["rn", "rd", "ru", "rz"])
    args = ap.parse_args()
    if args.out_dir is None:
        args.out_dir = OUT_DIR if args.mode == "rn" else OUT_DIR + "_" + args.mode
    os.makedirs(args.out_dir, exist_ok=True)
    w1, w2 = EH.weights()
    for f in args.funcs:
        if f not in O.FUNCS[:19] or f == "sincosf":
            raise SystemExit(f"{f}: not a single-output binary32 function")
        path = os.path.join(args.out_dir, f + ".txt")
        done = EH.read_fixture(path) if os.path.exists(path) else {}
        if not os.path.exists(path):
            with open(path, "w") as fh:
                how = "" if args.mode == "rn" else f", rounded {args.mode.upper()}"
                fh.write(f"# {f}: oracle results over all 2^32 binary32 inputs{how}, {EH.NCHUNKS} chunks"
                         f" of 2^{EH.CHUNK_LOG2} consecutive bit patterns\n")
                fh.write("# columns: chunk s h1 h2 (digest defined in tests/exhaustive_hash.py)\n")
                opt = "" if args.mode == "rn" else f" --mode {args.mode}"
                fh.write(f"# written by: python tests/golden/make_exhaustive.py{opt} {f}\n")
        t0 = time.time()
        for c in range(EH.NCHUNKS):
            if c in done:
                continue
            y = O.eval_bits(f, EH.chunk_bits(c), args.threads, mode=args.mode)
            s, h1, h2 = EH.digest_np(y, w1, w2)
            with open(path, "a") as fh:
                fh.write(f"{c} {s} {h1} {h2}\n")
            print(f"{f} chunk {c} {time.time() - t0:.0f}s", flush=True)


if __name__ == "__main__":
    main()
