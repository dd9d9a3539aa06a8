"""Writes tests/golden/partition_ref.json: the paper's partition (Sec. 2.2) of the forward
grid (Ng = G) and of the inverse transform's 2G grid for a few (N, alpha, beta, M), computed
by oracle/partition.py (mpmath, 40 digits) and nothing else.  G is N, or the least power of
two >= N (the library's default grid for N not a power of two).
Run:  python tests/golden/make_partition.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import partition as P  # noqa: E402

CASES = [(1024, 0.1, -0.3, 7), (16384, 0.1, -0.3, 7), (4096, -0.45, 0.2, 13), (65536, 0.3, 0.1, 10),
         (3001, 0.2, -0.1, 7), (1 << 18, 0.1, -0.3, 13)]


def main():
    out = []
    for N, a, b, M in CASES:
        G = 1
        while G < N:
            G <<= 1
        for direction, Ng in (("forward", G), ("inverse", 2 * G)):
            nM, r, blocks = P.partition(Ng, N, M, a, b)
            out.append({"N": N, "alpha": a, "beta": b, "M": M, "direction": direction, "Ng": Ng, "n_M": nM,
                        "ratio": r, "blocks": [list(blk) for blk in blocks]})
            print(out[-1], flush=True)
    with open(os.path.join(HERE, "partition_ref.json"), "w") as f:
        json.dump({"source": "oracle/partition.py (mpmath, 40 digits), Sec. 2.2", "cases": out}, f, indent=1)


if __name__ == "__main__":
    main()
