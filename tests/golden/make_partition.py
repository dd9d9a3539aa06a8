"""Writes tests/golden/partition_ref.json: the paper's partition (Sec. 2.2) of the forward
grid (Ng = G) and of the inverse transform's 2G grid for a few (N, alpha, beta, M), computed
by oracle/partition.py (mpmath, 40 digits) and nothing else.  G is the grid a plan evaluates
on: for N of the forms 2^a, 3 2^a and 5 2^a, N itself; otherwise the least integer >= N of those
forms (the default, plan option grid = 0) and the least power of two >= N (grid = 1).
Run:  python tests/golden/make_partition.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import partition as P  # noqa: E402

CASES = [(1024, 0.1, -0.3, 7), (16384, 0.1, -0.3, 7), (4096, -0.45, 0.2, 13), (65536, 0.3, 0.1, 10),
         (3001, 0.2, -0.1, 7), (1 << 18, 0.1, -0.3, 13), (40000, -0.3, 0.35, 13)]


def main():
    out = []
    for N, a, b, M in CASES:
        G2 = 1
        while G2 < N:
            G2 <<= 1
        G3, G5 = 3, 5
        while G3 < N:
            G3 <<= 1
        while G5 < N:
            G5 <<= 1
        G0 = min(G2, G3, G5)
        grids = [(0, G0)] + ([(1, G2)] if G0 < G2 else [])
        for grid, G in grids:
            for direction, Ng in (("forward", G), ("inverse", 2 * G)):
                nM, r, blocks = P.partition(Ng, N, M, a, b)
                out.append({"N": N, "alpha": a, "beta": b, "M": M, "grid": grid, "direction": direction, "Ng": Ng,
                            "n_M": nM, "ratio": r, "blocks": [list(blk) for blk in blocks]})
                print(out[-1], flush=True)
    with open(os.path.join(HERE, "partition_ref.json"), "w") as f:
        json.dump({"source": "oracle/partition.py (mpmath, 40 digits), Sec. 2.2", "cases": out}, f, indent=1)


if __name__ == "__main__":
    main()
