"""Writes the full-size oracle fixtures under tests/golden/ (binary .npz files).

It calls only oracle/ (the CPU oracle) and paper_1602_02618_gb300/inputs.py (the
seeded generators, which hold no arithmetic of the method).  Each fixture holds the
oracle's output for one seeded workload item, so that the GPU parity tests can
compare the CUDA path element by element at the benchmark's sizes without running
an O(N^2) oracle at test time.

Items:
  * the single-transform workload (N = 2^12, 2^14, 2^16, 2^18, its seeded
    (alpha, beta) and coefficients c_n = g_n/(n+1)^1.5): the forward transform
    (Eq. "CJT") of c, and the inverse transform (Eq. "iCJT") of the same vector
    read as Chebyshev coefficients; double-double oracle, every output entry;
  * the inverse transform at N = 2^16 for the two shifted parameter pairs (one of
    alpha, beta in (1/2, 3/2], Sec. 1.2), double-double oracle, every output entry;
  * the first two items of the large mixed-precision workload (64 x N = 2^20):
    item 0 (forward) by the double-double oracle, item 1 (inverse) by the
    plain-double oracle (orc_inverse_f64; the double-double inverse at 2^20 takes
    hours on a CPU).  The plain-double error, measured against the double-double
    oracle at N = 2^14 and 2^16, is written beside it; it lies orders of magnitude
    below the mixed form's bound that the fixture is used against.  Both keep
    8192 sampled outputs (both ends and a seeded random sample).
An empty `idx` array means the fixture holds every output entry in order.

Run:  python tests/golden/make_fullsize.py [--only NAME ...] [--threads T]
Fixture names: fwd_N4096 ... inv_N262144, shift0_inv_N65536, shift1_inv_N65536,
fwd_N1048576, inv_N1048576.
"""
import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc  # noqa: E402
from paper_1602_02618_gb300 import inputs  # noqa: E402

SINGLE_NS = (1 << 12, 1 << 14, 1 << 16, 1 << 18)
BIG_N = 1 << 20
NSAMPLE = 8192


def digest(c):
    return hashlib.sha256(np.ascontiguousarray(c, dtype=np.float64).tobytes()).hexdigest()


def sample_indices(N, seed):
    ends = np.concatenate([np.arange(0, 128), np.arange(N - 127, N + 1)])
    rest = inputs.rng(seed).choice(np.arange(128, N - 127), NSAMPLE - ends.size, replace=False)
    return np.unique(np.concatenate([ends, rest])).astype(np.int64)


def items():
    """(name, N, alpha, beta, direction, input, oracle kind, workload description)."""
    out = []
    for N, a, b, c in inputs.single_workload(Ns=SINGLE_NS, seed=inputs.BASE_SEED):
        desc = "single-transform workload, c_n = g_n/(n+1)^1.5"
        out.append(("fwd_N%d" % N, N, a, b, 1, c, "double-double", desc))
        out.append(("inv_N%d" % N, N, a, b, -1, c, "double-double", desc + " read as Chebyshev coefficients"))
    for t, (N, a, b, c) in enumerate(inputs.shifted_workload()):
        out.append(("shift%d_inv_N%d" % (t, N), N, a, b, -1, c, "double-double",
                    "shifted parameters (%g, %g), c_n = g_n/(n+1)^1.5, read as Chebyshev coefficients" % (a, b)))
    big = inputs.mixed_large_workload(2, BIG_N, seed=inputs.BASE_SEED)
    (N0, a0, b0, d0, c0), (N1, a1, b1, d1, c1) = big
    desc = "mixed-precision workload (64 x N = 2^20), item %d, c_n = g_n/(n+1)"
    out.append(("fwd_N%d" % N0, N0, a0, b0, d0, c0, "double-double", desc % 0))
    out.append(("inv_N%d" % N1, N1, a1, b1, d1, c1, "plain double", desc % 1))
    return out


def plain_double_error():
    """max |inverse_f64 - inverse| / ||c||_1 at N = 2^14 and 2^16 on the single workload's inputs."""
    res = {}
    for N, a, b, c in inputs.single_workload(Ns=(1 << 14, 1 << 16), seed=inputs.BASE_SEED):
        ref = orc.inverse(c, a, b)
        res[N] = float(np.abs(orc.inverse_f64(c, a, b) - ref).max() / np.abs(c).sum())
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    orc.build()
    for name, N, a, b, d, c, kind, desc in items():
        if args.only and name not in args.only:
            continue
        t0 = time.perf_counter()
        if kind == "double-double":
            y = orc.forward(c, a, b, nthreads=args.threads) if d == 1 else orc.inverse(c, a, b, nthreads=args.threads)
        else:
            y = orc.inverse_f64(c, a, b, nthreads=args.threads)
        secs = time.perf_counter() - t0
        extra = {}
        if N == BIG_N:
            idx = sample_indices(N, inputs.BASE_SEED + 9000 + (0 if d == 1 else 1))
            y = y[idx]
            if kind == "plain double":
                err = plain_double_error()
                extra = {"f64_err_N16384": err[1 << 14], "f64_err_N65536": err[1 << 16]}
        else:
            idx = np.zeros(0, dtype=np.int64)   # empty: every output entry, in order
        np.savez(os.path.join(HERE, "oracle_%s.npz" % name), N=N, alpha=a, beta=b, direction=d,
                 idx=idx, out=y, input_sha256=digest(c), oracle=kind, workload=desc, seconds=secs,
                 threads=args.threads or (os.cpu_count() or 1), **extra)
        print("%s: %s oracle, %.1f s" % (name, kind, secs), flush=True)


if __name__ == "__main__":
    main()
