"""Writes the exact-rational golden fixtures under tests/golden/.

It calls only oracle/exact_rational.py (Rodrigues' formula in exact rational
arithmetic).  The parameters (alpha, beta) = (1/8, 3/8) are the ones of the
paper's Fig. 1 (Sec. 2.2); the input is c_n = 1/(n+1) rounded to double.
Run:  python tests/golden/make_golden.py
"""
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact_rational as ex  # noqa: E402


def write(name, N, alpha, beta, direction):
    c = [1.0 / (n + 1) for n in range(N + 1)]
    out = ex.forward_exact(c, alpha, beta) if direction == "forward" else ex.inverse_exact(c, alpha, beta)
    with open(os.path.join(HERE, name), "w") as f:
        f.write("# exact %s Chebyshev--Jacobi transform (Eq. %s), written by make_golden.py\n"
                % (direction, "CJT" if direction == "forward" else "iCJT"))
        f.write("# alpha: %s\n# beta: %s\n# N: %d\n" % (Fraction(alpha), Fraction(beta), N))
        f.write("# columns: input c_n (exact binary value of 1/(n+1)), exact output\n")
        for a, b in zip(c, out):
            f.write("%s %s\n" % (Fraction(a), b))


if __name__ == "__main__":
    write("forward_exact_N12_a1o8_b3o8.txt", 12, 0.125, 0.375, "forward")
    write("inverse_exact_N12_a1o8_b3o8.txt", 12, 0.125, 0.375, "inverse")
