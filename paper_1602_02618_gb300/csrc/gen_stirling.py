"""Generates stirling_coeffs.h: coefficients a_k of the Stirling series
Gamma(z) = sqrt(2 pi) z^(z-1/2) e^(-z) sum_k a_k z^(-k)   (Sec. 4.1, DLMF 5.11.10).

The a_k are derived here, in exact rational arithmetic, from the Bernoulli
numbers: log Gamma(z) - (z-1/2) log z + z - log(2 pi)/2 = sum_k B_2k / (2k(2k-1) z^(2k-1))
(DLMF 5.11.1), and the exponential of that power series in w = 1/z is built
with the recurrence  j a_j = sum_{i=1}^{j} i l_i a_{j-i}  (a_0 = 1).
Run:  python gen_stirling.py > stirling_coeffs.h
"""
from fractions import Fraction
from math import comb

NTERMS = 20


def bernoulli(nmax):
    B = [Fraction(1)]
    for m in range(1, nmax + 1):
        B.append(-sum(comb(m + 1, k) * B[k] for k in range(m)) / (m + 1))
    return B


def stirling(nterms):
    B = bernoulli(2 * nterms + 2)
    l = [Fraction(0)] * (nterms + 1)
    for k in range(1, nterms + 1):
        if 2 * k - 1 <= nterms:
            l[2 * k - 1] = B[2 * k] / (2 * k * (2 * k - 1))
    a = [Fraction(1)] + [Fraction(0)] * nterms
    for j in range(1, nterms + 1):
        a[j] = sum(i * l[i] * a[j - i] for i in range(1, j + 1)) / j
    return a


if __name__ == "__main__":
    a = stirling(NTERMS)
    print("/* Generated by gen_stirling.py -- do not edit. Stirling series coefficients")
    print(" * a_k of Gamma(z) = sqrt(2 pi) z^(z-1/2) e^(-z) sum_k a_k / z^k (Sec. 4.1). */")
    print("#pragma once")
    print("#define CJT_STIRLING_NCOEF %d" % (NTERMS + 1))
    print("#define CJT_STIRLING_LIST \\")
    for k, v in enumerate(a):
        tail = ", /* %s */ \\" % v if k + 1 < len(a) else " /* %s */" % v
        print("    %s%s" % (float(v).hex(), tail))
    print("static const double cjt_stirling_a_host[CJT_STIRLING_NCOEF] = {CJT_STIRLING_LIST};")
