"""Exact rational referee for small N (TEST INFRASTRUCTURE ONLY).

The forward Chebyshev--Jacobi map c_cheb = T_N^{-1} P_N c_jac does not depend
on the interpolation points: because a polynomial of degree <= N is
reproduced exactly by interpolation at N+1 distinct points, c_cheb is simply
the Chebyshev expansion of sum_n c_n P_n^{(alpha,beta)}.  This module
computes that expansion in exact rational arithmetic (``fractions``), with
P_n taken from Rodrigues' formula (Sec. 1.2) expanded by Leibniz' rule:

  P_n(x) = (-1)^n / (2^n n!) sum_k C(n,k) (-1)^k (alpha+n)_{(k)} (beta+n)_{(n-k)}
           (1-x)^{n-k} (1+x)^k

where (a)_{(k)} = a (a-1) ... (a-k+1) is the falling factorial.  It uses
neither the three-term recurrence nor any point set, so it pins the
recurrence coefficients and the DCT of the double-double oracle by an
independent route.  Parameters and inputs are converted with
``Fraction(float)``, i.e. exactly the binary value the other paths see.

The inverse map is obtained by exact back substitution, since the
Jacobi-to-Chebyshev connection matrix is upper triangular.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb


def _falling(a: Fraction, k: int) -> Fraction:
    r = Fraction(1)
    for i in range(k):
        r *= a - i
    return r


def _polymul(p, q):
    out = [Fraction(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        if a == 0:
            continue
        for j, b in enumerate(q):
            out[i + j] += a * b
    return out


def _polypow(p, e):
    r = [Fraction(1)]
    for _ in range(e):
        r = _polymul(r, p)
    return r


def jacobi_monomial(n: int, alpha, beta):
    """Monomial coefficients (lowest first) of P_n^{(alpha,beta)} via Rodrigues' formula."""
    a, b = Fraction(alpha), Fraction(beta)
    one_minus = [Fraction(1), Fraction(-1)]
    one_plus = [Fraction(1), Fraction(1)]
    acc = [Fraction(0)] * (n + 1)
    for k in range(n + 1):
        coef = comb(n, k) * (-1) ** k * _falling(a + n, k) * _falling(b + n, n - k)
        term = _polymul(_polypow(one_minus, n - k), _polypow(one_plus, k))
        for i, t in enumerate(term):
            acc[i] += coef * t
    scale = Fraction((-1) ** n, 2 ** n)
    for i in range(1, n + 1):
        scale /= i
    return [scale * t for t in acc]


def monomial_to_chebyshev_matrix(K: int):
    """M[k] = Chebyshev coefficients of x^k, using x T_0 = T_1, x T_j = (T_{j-1}+T_{j+1})/2."""
    M = [[Fraction(0)] * (K + 1) for _ in range(K + 1)]
    M[0][0] = Fraction(1)
    for k in range(K):
        row = M[k]
        nxt = M[k + 1]
        for j, v in enumerate(row):
            if v == 0:
                continue
            if j == 0:
                nxt[1] += v
            else:
                nxt[j - 1] += v / 2
                if j + 1 <= K:
                    nxt[j + 1] += v / 2
    return M


def connection_matrix(N: int, alpha, beta):
    """Q[n][k] = coefficient of T_k in P_n^{(alpha,beta)} (exact), n, k = 0..N."""
    M = monomial_to_chebyshev_matrix(N)
    Q = []
    for n in range(N + 1):
        mono = jacobi_monomial(n, alpha, beta)
        row = [Fraction(0)] * (N + 1)
        for i, m in enumerate(mono):
            if m == 0:
                continue
            for k, v in enumerate(M[i]):
                if v:
                    row[k] += m * v
        Q.append(row)
    return Q


def forward_exact(c_jac, alpha, beta):
    """Exact c_cheb for the given float coefficients (returned as Fractions)."""
    N = len(c_jac) - 1
    Q = connection_matrix(N, alpha, beta)
    out = [Fraction(0)] * (N + 1)
    for n, c in enumerate(c_jac):
        cf = Fraction(float(c))
        if cf == 0:
            continue
        for k in range(n + 1):
            out[k] += cf * Q[n][k]
    return out


def inverse_exact(c_cheb, alpha, beta):
    """Exact c_jac with sum_n c_jac_n P_n = sum_k c_cheb_k T_k (back substitution)."""
    N = len(c_cheb) - 1
    Q = connection_matrix(N, alpha, beta)
    rhs = [Fraction(float(c)) for c in c_cheb]
    out = [Fraction(0)] * (N + 1)
    for k in range(N, -1, -1):
        s = rhs[k]
        for n in range(k + 1, N + 1):
            s -= out[n] * Q[n][k]
        out[k] = s / Q[k][k]
    return out
