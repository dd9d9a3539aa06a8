"""The paper's partition of the matrix P_N (Sec. 2.2) in high precision (TEST INFRASTRUCTURE ONLY).

Only tests and tests/golden/make_partition.py use this module; the library never does.  It
evaluates, in mpmath at 40 digits and straight from the paper's formulas:

  C_{n,m}  = 2^(2n-m+a+b+1) B(n+a+1, n+b+1) / (pi (2n+a+b+2)_m)              (Eq. "Cnmab")
  g_m(t)   = sum_{l=0..m} (1/2+a)_l (1/2-a)_l (1/2+b)_{m-l} (1/2-b)_{m-l} / (l! (m-l)!)
             cos(t/2)^(l-m-b-1/2) / sin(t/2)^(l+a+1/2)         (the envelope of |f_m|, Sec. 2.2)
  n_M      = floor((eps 2^(2M-1) sqrt(pi) / g_M(pi/2))^(-1/(M+1/2)))
  alpha_N  = min(1/log(Ng/n_M), 1/2),  j_k = floor(alpha_N^k Ng) while j_k > n_M (and j_k >= 2)
  box k    = the rows i in (0, Ng) with 2 C_{j_k,M} g_M(pi i/Ng) < eps: an interval around the
             discrete minimiser of g_M (g_M is unimodal); the first empty box ends the blocks.

These follow the readings the library documents for the places where the paper is silent or
garbled: the envelope g_M(pi/2) in n_M (the paper writes |f_M(pi/2)|, which depends on n), j_k
rounded down, the strict inequality, interior rows only, and for the inverse transform the
2N grid with the blocks whose degrees all exceed N dropped (Sec. 3.2).  Ng is the evaluation
grid (N, or the power of two G >= N the library uses when N is not one).
"""
from __future__ import annotations

import math

import mpmath as mp

DPS = 40


def hahn_C(n, m, a, b):
    """C_{n,m}^{(a,b)} of Eq. "Cnmab"."""
    with mp.workdps(DPS):
        a, b = mp.mpf(a), mp.mpf(b)
        return mp.power(2, 2 * n - m + a + b + 1) * mp.beta(n + a + 1, n + b + 1) / (mp.pi * mp.rf(2 * n + a + b + 2, m))


def envelope(m, theta, a, b):
    """g_m(theta), the envelope of |f_m(theta)| (Sec. 2.2)."""
    with mp.workdps(DPS):
        a, b = mp.mpf(a), mp.mpf(b)
        s, c = mp.sin(theta / 2), mp.cos(theta / 2)
        total = mp.mpf(0)
        for l in range(m + 1):
            coef = (mp.rf(0.5 + a, l) * mp.rf(0.5 - a, l) * mp.rf(0.5 + b, m - l) * mp.rf(0.5 - b, m - l) /
                    (mp.factorial(l) * mp.factorial(m - l)))
            if coef == 0:
                continue
            total += coef * mp.power(c, l - m - b - 0.5) / mp.power(s, l + a + 0.5)
        return total


def n_M(M, a, b, eps=2.0 ** -52):
    with mp.workdps(DPS):
        v = (mp.mpf(eps) * mp.power(2, 2 * M - 1) * mp.sqrt(mp.pi) / envelope(M, mp.pi / 2, a, b)) ** (
            -mp.mpf(1) / (M + mp.mpf(0.5)))
        return int(mp.floor(v))


def criterion_margin(j, i, Ng, M, a, b, eps=2.0 ** -52):
    """eps - 2 C_{j,M} g_M(pi i / Ng): positive where the asymptotic formula is accurate."""
    with mp.workdps(DPS):
        return mp.mpf(eps) - 2 * hahn_C(j, M, a, b) * envelope(M, mp.pi * i / Ng, a, b)


def _argmin(Ng, M, a, b):
    """The discrete minimiser of the unimodal g_M over the interior rows (ternary search)."""
    lo, hi = 1, Ng - 1
    g = lambda i: envelope(M, mp.pi * i / Ng, a, b)
    while hi - lo > 2:
        m1 = lo + (hi - lo) // 3
        m2 = hi - (hi - lo) // 3
        if g(m1) < g(m2):
            hi = m2
        else:
            lo = m1
    return min(range(lo, hi + 1), key=g)


def partition(Ng, N, M, a, b, ratio=0.0, eps=2.0 ** -52):
    """(n_M, alpha_N, [(j_k, i_k^1, i_k^2), ...]) of the grid x_i = cos(pi i / Ng) for degree N
    (blocks with j_k > N dropped, as on the inverse transform's 2N grid)."""
    nM = n_M(M, a, b, eps)
    if nM < 1 or Ng <= nM:
        return nM, None, []
    r = ratio if ratio > 0 else min(1.0 / math.log(Ng / nM), 0.5)
    ibar = _argmin(Ng, M, a, b)
    blocks = []
    k = 1
    while True:
        with mp.workdps(DPS):
            j = int(mp.floor(mp.power(mp.mpf(r), k) * Ng))
        if j <= nM or j < 2:
            break
        ok = lambda i: criterion_margin(j, i, Ng, M, a, b, eps) > 0
        if not ok(ibar):
            break
        lo, hi = 1, ibar            # smallest row that satisfies it (g decreases up to ibar)
        while lo < hi:
            mid = (lo + hi) // 2
            if ok(mid):
                hi = mid
            else:
                lo = mid + 1
        i1 = lo
        lo, hi = ibar, Ng - 1       # largest row that satisfies it
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if ok(mid):
                lo = mid
            else:
                hi = mid - 1
        blocks.append((j, i1, lo))
        k += 1
    return nM, r, [blk for blk in blocks if blk[0] < N + 1]
