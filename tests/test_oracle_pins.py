"""Pins of the CPU oracle against things other than itself.

Each test ties an oracle routine to an independent fact fixed by the paper or
by mathematics: exact rational arithmetic through Rodrigues' formula (Sec. 1.2),
closed forms (alpha = beta = -1/2 scaled Chebyshev; alpha = beta = 0 Legendre
connection coefficients), endpoint values (Eq. "Pnendpts"), the symmetry
relation (Eq. "Pnsym"), library quadrature (Gauss--Jacobi from SciPy) for the
modified moments and the orthonormalisation constants (Eq. "Anab"),
mpmath Gamma functions, and a dense linear solve for the inverse map
(Eq. "iCJT").  Planted-mistake tests build copies of the oracle with one
plausible slip each (the mu_1 sign as printed in Sec. 3.1, a dropped B_n, the
missing halving of c_N, a Clenshaw--Curtis end factor, a wrong normalisation
constant) and show that a pin rejects every one.
"""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import mpmath
import numpy as np
import pytest
import scipy.special as sps

from oracle import exact_rational as ex
from paper_1602_02618_gb300 import inputs

mpmath.mp.prec = 160

PARAMS = [(0.125, 0.375), (0.1, -0.3), (-0.45, 0.45), (0.45, 0.45), (-0.3, -0.2), (0.0, 0.0),
          (-0.5, -0.5), (0.5, 0.5), (0.5, -0.5), (-0.5, 0.2)]


def l1(c):
    return float(np.sum(np.abs(c)))


# --------------------------------------------------------------------------
# Lobatto points
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p,q", [(1, 3), (1, 4), (1, 2), (0, 7), (7, 7), (5, 12), (3, 1024), (1000, 1024),
                                 (12345, 65536), (65535, 65536), (1, 262144), (131071, 262144), (-3, 5), (13, 5)])
def test_cospi_frac_matches_mpmath(orc, p, q):
    hi, lo = orc.cospi_frac(p, q)
    exact = mpmath.cos(mpmath.pi * p / q)
    err = abs(mpmath.mpf(hi) + mpmath.mpf(lo) - exact)
    assert err < 1e-30


def test_cospi_frac_rational_values(orc):
    assert orc.cospi_frac(1, 3) [0] == 0.5
    assert orc.cospi_frac(2, 3)[0] == -0.5
    assert orc.cospi_frac(1, 2) == (0.0, 0.0)
    assert orc.cospi_frac(0, 9)[0] == 1.0 and orc.cospi_frac(9, 9)[0] == -1.0
    # symmetry x_{N-j} = -x_j exactly
    for N in (10, 1024, 3001):
        for j in (1, 3, N // 3):
            a = orc.cospi_frac(j, N)
            b = orc.cospi_frac(N - j, N)
            assert a[0] == -b[0] and a[1] == -b[1]


# --------------------------------------------------------------------------
# Jacobi polynomials: recurrence vs Rodrigues' formula at rational points
# --------------------------------------------------------------------------
def _eval_poly(coeffs, x):
    r = Fraction(0)
    for c in reversed(coeffs):
        r = r * x + c
    return r


@pytest.mark.parametrize("alpha,beta", PARAMS)
def test_recurrence_matches_rodrigues(orc, alpha, beta):
    nmax = 24
    # grid_N = 3 gives the rational points 1, 1/2, -1/2, -1; grid_N = 2 gives 0
    for grid_N, j, x in [(3, 0, Fraction(1)), (3, 1, Fraction(1, 2)), (2, 1, Fraction(0)),
                         (3, 2, Fraction(-1, 2)), (3, 3, Fraction(-1))]:
        vals = orc.jacobi_values(nmax, alpha, beta, j, grid_N)
        for n in range(nmax + 1):
            exact = _eval_poly(ex.jacobi_monomial(n, alpha, beta), x)
            assert abs(vals[n] - float(exact)) <= 2e-15 * max(1.0, abs(float(exact))), (n, grid_N, j)


@pytest.mark.parametrize("alpha,beta", PARAMS)
def test_endpoint_values(orc, alpha, beta):
    """P_n(1) = C(n+alpha, n), P_n(-1) = (-1)^n C(n+beta, n)  (Eq. Pnendpts)."""
    nmax = 3000
    v1 = orc.jacobi_values(nmax, alpha, beta, 0, 5)
    vm1 = orc.jacobi_values(nmax, alpha, beta, 5, 5)
    for n in (0, 1, 2, 7, 100, 1999, 3000):
        b1 = mpmath.binomial(n + mpmath.mpf(alpha), n)
        bm1 = (-1) ** n * mpmath.binomial(n + mpmath.mpf(beta), n)
        assert abs(v1[n] - float(b1)) <= 1e-15 * max(1, abs(float(b1)))
        assert abs(vm1[n] - float(bm1)) <= 1e-15 * max(1, abs(float(bm1)))


def test_recurrence_matches_scipy_interior(orc):
    """Library check at irrational interior points (scipy eval_jacobi, double)."""
    alpha, beta = 0.1, -0.3
    for j, N in [(3, 7), (100, 257), (700, 1024)]:
        vals = orc.jacobi_values(60, alpha, beta, j, N)
        x = np.cos(np.pi * j / N)
        ref = sps.eval_jacobi(np.arange(61), alpha, beta, x)
        assert np.max(np.abs(vals - ref)) < 1e-12


# --------------------------------------------------------------------------
# forward transform
# --------------------------------------------------------------------------
@pytest.mark.parametrize("alpha,beta", PARAMS)
@pytest.mark.parametrize("N", [1, 2, 5, 12])
def test_forward_matches_exact_rational(orc, alpha, beta, N):
    c = inputs.decaying_coefficients(N, 1.0, seed=inputs.BASE_SEED + N)
    got = orc.forward(c, alpha, beta)
    exact = np.array([float(v) for v in ex.forward_exact(c, alpha, beta)])
    assert np.max(np.abs(got - exact)) <= 1e-15 * l1(c)


def test_forward_identity_at_N0(orc):
    assert orc.forward(np.array([3.25]), 0.2, 0.1)[0] == 3.25


def _read_golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    meta, rows = {}, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                if ":" in line:
                    k, v = line[1:].split(":", 1)
                    meta[k.strip()] = v.strip()
                continue
            rows.append([Fraction(t) for t in line.split()])
    return meta, rows


def test_forward_golden_fixture(orc):
    """Stored exact values (written by tests/golden/make_golden.py from the exact referee)."""
    meta, rows = _read_golden("forward_exact_N12_a1o8_b3o8.txt")
    alpha, beta = float(Fraction(meta["alpha"])), float(Fraction(meta["beta"]))
    c = np.array([float(r[0]) for r in rows])
    exact = np.array([float(r[1]) for r in rows])
    got = orc.forward(c, alpha, beta)
    assert np.max(np.abs(got - exact)) <= 1e-15 * l1(c)
    # and the referee still reproduces the stored fixture exactly
    again = ex.forward_exact(c, alpha, beta)
    assert all(a == r[1] for a, r in zip(again, rows))


def test_inverse_golden_fixture(orc):
    """Stored exact values of the inverse map (written by tests/golden/make_golden.py)."""
    meta, rows = _read_golden("inverse_exact_N12_a1o8_b3o8.txt")
    alpha, beta = float(Fraction(meta["alpha"])), float(Fraction(meta["beta"]))
    c = np.array([float(r[0]) for r in rows])
    exact = np.array([float(r[1]) for r in rows])
    got = orc.inverse(c, alpha, beta)
    assert np.max(np.abs(got - exact)) <= 1e-15 * l1(c)
    again = ex.inverse_exact(c, alpha, beta)
    assert all(a == r[1] for a, r in zip(again, rows))


def test_forward_chebyshev_closed_form(orc):
    """alpha = beta = -1/2: P_n = ((1/2)_n / n!) T_n, so c_cheb_n = ((1/2)_n/n!) c_n."""
    N = 300
    c = inputs.decaying_coefficients(N, 1.0, seed=7)
    got = orc.forward(c, -0.5, -0.5)
    scale = np.empty(N + 1)
    s = mpmath.mpf(1)
    for n in range(N + 1):
        scale[n] = float(s)
        s = s * (n + mpmath.mpf(0.5)) / (n + 1)
    assert np.max(np.abs(got - scale * c)) <= 2e-16 * l1(c)


def test_forward_legendre_closed_form(orc):
    """alpha = beta = 0: P_n = sum_k (2-delta_k0)/pi Lambda((n-k)/2) Lambda((n+k)/2) T_k, n-k even,
    Lambda(z) = Gamma(z+1/2)/Gamma(z+1) (the Legendre-to-Chebyshev connection coefficients)."""
    N = 160
    c = inputs.decaying_coefficients(N, 1.0, seed=11)
    lam = [mpmath.gamma(mpmath.mpf(z) / 2 + mpmath.mpf(0.5)) / mpmath.gamma(mpmath.mpf(z) / 2 + 1)
           for z in range(2 * N + 1)]   # lam[t] = Lambda(t/2)
    ref = np.zeros(N + 1)
    for k in range(N + 1):
        acc = mpmath.mpf(0)
        for n in range(k, N + 1, 2):
            acc += mpmath.mpf(c[n]) * lam[n - k] * lam[n + k]
        ref[k] = float(acc * (1 if k == 0 else 2) / mpmath.pi)
    got = orc.forward(c, 0.0, 0.0)
    assert np.max(np.abs(got - ref)) <= 2e-16 * l1(c) * 4


@pytest.mark.parametrize("alpha,beta", [(0.1, -0.3), (0.45, 0.45), (-0.45, 0.2)])
def test_forward_endpoint_sums_and_symmetry(orc, alpha, beta):
    N = 513
    c = inputs.decaying_coefficients(N, 1.5, seed=3)
    cc = orc.forward(c, alpha, beta)
    pa = np.empty(N + 1)
    pb = np.empty(N + 1)
    sa = sb = mpmath.mpf(1)
    for n in range(N + 1):
        pa[n], pb[n] = float(sa), float(sb)
        sa = sa * (n + 1 + mpmath.mpf(alpha)) / (n + 1)
        sb = sb * (n + 1 + mpmath.mpf(beta)) / (n + 1)
    sign = (-1.0) ** np.arange(N + 1)
    lhs1 = float(mpmath.fsum([mpmath.mpf(x) for x in cc]))
    rhs1 = float(mpmath.fsum([mpmath.mpf(x) * mpmath.mpf(y) for x, y in zip(c, pa)]))
    lhs2 = float(mpmath.fsum([mpmath.mpf(x) * s for x, s in zip(cc, sign)]))
    rhs2 = float(mpmath.fsum([mpmath.mpf(x) * mpmath.mpf(y) * s for x, y, s in zip(c, pb, sign)]))
    assert abs(lhs1 - rhs1) < 1e-14 * l1(c)
    assert abs(lhs2 - rhs2) < 1e-14 * l1(c)
    # Eq. Pnsym: F_{beta,alpha}((-1)^n c)_k = (-1)^k F_{alpha,beta}(c)_k
    cs = orc.forward(sign * c, beta, alpha)
    assert np.max(np.abs(cs - sign * cc)) < 1e-15 * l1(c)


def test_forward_f64_close_to_dd(orc):
    N = 700
    c = inputs.decaying_coefficients(N, 1.0, seed=5)
    a = orc.forward(c, 0.2, -0.1)
    b = orc.forward_f64(c, 0.2, -0.1)
    assert np.max(np.abs(a - b)) < 1e-13 * l1(c)


def test_series_evaluators(orc):
    N = 200
    c = inputs.decaying_coefficients(N, 1.0, seed=9)
    j = np.array([0, 1, 17, 100, 199, 200])
    # Chebyshev series vs numpy's chebval
    got = orc.cheb_series(c, j, N)
    ref = np.polynomial.chebyshev.chebval(np.cos(np.pi * j / N), c)
    assert np.max(np.abs(got - ref)) < 1e-13
    # Jacobi series vs dot with per-point values
    js = orc.jacobi_series(c, 0.3, -0.2, j, N)
    for q, jj in enumerate(j):
        v = orc.jacobi_values(N, 0.3, -0.2, int(jj), N)
        assert abs(js[q] - np.dot(v, c)) < 1e-13
    # values on the whole grid are what the forward transform interpolates
    hi, lo = orc.forward_values(c, 0.3, -0.2)
    cc = orc.forward(c, 0.3, -0.2)
    back = orc.cheb_series(cc, np.arange(N + 1), N)
    assert np.max(np.abs(back - hi)) < 1e-14 * l1(c)


def test_double_double_series_accuracy(orc):
    """The parity oracle evaluates sum_n c_n P_n(x_j) in double-double: hi + lo must agree
    with a 50-digit evaluation far beyond double precision, near x = +-1 too, where a
    plain-double recurrence loses about n^2 eps.  A slip in the error-free transformations
    (a dropped low part) would leave every double-precision pin passing but fail here."""
    mpmath.mp.dps = 50
    N, a, b = 1500, 0.1, -0.3
    c = inputs.decaying_coefficients(N, 1.0, seed=inputs.BASE_SEED + 55)
    j = np.array([1, 2, 7, N // 2, N - 3, N - 1])
    hi, lo = orc.jacobi_series(c, a, b, j, N, lo=True)
    A_, B_ = mpmath.mpf(a), mpmath.mpf(b)
    # the recurrence checked against mpmath's hypergeometric Jacobi polynomials first
    x_chk = mpmath.cos(mpmath.pi * 7 / N)
    for jj, x in zip(j, [mpmath.cos(mpmath.pi * int(q) / N) for q in j]):
        pm, p, s, mag = mpmath.mpf(0), mpmath.mpf(1), mpmath.mpf(c[0]), abs(mpmath.mpf(c[0]))
        for n in range(N):
            nn = mpmath.mpf(n)
            if n == 0:
                An, Bn, Cn = (A_ + B_ + 2) / 2, (A_ - B_) / 2, mpmath.mpf(0)
            else:
                t0 = 2 * nn + A_ + B_
                den = 2 * (nn + 1) * (nn + A_ + B_ + 1) * t0
                An = (t0 + 1) * (t0 + 2) * t0 / den
                Bn = (A_ * A_ - B_ * B_) * (t0 + 1) / den
                Cn = 2 * (nn + A_) * (nn + B_) * (t0 + 2) / den
            pm, p = p, (An * x + Bn) * p - Cn * pm
            if jj == 7 and n + 1 in (2, 500, N):
                assert abs(p - mpmath.jacobi(n + 1, A_, B_, x_chk)) < mpmath.mpf(10) ** -40 * (1 + abs(p))
            s += mpmath.mpf(c[n + 1]) * p
            mag += abs(mpmath.mpf(c[n + 1]) * p)
        q = list(j).index(jj)
        err = abs(mpmath.mpf(hi[q]) + mpmath.mpf(lo[q]) - s)
        assert err <= mpmath.mpf(10) ** -27 * mag, (int(jj), float(err), float(mag))
    # the Chebyshev side of the grid evaluation likewise
    hc, lc = orc.cheb_series(c, j, N, lo=True)
    for q, jj in enumerate(j):
        th = mpmath.pi * int(jj) / N
        s = mpmath.fsum(mpmath.mpf(c[k]) * mpmath.cos(k * th) for k in range(N + 1))
        assert abs(mpmath.mpf(hc[q]) + mpmath.mpf(lc[q]) - s) <= mpmath.mpf(10) ** -27 * l1(c)


# --------------------------------------------------------------------------
# inverse transform and its ingredients
# --------------------------------------------------------------------------
@pytest.mark.parametrize("alpha,beta", [(0.125, 0.375), (0.1, -0.3), (-0.5, -0.5), (0.5, 0.5), (0.45, -0.45)])
def test_moments_match_gauss_jacobi(orc, alpha, beta):
    """mu_k = int T_k (1-x)^a (1+x)^b dx vs SciPy's Gauss-Jacobi rule (exact to degree 2q-1)."""
    K = 100
    mu = orc.moments(K, alpha, beta)
    x, w = sps.roots_jacobi(80, alpha, beta)
    ref = np.array([np.sum(w * np.cos(k * np.arccos(x))) for k in range(K + 1)])
    # SciPy's double-precision nodes are good to a few 1e-13 near the singular weights
    assert np.max(np.abs(mu - ref)) < 2e-12 * abs(ref[0])
    # tighter: adaptive mpmath quadrature of the definition for the first moments
    a, b = mpmath.mpf(alpha), mpmath.mpf(beta)
    for k in range(5):
        v = mpmath.quad(lambda t: mpmath.chebyt(k, t) * (1 - t) ** a * (1 + t) ** b, [-1, 0, 1])
        assert abs(mu[k] - float(v)) < 4e-16 * abs(ref[0]), k


def test_moments_closed_forms(orc):
    K = 60
    mu = orc.moments(K, 0.0, 0.0)
    ref = np.array([0.0 if k == 1 else (1 + (-1) ** k) / (1 - k * k) for k in range(K + 1)])
    assert np.max(np.abs(mu - ref)) < 1e-15
    mu = orc.moments(K, -0.5, -0.5)
    assert abs(mu[0] - np.pi) < 1e-15 and np.max(np.abs(mu[1:])) < 1e-15


@pytest.mark.parametrize("alpha,beta", [(0.1, -0.3), (0.45, 0.45), (-0.5, 0.5)])
def test_cc_weights_exactness(orc, alpha, beta):
    """w^T T_k(x) = mu_k for every k <= Ng (Sec. 3.1), hence sum w = mu_0."""
    Ng = 96
    w = orc.cc_weights(Ng, alpha, beta)
    mu = orc.moments(Ng, alpha, beta)
    i = np.arange(Ng + 1)
    for k in range(Ng + 1):
        Tk = np.cos(np.pi * ((i * k) % (2 * Ng)) / Ng)
        assert abs(np.dot(w, Tk) - mu[k]) < 1e-14 * mu[0]


@pytest.mark.parametrize("alpha,beta", [(0.1, -0.3), (0.0, 0.0), (-0.5, -0.5), (0.45, 0.45)])
def test_norm_consts(orc, alpha, beta):
    N = 5000
    A = orc.norm_consts(N, alpha, beta)
    a, b = mpmath.mpf(alpha), mpmath.mpf(beta)
    for n in (0, 1, 2, 3, 10, 777, 5000):
        if n == 0:
            ref = 2 ** (a + b + 1) * mpmath.gamma(a + 1) * mpmath.gamma(b + 1) / mpmath.gamma(a + b + 2)
        else:
            ref = (2 ** (a + b + 1) * mpmath.gamma(n + a + 1) * mpmath.gamma(n + b + 1)
                   / ((2 * n + a + b + 1) * mpmath.gamma(n + a + b + 1) * mpmath.factorial(n)))
        assert abs(A[n] / float(ref) - 1) < 1e-14, n
    if alpha == 0.0 and beta == 0.0:
        assert np.max(np.abs(A - 2.0 / (2 * np.arange(N + 1) + 1))) < 1e-16
    # int P_n^2 w by Gauss-Jacobi quadrature (library values of P_n)
    x, w = sps.roots_jacobi(40, alpha, beta)
    for n in range(20):
        q = np.sum(w * sps.eval_jacobi(n, alpha, beta, x) ** 2)
        assert abs(q - A[n]) < 1e-13 * A[0]


@pytest.mark.parametrize("alpha,beta", [(0.125, 0.375), (0.1, -0.3), (0.5, 0.5), (-0.5, 0.2)])
def test_inverse_matches_exact_rational(orc, alpha, beta):
    N = 10
    c = inputs.decaying_coefficients(N, 1.0, seed=21)
    got = orc.inverse(c, alpha, beta)
    exact = np.array([float(v) for v in ex.inverse_exact(c, alpha, beta)])
    assert np.max(np.abs(got - exact)) <= 1e-14 * l1(c)


@pytest.mark.parametrize("alpha,beta", [(0.1, -0.3), (0.45, 0.45), (-0.5, 0.5)])
def test_plain_double_baselines(orc, alpha, beta):
    """The timed plain-double forward and inverse compute the same maps as the double-double
    oracle, within plain-double rounding: the three-term recurrence near x = +-1 loses about
    n^2 eps, so the bound grows with N (measured 2e-14 at N = 257, 2.5e-12 at N = 4096)."""
    for N, bound in ((1, 1e-15), (12, 1e-15), (257, 1e-13), (2048, 1e-11)):
        c = inputs.decaying_coefficients(N, 1.0, seed=inputs.BASE_SEED + 3 * N)
        assert np.max(np.abs(orc.forward_f64(c, alpha, beta) - orc.forward(c, alpha, beta))) <= bound * l1(c)
        assert np.max(np.abs(orc.inverse_f64(c, alpha, beta) - orc.inverse(c, alpha, beta))) <= bound * l1(c)
    assert orc.inverse_f64(np.array([2.5]), alpha, beta)[0] == 2.5


@pytest.mark.parametrize("alpha,beta", [(0.1, -0.3), (0.45, 0.45)])
def test_inverse_matches_dense_solve(orc, alpha, beta):
    """Route (i): solve P_N c_jac = T_N c_cheb with LAPACK (Eq. iCJT)."""
    N = 48
    c = inputs.decaying_coefficients(N, 1.0, seed=31)
    j = np.arange(N + 1)
    x = np.cos(np.pi * j / N)
    P = np.stack([sps.eval_jacobi(n, alpha, beta, x) for n in range(N + 1)], axis=1)  # rows = points
    T = np.cos(np.pi * np.outer(j, np.arange(N + 1)) / N)
    ref = np.linalg.solve(P, T @ c)
    got = orc.inverse(c, alpha, beta)
    assert np.max(np.abs(got - ref)) < 1e-11 * l1(c)


@pytest.mark.parametrize("alpha,beta", [(0.1, -0.3), (-0.45, 0.45)])
def test_round_trips_and_first_coefficient(orc, alpha, beta):
    N = 257
    c = inputs.decaying_coefficients(N, 1.0, seed=41)
    fwd = orc.forward(c, alpha, beta)
    assert np.max(np.abs(orc.inverse(fwd, alpha, beta) - c)) < 1e-14 * l1(c)
    inv = orc.inverse(c, alpha, beta)
    assert np.max(np.abs(orc.forward(inv, alpha, beta) - c)) < 1e-14 * l1(c)
    # Eq. cjintdefn at n = 0: c_jac_0 = sum_k c_cheb_k mu_k / mu_0
    mu = orc.moments(N, alpha, beta)
    assert abs(inv[0] - np.dot(c, mu) / mu[0]) < 1e-14 * l1(c)


# --------------------------------------------------------------------------
# a planted mistake in a copy of the oracle is caught by the pins
# --------------------------------------------------------------------------
def _build_mutant(tmp_path, old, new):
    src = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "cjt_oracle.c")
    text = open(src).read()
    assert text.count(old) == 1
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
                    "-D_DEFAULT_SOURCE", str(path), "-o", str(lib), "-lm"], check=True)
    return ctypes.CDLL(str(lib))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_planted_printed_mu1_sign_is_caught(tmp_path):
    """The mu_1 printed in Sec. 3.1 has the opposite sign; the quadrature pin rejects it."""
    lib = _build_mutant(tmp_path, "mu[1] = dd_div(dd_mul(dd_sub(dd_d(b), dd_d(a)), mu[0])",
                        "mu[1] = dd_div(dd_mul(dd_sub(dd_d(a), dd_d(b)), mu[0])")
    lib.orc_moments.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_double)]
    mu = np.empty(41)
    lib.orc_moments(40, 0.1, -0.3, mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    x, w = sps.roots_jacobi(40, 0.1, -0.3)
    ref = np.array([np.sum(w * np.cos(k * np.arccos(x))) for k in range(41)])
    assert np.max(np.abs(mu - ref)) > 1e-3


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_planted_dropped_B_term_is_caught(tmp_path):
    """Dropping B_n from the recurrence breaks agreement with Rodrigues' formula."""
    lib = _build_mutant(tmp_path, "dd pn = dd_sub(dd_mul(dd_add(dd_mul(t.A[n], x), t.B[n]), p), dd_mul(t.C[n], pm));\n        pm = p; p = pn;\n        out[n + 1]",
                        "dd pn = dd_sub(dd_mul(dd_mul(t.A[n], x), p), dd_mul(t.C[n], pm));\n        pm = p; p = pn;\n        out[n + 1]")
    lib.orc_jacobi_values.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    out = np.empty(9)
    lib.orc_jacobi_values(8, 0.1, -0.3, 1, 3, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    exact = float(_eval_poly(ex.jacobi_monomial(5, 0.1, -0.3), Fraction(1, 2)))
    assert abs(out[5] - exact) > 1e-6


_dp = ctypes.POINTER(ctypes.c_double)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_planted_missing_last_halving_is_caught(tmp_path):
    """T_N^{-1} halves c_N as well as c_0 (aliasing of T_N on N+1 Lobatto points); a copy
    that halves c_0 only fails the exact-rational pin of the forward map."""
    lib = _build_mutant(tmp_path, "if (k == 0 || k == N) s = dd_mul_d(s, 0.5);\n        c[k] = s.hi + s.lo;",
                        "if (k == 0) s = dd_mul_d(s, 0.5);\n        c[k] = s.hi + s.lo;")
    lib.orc_forward.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, _dp, _dp, ctypes.c_int]
    N, a, b = 5, 0.1, -0.3
    c = inputs.decaying_coefficients(N, 1.0, seed=inputs.BASE_SEED + N)
    got = np.empty(N + 1)
    lib.orc_forward(N, a, b, c.ctypes.data_as(_dp), got.ctypes.data_as(_dp), 1)
    exact = np.array([float(v) for v in ex.forward_exact(c, a, b)])
    assert np.max(np.abs(got - exact)) > 1e-3 * np.abs(exact).max()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_planted_cc_weight_end_factor_is_caught(tmp_path):
    """The Clenshaw--Curtis weights carry eps_i = 1/2 at both ends; a copy without it at
    i = Ng fails the exactness pin w^T T_k = mu_k."""
    lib = _build_mutant(tmp_path, "if (i == 0 || i == Ng) s = dd_mul_d(s, 0.5);\n        w[i] = s;",
                        "if (i == 0) s = dd_mul_d(s, 0.5);\n        w[i] = s;")
    lib.orc_cc_weights.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int]
    lib.orc_moments.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, _dp]
    Ng = 32
    w, mu = np.empty(Ng + 1), np.empty(Ng + 1)
    lib.orc_cc_weights(Ng, 0.1, -0.3, w.ctypes.data_as(_dp), 1)
    lib.orc_moments(Ng, 0.1, -0.3, mu.ctypes.data_as(_dp))
    i = np.arange(Ng + 1)
    err = max(abs(np.dot(w, np.cos(np.pi * ((i * k) % (2 * Ng)) / Ng)) - mu[k]) for k in range(Ng + 1))
    assert err > 1e-3 * mu[0]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_planted_norm_constant_slip_is_caught(tmp_path):
    """A_1 = mu_0 (a+1)(b+1)/(a+b+3) (Eq. "Anab"); a copy with a+b+2 in the denominator
    fails the Gamma-function pin from n = 1 on."""
    lib = _build_mutant(tmp_path, "dd_add(ab, dd_d(3.0)));", "dd_add(ab, dd_d(2.0)));")
    lib.orc_norm_consts.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, _dp]
    N, a, b = 50, 0.1, -0.3
    A = np.empty(N + 1)
    lib.orc_norm_consts(N, a, b, A.ctypes.data_as(_dp))
    am, bm = mpmath.mpf(a), mpmath.mpf(b)
    n = 10
    ref = (2 ** (am + bm + 1) * mpmath.gamma(n + am + 1) * mpmath.gamma(n + bm + 1)
           / ((2 * n + am + bm + 1) * mpmath.gamma(n + am + bm + 1) * mpmath.factorial(n)))
    assert abs(A[n] / float(ref) - 1) > 1e-3


def two_term_raise(a_coef, alpha, beta, which):
    """Coefficients in P^{(alpha+1,beta)} (which='alpha') or P^{(alpha,beta+1)} (which='beta') of
    sum_n a_n P_n^{(alpha,beta)}, in exact rationals, from the two-term connection relations
    P_n^{(a,b)} = [(n+a+b+1) P_n^{(a,b+1)} + (n+a) P_{n-1}^{(a,b+1)}] / (2n+a+b+1) and
    P_n^{(a,b)} = [(n+a+b+1) P_n^{(a+1,b)} - (n+b) P_{n-1}^{(a+1,b)}] / (2n+a+b+1)
    (DLMF 18.9.5 and 18.9.6)."""
    A, B = Fraction(alpha), Fraction(beta)
    a = [Fraction(float(x)) for x in a_coef]
    N = len(a) - 1
    other = A if which == "beta" else B
    sign = 1 if which == "beta" else -1
    out = []
    for n in range(N + 1):
        v = a[n] * ((n + A + B + 1) / (2 * n + A + B + 1) if n > 0 else 1)   # P_0 = 1 in every basis
        if n < N:
            v += sign * a[n + 1] * (n + 1 + other) / (2 * n + A + B + 3)
        out.append(v)
    return np.array([float(v) for v in out])


@pytest.mark.parametrize("alpha,beta,which", [(0.2, -0.5, "beta"), (-0.5, 0.3, "alpha"), (0.0, -0.5, "beta"),
                                              (-0.5, -0.5, "alpha")])
def test_jacobi_to_jacobi_two_term_connection(orc, alpha, beta, which):
    """Jacobi-to-Jacobi conversion (forward then inverse, Sec. 5) against the two-term
    connection of a unit parameter raise, an independent closed form."""
    N = 200
    c = inputs.decaying_coefficients(N, 1.0, seed=31)
    g, d = (alpha + 1, beta) if which == "alpha" else (alpha, beta + 1)
    got = orc.jacobi_to_jacobi(c, alpha, beta, g, d)
    want = two_term_raise(c, alpha, beta, which)
    assert np.max(np.abs(got - want)) <= 1e-14 * l1(c)


def test_jacobi_to_jacobi_identity(orc):
    c = inputs.decaying_coefficients(300, 1.0, seed=32)
    assert np.max(np.abs(orc.jacobi_to_jacobi(c, 0.3, -0.1, 0.3, -0.1) - c)) <= 1e-14 * l1(c)


# Parameters outside [-1/2, 1/2]^2, reached from the square by one integer shift (Sec. 1.2):
# the oracle evaluates the definitions directly.  Its modified-moment recurrence loses
# accuracy for alpha or beta above about 2, so the pinned domain is (-1, 3/2]^2.
SHIFTED = [(1.5, 0.25), (-0.8, 0.4), (1.2, -0.9), (0.3, 1.5), (1.4, 1.1), (-0.95, -0.7)]


@pytest.mark.parametrize("alpha,beta", SHIFTED)
@pytest.mark.parametrize("N", [2, 7, 12])
def test_forward_exact_rational_shifted_parameters(orc, alpha, beta, N):
    c = inputs.decaying_coefficients(N, 1.0, seed=inputs.BASE_SEED + 5 * N)
    exact = np.array([float(v) for v in ex.forward_exact(c, alpha, beta)])
    assert np.max(np.abs(orc.forward(c, alpha, beta) - exact)) <= 1e-15 * l1(c)


@pytest.mark.parametrize("alpha,beta", SHIFTED)
def test_inverse_exact_rational_shifted_parameters(orc, alpha, beta):
    N = 10
    c = inputs.decaying_coefficients(N, 1.0, seed=23)
    exact = np.array([float(v) for v in ex.inverse_exact(c, alpha, beta)])
    assert np.max(np.abs(orc.inverse(c, alpha, beta) - exact)) <= 1e-14 * l1(c)


def moment_closed_form(k, alpha, beta):
    """mu_k = int T_k (1-x)^a (1+x)^b dx as a terminating sum: with T_k(x) the hypergeometric
    polynomial 2F1(-k, k; 1/2; (1-x)/2) and Beta integrals term by term,
    mu_k = mu_0 3F2(-k, k, a+1; 1/2, a+b+2; 1), mu_0 = 2^(a+b+1) G(a+1) G(b+1) / G(a+b+2)
    (60 digits)."""
    mpmath.mp.dps = 60
    a, b = mpmath.mpf(alpha), mpmath.mpf(beta)
    mu0 = 2 ** (a + b + 1) * mpmath.gamma(a + 1) * mpmath.gamma(b + 1) / mpmath.gamma(a + b + 2)
    s, t = mpmath.mpf(0), mpmath.mpf(1)
    for j in range(k + 1):
        s += t
        t *= (j - k) * (k + j) * (a + 1 + j) / ((mpmath.mpf(0.5) + j) * (j + 1) * (a + b + 2 + j))
    return float(mu0 * s)


@pytest.mark.parametrize("alpha,beta", SHIFTED + [(0.1, -0.3), (-0.5, -0.5)])
def test_moments_closed_form(orc, alpha, beta):
    K = 40
    mu = orc.moments(K, alpha, beta)
    for k in (0, 1, 2, 5, 12, 40):
        ref = moment_closed_form(k, alpha, beta)
        assert abs(mu[k] - ref) <= 1e-15 * max(1.0, abs(ref))


@pytest.mark.parametrize("alpha,beta", SHIFTED)
def test_round_trip_shifted_parameters(orc, alpha, beta):
    N = 400
    c = inputs.decaying_coefficients(N, 1.0, seed=24)
    back = orc.inverse(orc.forward(c, alpha, beta), alpha, beta)
    assert np.max(np.abs(back - c)) <= 1e-13 * l1(c)
