"""Pins of the asymptotic expansions the plans use, evaluated on the host through the C ABI
(cjt_asy_coefficient, cjt_asy_eval: the same functions the plan kernels call, no GPU).

* C_{n,m} against its definition: Hahn's (Eq. "Cnmab", a beta function) and the
  ultraspherical C^lambda_{n,m} (App. B.1, gamma functions and Pochhammer symbols),
  both at 40 digits.
* The M-term expansion against P_n^{(alpha,beta)}(cos theta) at 30 digits: the error stays
  below the remainder bound the partition uses (Sec. 2.2; App. B.1).
* The collapses of App. B.2-B.3 (alpha or beta = 1/2: one cosine per term) and the
  ultraspherical formula of App. B.1, each written out term by term in mpmath, to
  rounding relative to the sum of the terms' envelopes.
"""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from paper_1602_02618_gb300 import cjt  # noqa: E402

HAHN, ULTRA, AUTO = cjt.CJT_EXPANSION_HAHN, cjt.CJT_EXPANSION_ULTRASPHERICAL, cjt.CJT_EXPANSION_AUTO


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1602_02618_gb300 import build
    build.build()
    return cjt.load()


def hahn_C_exact(n, m, a, b):
    a, b = mp.mpf(a), mp.mpf(b)
    return mp.power(2, 2 * n - m + a + b + 1) * mp.beta(n + a + 1, n + b + 1) / (mp.pi * mp.rf(2 * n + a + b + 2, m))


def ultra_C_exact(n, m, lam):
    lam = mp.mpf(lam)
    c0 = mp.power(2, lam) * mp.gamma(n + lam + mp.mpf(1) / 2) / (mp.sqrt(mp.pi) * mp.gamma(n + lam + 1))
    return c0 * mp.rf(lam, m) * mp.rf(1 - lam, m) / (mp.power(2, m) * mp.factorial(m) * mp.rf(n + lam + 1, m))


@pytest.mark.parametrize("lam", [0.05, 0.3, 0.5, 0.7, 0.95])
def test_ultraspherical_coefficients(lam):
    mp.mp.dps = 40
    a = lam - 0.5
    for n in [0, 1, 2, 7, 8, 9, 10, 50, 1000, 1 << 20]:
        for m in [0, 1, 5, 13, 20]:
            got = cjt.asy_coefficient(a, a, n, m, ULTRA)
            ref = ultra_C_exact(n, m, lam)
            assert abs(got - ref) <= 2e-14 * abs(ref), (n, m, got, float(ref))


@pytest.mark.parametrize("a,b", [(0.1, -0.3), (0.45, 0.45), (-0.45, 0.2), (0.5, 0.1), (-0.5, -0.2), (0.0, 0.0)])
def test_hahn_coefficients(a, b):
    mp.mp.dps = 40
    for n in [0, 1, 2, 7, 8, 9, 10, 50, 1000, 1 << 20]:
        for m in [0, 1, 5, 13, 20]:
            got = cjt.asy_coefficient(a, b, n, m, HAHN)
            ref = hahn_C_exact(n, m, a, b)
            assert abs(got - ref) <= 2e-14 * abs(ref), (n, m, got, float(ref))


CASES = [(0.1, -0.3, AUTO), (0.45, 0.45, AUTO), (0.45, 0.45, HAHN), (0.0, 0.0, AUTO), (0.0, 0.0, HAHN),
         (-0.45, -0.45, AUTO), (0.25, 0.25, ULTRA), (0.5, 0.1, AUTO), (-0.5, 0.3, AUTO), (0.2, 0.5, AUTO),
         (0.3, -0.5, AUTO)]


@pytest.mark.parametrize("a,b,exp", CASES)
def test_expansion_within_remainder_bound(orc, a, b, exp):
    """|P_n(cos theta) - sum_{m<M} ...| <= 2 C_{n,M} g_M(theta) (plus rounding) on a grid of
    (n, theta) that reaches both ends of the interval and the low degrees; P_n from the
    oracle's double-double recurrence."""
    Ng = 256
    rows = [1, 2, 5, 17, 64, 128, 191, 250, 254, 255]
    P = {i: orc.jacobi_values(5000, a, b, i, Ng) for i in rows}
    worst = 0.0
    for M in [3, 7, 13]:
        for n in [2, 3, 10, 40, 200, 1000, 5000]:
            for i in rows:
                val, bound = cjt.asy_eval(a, b, M, n, i, Ng, exp)
                ref = P[i][n]
                err = abs(val - ref)
                assert err <= bound + 1e-14 * max(1.0, abs(ref)), (M, n, i, val, ref, bound)
                if bound > 1e-10:
                    worst = max(worst, err / bound)
    assert worst > 0.05   # the bound is not vacuous: errors reach a good fraction of it


def _theta(i, Ng):
    return mp.pi * mp.mpf(i) / Ng


@pytest.mark.parametrize("b", [0.1, -0.35, 0.45])
def test_alpha_half_collapse(b):
    """alpha = 1/2 (App. B.2): each term of Hahn's formula is the single cosine
    h_m(beta) cos(theta_{n,m,0}) / (sin(theta/2) cos^{m+beta+1/2}(theta/2))."""
    mp.mp.dps = 30
    a, Ng, M = 0.5, 512, 7
    for n in [5, 60, 700]:
        for i in [40, 256, 470]:
            th = _theta(i, Ng)
            s = scale = mp.mpf(0)
            for m in range(M):
                h = mp.rf(mp.mpf(0.5) + b, m) * mp.rf(mp.mpf(0.5) - b, m) / mp.factorial(m)
                ph = (n + (mp.mpf(a) + b + m + 1) / 2) * th - (a + mp.mpf(0.5)) * mp.pi / 2
                mag = hahn_C_exact(n, m, a, b) * h / (mp.sin(th / 2) * mp.cos(th / 2) ** (m + b + 0.5))
                s += mag * mp.cos(ph)
                scale += abs(mag)
            val, _ = cjt.asy_eval(a, b, M, n, i, Ng, HAHN)
            assert abs(val - s) <= 2e-14 * scale, (n, i, val, float(s))


@pytest.mark.parametrize("a", [0.1, -0.35, 0.45])
def test_beta_half_collapse(a):
    """beta = 1/2 (App. B.3): each term is h_m(alpha) cos(theta_{n,m,m}) /
    (sin^{m+alpha+1/2}(theta/2) cos(theta/2))."""
    mp.mp.dps = 30
    b, Ng, M = 0.5, 512, 7
    for n in [5, 60, 700]:
        for i in [40, 256, 470]:
            th = _theta(i, Ng)
            s = scale = mp.mpf(0)
            for m in range(M):
                h = mp.rf(mp.mpf(0.5) + a, m) * mp.rf(mp.mpf(0.5) - a, m) / mp.factorial(m)
                ph = (n + (mp.mpf(a) + b + m + 1) / 2) * th - (a + m + mp.mpf(0.5)) * mp.pi / 2
                mag = hahn_C_exact(n, m, a, b) * h / (mp.sin(th / 2) ** (m + a + 0.5) * mp.cos(th / 2))
                s += mag * mp.cos(ph)
                scale += abs(mag)
            val, _ = cjt.asy_eval(a, b, M, n, i, Ng, HAHN)
            assert abs(val - s) <= 2e-14 * scale, (n, i, val, float(s))


@pytest.mark.parametrize("lam", [0.2, 0.5, 0.85])
def test_ultraspherical_formula(lam):
    """App. B.1 written out: sum_m C^lambda_{n,m} cos(n theta - (m+lambda)(pi/2 - theta)) /
    sin^{m+lambda}(theta), and its bound 2 C^lambda_{n,M} / sin^{M+lambda}(theta)."""
    mp.mp.dps = 30
    a, Ng, M = lam - 0.5, 512, 9
    lam = mp.mpf(lam)
    for n in [3, 90, 1500]:
        for i in [7, 200, 256, 505]:
            th = _theta(i, Ng)
            s = scale = mp.mpf(0)
            for m in range(M):
                mag = ultra_C_exact(n, m, lam) / mp.sin(th) ** (m + lam)
                s += mag * mp.cos(n * th - (m + lam) * (mp.pi / 2 - th))
                scale += abs(mag)
            bound = 2 * ultra_C_exact(n, M, lam) / mp.sin(th) ** (M + lam)
            val, bd = cjt.asy_eval(a, a, M, n, i, Ng, AUTO)
            assert abs(val - s) <= 2e-14 * scale, (n, i, val, float(s))
            assert abs(bd - bound) <= 5e-13 * bound


def test_auto_picks_ultraspherical_only_on_the_diagonal():
    """AUTO evaluates the ultraspherical formula when alpha = beta in (-1/2, 1/2) and Hahn's
    otherwise; the two formulas differ term by term but approximate the same polynomial."""
    n, i, Ng, M = 300, 100, 512, 7
    for a in (0.0, 0.3, -0.2):
        assert cjt.asy_eval(a, a, M, n, i, Ng, AUTO) == cjt.asy_eval(a, a, M, n, i, Ng, ULTRA)
        assert cjt.asy_coefficient(a, a, n, 1, AUTO) != cjt.asy_coefficient(a, a, n, 1, HAHN)
        vu, bu = cjt.asy_eval(a, a, M, n, i, Ng, ULTRA)
        vh, bh = cjt.asy_eval(a, a, M, n, i, Ng, HAHN)
        assert abs(vu - vh) <= bu + bh + 1e-14
    assert cjt.asy_eval(0.1, -0.3, M, n, i, Ng, AUTO) == cjt.asy_eval(0.1, -0.3, M, n, i, Ng, HAHN)
    # at the corners both series end after one term; the corner uses Hahn's formula
    assert cjt.asy_eval(0.5, 0.5, 1, n, i, Ng, AUTO) == cjt.asy_eval(0.5, 0.5, 1, n, i, Ng, HAHN)


def test_host_expansion_errors():
    with pytest.raises(cjt.CJTError) as e:
        cjt.asy_eval(0.1, 0.2, 7, 10, 5, 64, ULTRA)
    assert e.value.code == cjt.CJT_EINVAL
    with pytest.raises(cjt.CJTError) as e:
        cjt.asy_eval(0.6, 0.2, 7, 10, 5, 64, AUTO)
    assert e.value.code == cjt.CJT_EDOMAIN
    for bad in [dict(i=0), dict(i=64), dict(M=0), dict(M=21), dict(n=-1)]:
        kw = dict(M=7, n=10, i=5, Ng=64)
        kw.update(bad)
        with pytest.raises(cjt.CJTError) as e:
            cjt.asy_eval(0.1, 0.2, kw["M"], kw["n"], kw["i"], kw["Ng"], AUTO)
        assert e.value.code == cjt.CJT_EINVAL
    with pytest.raises(cjt.CJTError) as e:
        cjt.asy_coefficient(0.1, 0.2, 5, 21, AUTO)
    assert e.value.code == cjt.CJT_EINVAL
    assert np.isfinite(cjt.asy_coefficient(0.5, -0.5, 5, 0, AUTO))
