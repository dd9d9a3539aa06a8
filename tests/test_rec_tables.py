"""The plan's recurrence tables on the CPU (host entry point cjt_rec_coefficients, the
same function as the plan kernel that fills them), pinned against their definitions:

* A_n, B_n, C_n: the three-term recurrence (Sec. 1.2) reproduces mpmath's Jacobi
  polynomials at interior points, including the n = 0 step from P_0 to P_1;
* r^f_n(+-1): the ratio P_{n+1}(x0)/P_n(x0) of the endpoint values (Eq. "Pnendpts");
* r^b_n(+-1): the ratio v_{n+1}/v_n of the homogeneous adjoint recurrence
  v_n = (A_n x0 + B_n) v_{n+1} - C_{n+1} v_{n+2}, v_0 = 0, v_1 = 1 (Sec. 4.2), run in
  80-digit arithmetic from its definition, so the Lemma's closed form is checked and not
  restated;
* C_{n+1} r^b_{n+1}(+-1) = r^f_n(+-1), the identity the recurrence kernels use to join
  degree segments without cancellation.
"""
import mpmath
import numpy as np
import pytest

PARAMS = [(0.1, -0.3), (0.45, 0.45), (-0.5, -0.5), (0.5, -0.5), (-0.5, 0.5), (0.0, 0.0), (0.25, -0.45)]
NMAX = 60


@pytest.fixture(scope="module")
def cjt():
    from paper_1602_02618_gb300 import build
    build.build()
    from paper_1602_02618_gb300 import cjt as mod
    return mod


def tables(cjt, a, b):
    return [cjt.rec_coefficients(a, b, n) for n in range(NMAX + 2)]


def exact_abc(n, a, b):
    """A_n, B_n, C_n at 80 digits from the standard three-term recurrence of the Jacobi
    polynomials (DLMF 18.9.1-18.9.2), with the n = 0 step taken from P_1."""
    a, b, n = mpmath.mpf(a), mpmath.mpf(b), mpmath.mpf(n)
    if n == 0:
        return (a + b + 2) / 2, (a - b) / 2, mpmath.mpf(0)
    t0 = 2 * n + a + b
    den = 2 * (n + 1) * (n + a + b + 1) * t0
    A = (t0 + 1) * (t0 + 2) * t0 / den
    B = (a * a - b * b) * (t0 + 1) / den
    C = 2 * (n + a) * (n + b) * (t0 + 2) / den
    return A, B, C


@pytest.mark.parametrize("a,b", PARAMS)
def test_three_term_recurrence_reproduces_jacobi(cjt, a, b):
    mpmath.mp.dps = 40
    T = tables(cjt, a, b)
    for x in (0.3, -0.7, 0.95):
        P = [mpmath.jacobi(n, a, b, x) for n in range(NMAX + 2)]
        for n in range(NMAX + 1):
            prev = P[n - 1] if n > 0 else 0
            pred = (T[n]["A"] * x + T[n]["B"]) * P[n] - T[n]["C"] * prev
            scale = abs(T[n]["A"] * x * P[n]) + abs(T[n]["B"] * P[n]) + abs(T[n]["C"] * prev) + 1e-300
            assert abs(float(pred - P[n + 1])) <= 4e-16 * float(scale), (x, n)


@pytest.mark.parametrize("a,b", PARAMS)
def test_forward_ratios_are_endpoint_ratios(cjt, a, b):
    mpmath.mp.dps = 40
    T = tables(cjt, a, b)
    for n in range(NMAX + 1):
        for key, x0 in (("rf_p", 1), ("rf_m", -1)):
            want = mpmath.jacobi(n + 1, a, b, x0) / mpmath.jacobi(n, a, b, x0)
            assert abs(T[n][key] / float(want) - 1) <= 4e-16, (key, n)


@pytest.mark.parametrize("a,b", PARAMS)
def test_backward_ratios_from_the_adjoint_recurrence(cjt, a, b):
    mpmath.mp.dps = 80
    T = tables(cjt, a, b)
    abc = [exact_abc(n, a, b) for n in range(NMAX + 3)]
    for key, x0 in (("rb_p", 1), ("rb_m", -1)):
        # v_n = (A_n x0 + B_n) v_{n+1} - C_{n+1} v_{n+2}  =>  v_{n+2} from v_n, v_{n+1}
        v = [mpmath.mpf(0), mpmath.mpf(1)]
        for n in range(NMAX + 1):
            A, B, _ = abc[n]
            C1 = abc[n + 1][2]
            v.append(((A * x0 + B) * v[n + 1] - v[n]) / C1)
        for n in range(1, NMAX + 1):
            want = v[n + 1] / v[n]
            assert abs(T[n][key] / float(want) - 1) <= 1e-15, (key, n)
        assert T[0][key] == 0.0


@pytest.mark.parametrize("a,b", PARAMS)
def test_segment_join_identity_and_derived_entries(cjt, a, b):
    T = tables(cjt, a, b)
    for n in range(NMAX + 1):
        for s in ("p", "m"):
            # C_{n+1} r^b_{n+1}(x0) = r^f_n(x0), each side a dozen roundings from exact
            assert T[n + 1]["Cr_" + s] == pytest.approx(T[n]["rf_" + s], rel=2e-15, abs=0)
            assert T[n + 1]["Cr_" + s] == pytest.approx(T[n + 1]["C"] * T[n + 1]["rb_" + s], rel=2e-16, abs=0)
            assert T[n + 1]["Ce_" + s] == pytest.approx(T[n + 1]["C"] / T[n]["rf_" + s], rel=1e-15, abs=0)
    assert T[0]["C"] == 0.0 and T[0]["Ce_p"] == 0.0 and T[0]["Cr_m"] == 0.0


def test_rec_coefficients_errors(cjt):
    with pytest.raises(cjt.CJTError) as e:
        cjt.rec_coefficients(0.6, 0.0, 3)
    assert e.value.code == cjt.CJT_EDOMAIN
    with pytest.raises(cjt.CJTError) as e:
        cjt.rec_coefficients(0.1, 0.0, -1)
    assert e.value.code == cjt.CJT_EINVAL
    assert np.isfinite(list(cjt.rec_coefficients(0.1, -0.3, 1 << 30).values())).all()
