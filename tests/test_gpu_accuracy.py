"""Accuracy experiments after the paper's Figs. 2 and 3 (Sec. 4.2 and the numerical
discussion), on the GPU through the C ABI.  Run with `-s` to print the tables.

* Fig. 2: P_10000^{(0,0)}(cos theta) at the 10 001 equally spaced angles theta_i = pi i/N
  (the Lobatto grid), read off the forward transform of the unit coefficient vector e_N
  (its Chebyshev coefficients summed in double-double by the oracle), against the
  oracle's double-double values.
* Fig. 3: Chebyshev -> Jacobi -> Chebyshev round trips (inverse, then forward) for
  coefficients of an irregular function (U(0,1)) and of a continuous function
  (U(-1,1)/(n+1)^2), over N, mean and max over 10 random (alpha, beta) ~ U(-1/2, 1/2).
  Each round trip is held to the inverse's error bound of Sec. 3.3 with constant one,
  N^(1 + max(alpha, beta, 0)) log2(N) eps ||c||_1 (the paper calls it pessimistic; the
  measured errors are far below it and are printed).
"""
import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cjt():
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt as mod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mod


def run(cjt, plan, c, direction):
    fn = cjt.cjt_forward if direction == cjt.CJT_FWD else cjt.cjt_inverse
    y = fn(plan, torch.from_numpy(np.ascontiguousarray(c)).cuda())
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_fig2_legendre_10000_values(cjt, orc, precision):
    N = 10000
    prec = cjt.CJT_FP64 if precision == "fp64" else cjt.CJT_DFLOAT
    e = np.zeros(N + 1)
    e[N] = 1.0
    plan = cjt.Plan(N, 0.0, 0.0, precision=prec, directions=cjt.CJT_FWD)
    cheb = run(cjt, plan, e, cjt.CJT_FWD)
    j = np.arange(N + 1)
    got = orc.cheb_series(cheb, j, N)
    ref = orc.jacobi_series(e, 0.0, 0.0, j, N)
    err = np.abs(got - ref)
    # relative to the envelope of P_N (|P_N(cos theta)| <~ sqrt(2 / (pi N sin theta)), and 1 at the ends)
    theta = np.pi * j / N
    env = np.minimum(1.0, np.sqrt(2.0 / (np.pi * N * np.maximum(np.sin(theta), 1e-300))))
    rel = err / env
    print("\nFig. 2 (%s): P_10000^(0,0) at 10001 angles: max abs error %.2e, max error / envelope %.2e, "
          "median %.2e" % (precision, err.max(), rel.max(), np.median(rel)))
    assert err.max() <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_fig3_round_trips(cjt, precision):
    prec = cjt.CJT_FP64 if precision == "fp64" else cjt.CJT_DFLOAT
    rows = []
    for N in (256, 1024, 4096, 16384, 65536):
        for kind, gen in (("U(0,1)", inputs.irregular_coefficients), ("U(-1,1)/(n+1)^2", inputs.continuous_coefficients)):
            errs = []
            for t in range(10):
                a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 9000 + t, -0.5, 0.5)
                c = gen(N, inputs.BASE_SEED + 9100 + 37 * t + N)
                plan = cjt.Plan(N, a, b, precision=prec, M=13)
                back = run(cjt, plan, run(cjt, plan, c, cjt.CJT_INV), cjt.CJT_FWD)
                errs.append(np.abs(back - c).max())
                plan.close()
                bound = N ** (1.0 + max(a, b, 0.0)) * np.log2(N) * 2.0 ** -52 * np.abs(c).sum()
                assert errs[-1] <= bound
            rows.append((N, kind, float(np.mean(errs)), float(np.max(errs)), float(np.abs(c).sum())))
    print("\nFig. 3 (%s): max |c - forward(inverse(c))|, mean and max over 10 (alpha, beta)" % precision)
    for N, kind, mean, mx, l1 in rows:
        print("  N=%6d  %-16s mean %.2e  max %.2e  (||c||_1 of the last draw %.3g)" % (N, kind, mean, mx, l1))
