"""Transforms of length 3 2^b (Lobatto grids G = 3 2^a, the default for N in (2^a, 3 2^(a-1)]):
one radix-3 step X[k1 + 3 k2] = FFT_{L/3}(omega_L^{n2 k1} sum_{n1} x[n1 L/3 + n2] omega_3^{n1 k1})
followed by power-of-two FFTs of the three rows.  The full transforms match the oracle in
all three precision forms, for rows done in one pass (L/3 <= 4096) and by the four-step
split (L/3 > 4096), and agree with the power-of-two grid."""
import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def cjt():
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt as mod
    assert torch.cuda.is_available()
    return mod


def run(cjt, plan, c, fwd):
    x = torch.from_numpy(c).cuda()
    y = cjt.cjt_forward(plan, x) if fwd else cjt.cjt_inverse(plan, x)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("N", [3, 6, 12, 96, 700, 1536, 2500, 5000, 9000])
def test_radix3_grid_matches_oracle(cjt, orc, N, precision):
    a, b = 0.21, -0.37
    c = inputs.decaying_coefficients(N, 1.0, 777 + N)
    plan = cjt.Plan(N, a, b, precision=precision, rec_store=1 if precision == 2 else 0)
    G = plan.info()["grid_fwd"]
    assert G % 3 == 0 and (G // 3) & (G // 3 - 1) == 0 and N <= G < 2 * N + 3
    f, i = run(cjt, plan, c, True), run(cjt, plan, c, False)
    ef = np.max(np.abs(f - orc.forward(c, a, b)))
    ei = np.max(np.abs(i - orc.inverse(c, a, b)))
    l1 = np.abs(c).sum()
    if precision == 1:
        assert ef <= cjt.error_bound(plan, cjt.CJT_FWD) * l1 and ei <= cjt.error_bound(plan, cjt.CJT_INV) * l1
    else:
        assert ef <= TOL * l1 and ei <= TOL * l1, (ef, ei)


def test_radix3_agrees_with_power_of_two_grid(cjt):
    """N = 20000: grid 24576 (rows of 8192 and 16384 points by the four-step split) against
    grid 32768, forward and inverse."""
    N, a, b = 20000, -0.12, 0.33
    c = inputs.decaying_coefficients(N, 1.0, 31)
    p3 = cjt.Plan(N, a, b, M=10)
    p2 = cjt.Plan(N, a, b, M=10, grid=1)
    assert p3.info()["grid_fwd"] == 24576 and p2.info()["grid_fwd"] == 32768
    l1 = np.abs(c).sum()
    assert np.max(np.abs(run(cjt, p3, c, True) - run(cjt, p2, c, True))) <= TOL * l1
    assert np.max(np.abs(run(cjt, p3, c, False) - run(cjt, p2, c, False))) <= TOL * l1
