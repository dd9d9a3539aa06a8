"""Transforms of length q 2^b, q = 3 or 5 (Lobatto grids G = q 2^a, the default when q 2^a is
the least of 2^a', 3 2^a'', 5 2^a''' at or above N): one radix-q step
X[k1 + q k2] = FFT_{L/q}(omega_L^{n2 k1} sum_{n1} x[n1 L/q + n2] omega_q^{n1 k1}) followed by
power-of-two FFTs of the q rows.  The full transforms match the oracle in all three
precision forms, for rows done in one pass (L/q <= 4096) and by the four-step split
(L/q > 4096), and agree with the power-of-two grid."""
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


def least_grid(N):
    """(G, q): the least G >= N of the forms 2^a (q = 1), 3 2^a and 5 2^a."""
    best = None
    for q in (1, 3, 5):
        G = q
        while G < N:
            G <<= 1
        if best is None or G < best[0]:
            best = (G, q)
    return best


# q = 3: 3, 6, 12, 96, 700, 1536, 6000 (inverse rows 8192: four-step);
# q = 5: 5, 10, 20, 80, 300, 1200, 2500, 9000 (inverse rows 8192: four-step)
NS = [3, 6, 12, 96, 700, 1536, 6000, 5, 10, 20, 80, 300, 1200, 2500, 9000]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("N", NS)
def test_odd_radix_grid_matches_oracle(cjt, orc, N, precision):
    a, b = 0.21, -0.37
    c = inputs.decaying_coefficients(N, 1.0, 777 + N)
    plan = cjt.Plan(N, a, b, precision=precision, rec_store=1 if precision == 2 else 0)
    G, q = least_grid(N)
    assert q in (3, 5) and plan.info()["grid_fwd"] == G and N <= G
    f, i = run(cjt, plan, c, True), run(cjt, plan, c, False)
    ef = np.max(np.abs(f - orc.forward(c, a, b)))
    ei = np.max(np.abs(i - orc.inverse(c, a, b)))
    l1 = np.abs(c).sum()
    if precision == 1:
        assert ef <= cjt.error_bound(plan, cjt.CJT_FWD) * l1 and ei <= cjt.error_bound(plan, cjt.CJT_INV) * l1
    else:
        assert ef <= TOL * l1 and ei <= TOL * l1, (ef, ei)


@pytest.mark.parametrize("N,G", [(23000, 24576), (20000, 20480)])
def test_odd_radix_agrees_with_power_of_two_grid(cjt, N, G):
    """Grids 24576 = 3 2^13 and 20480 = 5 2^12 (rows of 8192 or 16384 points by the four-step
    split) against grid 32768, forward and inverse."""
    a, b = -0.12, 0.33
    c = inputs.decaying_coefficients(N, 1.0, 31)
    pq = cjt.Plan(N, a, b, M=10)
    p2 = cjt.Plan(N, a, b, M=10, grid=1)
    assert pq.info()["grid_fwd"] == G and p2.info()["grid_fwd"] == 32768
    l1 = np.abs(c).sum()
    assert np.max(np.abs(run(cjt, pq, c, True) - run(cjt, p2, c, True))) <= TOL * l1
    assert np.max(np.abs(run(cjt, pq, c, False) - run(cjt, p2, c, False))) <= TOL * l1
