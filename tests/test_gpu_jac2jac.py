"""Jacobi-to-Jacobi conversion on the GPU (Sec. 5: the forward transform of one parameter
pair composed with the inverse transform of another), through the C ABI.

Checked against the oracle's composition, and at full size against the two-term
connection of a unit parameter raise (DLMF 18.9.5-6), which holds at any N.
"""
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
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def l1(c):
    return float(np.abs(c).sum())


def raise_one(a, alpha, beta, which):
    """Two-term connection (DLMF 18.9.5 for beta, 18.9.6 for alpha), in float64."""
    N = a.size - 1
    n = np.arange(N + 1, dtype=np.float64)
    f0 = np.ones(N + 1)
    f0[1:] = (n[1:] + alpha + beta + 1) / (2 * n[1:] + alpha + beta + 1)   # P_0 = 1 in every basis
    out = a * f0
    other = alpha if which == "beta" else beta
    sign = 1.0 if which == "beta" else -1.0
    out[:-1] += sign * a[1:] * (n[:-1] + 1 + other) / (2 * n[:-1] + alpha + beta + 3)
    return out


def convert(cjt, pf, pt, c):
    y = cjt.cjt_jacobi_to_jacobi(pf, pt, dev(c))
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("src,dst", [((0.1, -0.3), (0.4, 0.2)), ((-0.5, -0.5), (0.0, 0.0)),
                                     ((0.45, 0.45), (-0.45, 0.1)), ((0.2, -0.5), (0.2, 0.5))])
@pytest.mark.parametrize("N", [64, 1000, 4096])
def test_jac2jac_matches_oracle(cjt, orc, N, src, dst):
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 17 * N)
    pf = cjt.Plan(N, *src, directions=cjt.CJT_FWD)
    pt = cjt.Plan(N, *dst, directions=cjt.CJT_INV)
    got = convert(cjt, pf, pt, c)
    assert np.max(np.abs(got - orc.jacobi_to_jacobi(c, *src, *dst))) <= TOL * l1(c)


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("alpha,beta,which", [(0.2, -0.5, "beta"), (-0.5, 0.3, "alpha"), (-0.5, -0.5, "alpha")])
def test_jac2jac_two_term_connection_full_size(cjt, alpha, beta, which, precision):
    N = 1 << 16
    prec = cjt.CJT_FP64 if precision == "fp64" else cjt.CJT_DFLOAT
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 99)
    g, d = (alpha + 1, beta) if which == "alpha" else (alpha, beta + 1)
    pf = cjt.Plan(N, alpha, beta, precision=prec, M=13, rec_store=1)
    pt = cjt.Plan(N, g, d, precision=prec, M=13, rec_store=1)
    got = convert(cjt, pf, pt, c)
    assert np.max(np.abs(got - raise_one(c, alpha, beta, which))) <= TOL * l1(c)
    # in place
    x = dev(c)
    cjt.cjt_jacobi_to_jacobi(pf, pt, x, x)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), got)


def test_jac2jac_errors(cjt):
    a = cjt.Plan(64, 0.1, 0.2)
    b = cjt.Plan(65, 0.1, 0.2)
    with pytest.raises(cjt.CJTError) as e:
        cjt.cjt_jacobi_to_jacobi(a, b, dev(np.zeros(65)))
    assert e.value.code == cjt.CJT_EINVAL
    f_only = cjt.Plan(64, 0.3, 0.2, directions=cjt.CJT_FWD)
    with pytest.raises(cjt.CJTError) as e:
        cjt.cjt_jacobi_to_jacobi(a, f_only, dev(np.zeros(65)))
    assert e.value.code == cjt.CJT_EDIRECTION
