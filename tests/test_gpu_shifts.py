"""Jacobi parameters in (1/2, 3/2] (Sec. 1.2): one integer step per parameter down into the
square, applied as an O(N) coefficient conversion before the forward transform (a
bidiagonal solve on the input) and after the inverse transform (a bidiagonal product on
the output).  GPU (through the C ABI) against the oracle, which evaluates the definitions
at the caller's parameters directly.
"""
import hashlib
import os

import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SHIFTED = [(1.5, 0.25), (0.75, -0.4), (1.2, -0.5), (0.3, 1.5), (1.4, 1.1), (-0.5, 0.9)]


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


def run(cjt, plan, c, direction):
    fn = cjt.cjt_forward if direction == cjt.CJT_FWD else cjt.cjt_inverse
    y = fn(plan, dev(c))
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("alpha,beta", SHIFTED)
@pytest.mark.parametrize("N", [1, 2, 64, 1024, 4096])
def test_shifted_parameters_match_oracle(cjt, orc, N, alpha, beta, precision):
    prec = cjt.CJT_FP64 if precision == "fp64" else cjt.CJT_DFLOAT
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 19 * N)
    plan = cjt.Plan(N, alpha, beta, precision=prec)
    info = plan.info()
    assert (info["alpha"], info["beta"]) == (alpha, beta)
    assert -0.5 <= alpha - info["shift_alpha"] <= 0.5 and -0.5 <= beta - info["shift_beta"] <= 0.5
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_FWD) - orc.forward(c, alpha, beta))) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - orc.inverse(c, alpha, beta))) <= TOL * l1(c)


@pytest.mark.parametrize("t", [0, 1])
def test_shifted_parameters_full_size(cjt, orc, t):
    """N = 2^16 with stored recurrence values.  Forward: sampled value identities
    (double-double oracle), each within TOL times the sum of the absolute terms
    sum_n |c_n P_n(x_j)|, which grows like N^(beta+1/2) near x = -1 for beta > 1/2.
    Inverse: every coefficient against the stored double-double oracle output.  And the
    forward-then-inverse round trip."""
    N, alpha, beta, c = inputs.shifted_workload()[t]
    plan = cjt.Plan(N, alpha, beta, M=13, rec_store=1)
    j = np.unique(np.concatenate([np.arange(0, 12), N - np.arange(0, 12), inputs.rng(9).integers(0, N + 1, 40)]))
    fwd = run(cjt, plan, c, cjt.CJT_FWD)
    err = np.abs(orc.cheb_series(fwd, j, N) - orc.jacobi_series(c, alpha, beta, j, N))
    for q, jj in enumerate(j):
        scale = float(np.abs(c * orc.jacobi_values(N, alpha, beta, int(jj), N)).sum())
        assert err[q] <= TOL * max(l1(c), scale)
    assert np.max(np.abs(run(cjt, plan, fwd, cjt.CJT_INV) - c)) <= TOL * l1(c)
    fx = np.load(os.path.join(GOLDEN, "oracle_shift%d_inv_N%d.npz" % (t, N)))
    assert str(fx["input_sha256"]) == hashlib.sha256(np.ascontiguousarray(c).tobytes()).hexdigest()
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - fx["out"])) <= TOL * l1(c)


def test_shifted_in_a_batch_equals_alone(cjt):
    plans, cs, dirs, offs, pos = [], [], [], [], 0
    for t, (N, a, b) in enumerate([(300, 1.5, 0.25), (1024, 0.8, 0.4), (777, 0.1, 1.2), (64, 1.5, 1.5)]):
        plans.append(cjt.Plan(N, a, b, shared_workspace=True))
        cs.append(inputs.decaying_coefficients(N, 1.0, 800 + t))
        dirs.append(cjt.CJT_FWD if t % 2 == 0 else cjt.CJT_INV)
        offs.append(pos)
        pos += N + 1
    x = dev(np.concatenate(cs))
    out = torch.full_like(x, float("nan"))
    cjt.cjt_execute_batched(plans, dirs, offs, x, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    for p, d, c, off in zip(plans, dirs, cs, offs):
        arena = torch.empty(max(p.info()["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
        fn = cjt.cjt_forward_ws if d == cjt.CJT_FWD else cjt.cjt_inverse_ws
        xa = dev(c)
        alone = torch.empty_like(xa)
        fn(p, xa, alone, arena)
        torch.cuda.synchronize()
        assert np.array_equal(alone.cpu().numpy(), o[off:off + c.size])


@pytest.mark.parametrize("alpha,beta", [(-0.6, 0.0), (1.6, 0.0), (0.0, 2.0), (0.0, -0.51), (0.0, float("nan"))])
def test_domain(cjt, alpha, beta):
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(64, alpha, beta)
    assert e.value.code == cjt.CJT_EDOMAIN
