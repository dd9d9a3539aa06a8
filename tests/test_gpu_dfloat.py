"""GPU parity of the double-float form (CJT_DFLOAT) against the CPU oracle.

In this form the asymptotic transforms (Eq. "PNASY" and its transpose), their pre-scaled
inputs and the stored recurrence values are evaluated in double-float arithmetic (pairs of
floats, about 48 significant bits, on the FP32 pipe); the Hahn coefficients and scalings,
the recurrences and the final DCT-I stay in FP64.  It is held to the FP64 tolerance
max |c_gpu - c_oracle| <= 1e-12 ||c||_1.
"""
import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12
PARAMS = [(0.1, -0.3), (0.45, 0.45), (-0.45, 0.2), (0.0, 0.0), (-0.5, -0.5), (0.5, -0.5)]


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


@pytest.mark.parametrize("alpha,beta", PARAMS)
@pytest.mark.parametrize("N", [1, 2, 8, 64, 1024, 4096])
def test_dfloat_matches_oracle(cjt, orc, N, alpha, beta):
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 11 * N)
    plan = cjt.Plan(N, alpha, beta, precision=cjt.CJT_DFLOAT)
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_FWD) - orc.forward(c, alpha, beta))) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - orc.inverse(c, alpha, beta))) <= TOL * l1(c)


@pytest.mark.parametrize("opts", [dict(rec_store=1), dict(M=13, rec_store=1, ratio=0.05, seg_len=1024),
                                  dict(M=20), dict(M=3, rec_store=1), dict(use_asy=-1, rec_store=1),
                                  dict(rec_store=1, seg_len=32), dict(M=16, ratio=0.2)])
def test_dfloat_options(cjt, orc, opts):
    """Partition, M, the work split and stored recurrence values change only the rounding."""
    N, a, b = 4096, -0.3, 0.45
    c = inputs.decaying_coefficients(N, 1.5, 321)
    plan = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, **opts)
    info = plan.info()
    assert info["precision"] == cjt.CJT_DFLOAT
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_FWD) - orc.forward(c, a, b))) <= TOL * l1(c), info
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - orc.inverse(c, a, b))) <= TOL * l1(c), info


@pytest.mark.parametrize("N", [3, 100, 1000, 3001, 10007])
def test_dfloat_general_N(cjt, orc, N):
    """N not a power of two: double-float Bluestein transforms."""
    a, b = 0.2, -0.45
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 13 * N)
    plan = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, rec_store=1)
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_FWD) - orc.forward(c, a, b))) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - orc.inverse(c, a, b))) <= TOL * l1(c)


def test_dfloat_16384_elementwise(cjt, orc):
    N = 1 << 14
    a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 2001)
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED + 21)
    plan = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, M=13, rec_store=1)
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_FWD) - orc.forward(c, a, b))) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - orc.inverse(c, a, b))) <= TOL * l1(c)


@pytest.mark.parametrize("logN", [16, 18])
def test_dfloat_full_size(cjt, orc, logN):
    """At full size: sampled value identities (double-double oracle), c_jac_0 from the
    moments, the forward-then-inverse round trip, and agreement with the FP64 GPU form.
    Every coefficient of both directions is compared with the double-double oracle at these
    sizes by the full-size parity tests."""
    N = 1 << logN
    a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 3000 + logN)
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED + 30 + logN)
    plan = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, M=13, rec_store=1)
    rng = inputs.rng(6)
    j = np.unique(np.concatenate([np.arange(0, 40), N - np.arange(0, 40), rng.integers(0, N + 1, 400)]))
    fwd = run(cjt, plan, c, cjt.CJT_FWD)
    assert np.max(np.abs(orc.cheb_series(fwd, j, N) - orc.jacobi_series(c, a, b, j, N))) <= TOL * l1(c)
    inv = run(cjt, plan, c, cjt.CJT_INV)
    mu = orc.moments(N, a, b)
    assert abs(inv[0] - np.dot(c, mu) / mu[0]) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, plan, fwd, cjt.CJT_INV) - c)) <= TOL * l1(c)
    p64 = cjt.Plan(N, a, b, M=13, rec_store=1)
    assert np.max(np.abs(fwd - run(cjt, p64, c, cjt.CJT_FWD))) <= TOL * l1(c)
    assert np.max(np.abs(inv - run(cjt, p64, c, cjt.CJT_INV))) <= TOL * l1(c)


def test_dfloat_is_a_different_rounding(cjt):
    """The double-float kernels run (their rounding differs from the FP64 form's) and the
    stored values take the same 8 bytes per recurrence step."""
    N, a, b = 4096, 0.1, -0.3
    c = inputs.decaying_coefficients(N, 1.0, 5)
    pd = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, rec_store=1, M=10)
    p64 = cjt.Plan(N, a, b, rec_store=1, M=10)
    assert pd.info()["rec_store_bytes"] == p64.info()["rec_store_bytes"] > 0
    for d in (cjt.CJT_FWD, cjt.CJT_INV):
        yd, y64 = run(cjt, pd, c, d), run(cjt, p64, c, d)
        assert not np.array_equal(yd, y64)
        assert np.max(np.abs(yd - y64)) <= TOL * l1(c)
        assert np.array_equal(yd, run(cjt, pd, c, d))   # deterministic


def test_dfloat_in_a_batch_equals_alone(cjt):
    """Double-float and FP64 plans mixed in one batched execution give each item's result
    bit for bit as alone."""
    rng = inputs.rng(77)
    plans, cs, dirs, offs, pos = [], [], [], [], 0
    for t, N in enumerate([300, 1024, 4096, 777, 2048, 64]):
        prec = cjt.CJT_DFLOAT if t % 2 == 0 else cjt.CJT_FP64
        a, b = rng.uniform(-0.45, 0.45, 2)
        plans.append(cjt.Plan(N, float(a), float(b), precision=prec, shared_workspace=True,
                              rec_store=int(t % 3 == 0)))
        cs.append(inputs.decaying_coefficients(N, 1.0, 900 + t))
        dirs.append(cjt.CJT_FWD if t % 4 < 2 else cjt.CJT_INV)
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


@pytest.mark.parametrize("store", [0, 1])
@pytest.mark.parametrize("s", [2.0 ** -600, 2.0 ** 600, 1e-200, 3.7e150])
def test_dfloat_input_scale(cjt, orc, s, store):
    """The double-float form scales its input by an exact power of two (from max |c|) before
    converting it, so inputs anywhere in the FP64 range keep their relative accuracy, and a
    power-of-two scaling of the input scales the result exactly."""
    N, a, b = 4096, 0.3, -0.2
    c = inputs.decaying_coefficients(N, 1.0, 17)
    plan = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, M=13, rec_store=store)
    for d, ref in ((cjt.CJT_FWD, orc.forward(c, a, b)), (cjt.CJT_INV, orc.inverse(c, a, b))):
        y1 = run(cjt, plan, c, d)
        ys = run(cjt, plan, c * s, d)
        assert np.max(np.abs(ys / s - ref)) <= TOL * l1(c)
        if s == 2.0 ** round(np.log2(s)):
            assert np.array_equal(ys, y1 * s)


def test_dfloat_at_2_20(cjt, orc):
    """N = 2^20 (the size of the large mixed-precision workload): the double-float form
    stays within the FP64 bound of the FP64 GPU form, and of the sampled oracle values."""
    N = 1 << 20
    a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 4020)
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 40)
    pd = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, M=16, seg_len=1024, rec_store=1)
    p64 = cjt.Plan(N, a, b, M=16, seg_len=1024)
    for d in (cjt.CJT_FWD, cjt.CJT_INV):
        assert np.max(np.abs(run(cjt, pd, c, d) - run(cjt, p64, c, d))) <= TOL * l1(c)
    j = inputs.rng(8).integers(0, N + 1, 64)
    fwd = run(cjt, pd, c, cjt.CJT_FWD)
    assert np.max(np.abs(orc.cheb_series(fwd, j, N) - orc.jacobi_series(c, a, b, j, N))) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, pd, fwd, cjt.CJT_INV) - c)) <= TOL * l1(c)
