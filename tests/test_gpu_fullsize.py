"""GPU parity at the benchmark's sizes, element by element, against stored oracle outputs.

The fixtures under tests/golden/oracle_*.npz were written by tests/golden/make_fullsize.py,
which calls only the CPU oracle (double-double O(N^2) definitions of Eq. "CJT" and
Eq. "iCJT").  Each test regenerates the seeded input, checks it against the digest stored
in the fixture, runs the CUDA path through the C ABI and compares every stored entry:

  FP64 and double-float forms:  max |c_gpu - c_oracle| <= 1e-12 ||c_in||_1
                                (the library's bound, forward and inverse alike)
  mixed form (FP32 transforms):  max |c_gpu - c_oracle| <= the plan's stated bound
                                (cjt_error_bound: the componentwise FP32 transform error
                                carried through C_{n,m}, u_m, v_m, the weights and 1/A_n)

Option sets: the defaults, the option sets the autotuner picks for the single-transform
benchmark (stored recurrence values, coarse block ratio), so the configuration the benchmark
times is the one checked here, and the serving loop's one-shot options (whole rows).
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

SINGLE = [1 << 12, 1 << 14, 1 << 16, 1 << 18]
FP64_OPTIONS = [dict(), dict(M=10, ratio=0.05, rec_store=1, seg_len=1024),
                dict(M=13, ratio=0.05, rec_store=1, seg_len=1024), dict(M=16, seg_len=256),
                dict(M=13, seg_len=256, seg_whole=8192)]
DF_OPTIONS = [dict(), dict(M=13, ratio=0.05, rec_store=1, seg_len=1024)]


@pytest.fixture(scope="module")
def cjt():
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt as mod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mod


def fixture(name):
    path = os.path.join(GOLDEN, "oracle_%s.npz" % name)
    if not os.path.exists(path):
        pytest.fail("missing oracle fixture %s (run tests/golden/make_fullsize.py)" % path)
    return np.load(path)


def single_input(N):
    for n, a, b, c in inputs.single_workload(Ns=tuple(SINGLE), seed=inputs.BASE_SEED):
        if n == N:
            return a, b, c
    raise KeyError(N)


def checked(fx, c):
    assert hashlib.sha256(np.ascontiguousarray(c).tobytes()).hexdigest() == str(fx["input_sha256"])
    return fx["idx"], fx["out"]


def run(cjt, plan, c, direction):
    x = torch.from_numpy(np.ascontiguousarray(c)).to("cuda")
    y = cjt.cjt_forward(plan, x) if direction == 1 else cjt.cjt_inverse(plan, x)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def compare(got, idx, ref):
    g = got if idx.size == 0 else got[idx]
    assert g.shape == ref.shape
    return float(np.max(np.abs(g - ref)))


@pytest.mark.parametrize("opts", FP64_OPTIONS, ids=lambda o: ",".join("%s=%s" % kv for kv in o.items()) or "default")
@pytest.mark.parametrize("N", SINGLE)
@pytest.mark.parametrize("direction", [1, -1], ids=["forward", "inverse"])
def test_fp64_elementwise_vs_oracle(cjt, N, direction, opts):
    a, b, c = single_input(N)
    idx, ref = checked(fixture(("fwd_N%d" if direction == 1 else "inv_N%d") % N), c)
    plan = cjt.Plan(N, a, b, **opts)
    err = compare(run(cjt, plan, c, direction), idx, ref)
    assert err <= TOL * float(np.abs(c).sum()), (err, plan.info())


@pytest.mark.parametrize("opts", DF_OPTIONS, ids=lambda o: ",".join("%s=%s" % kv for kv in o.items()) or "default")
@pytest.mark.parametrize("N", SINGLE)
@pytest.mark.parametrize("direction", [1, -1], ids=["forward", "inverse"])
def test_dfloat_elementwise_vs_oracle(cjt, N, direction, opts):
    a, b, c = single_input(N)
    idx, ref = checked(fixture(("fwd_N%d" if direction == 1 else "inv_N%d") % N), c)
    plan = cjt.Plan(N, a, b, precision=cjt.CJT_DFLOAT, **opts)
    err = compare(run(cjt, plan, c, direction), idx, ref)
    assert err <= TOL * float(np.abs(c).sum()), (err, plan.info())


@pytest.mark.parametrize("N", SINGLE)
@pytest.mark.parametrize("direction", [1, -1], ids=["forward", "inverse"])
def test_mixed_within_stated_bound_vs_oracle(cjt, N, direction):
    a, b, c = single_input(N)
    idx, ref = checked(fixture(("fwd_N%d" if direction == 1 else "inv_N%d") % N), c)
    plan = cjt.Plan(N, a, b, precision=cjt.CJT_MIXED, M=13, ratio=0.05, rec_store=1, seg_len=1024)
    err = compare(run(cjt, plan, c, direction), idx, ref)
    bound = cjt.error_bound(plan, cjt.CJT_FWD if direction == 1 else cjt.CJT_INV) * float(np.abs(c).sum())
    assert err <= bound, (err, bound)


def big_item(t):
    N, a, b, d, c = inputs.mixed_large_workload(2, 1 << 20, seed=inputs.BASE_SEED)[t]
    return N, a, b, d, c


@pytest.mark.parametrize("precision", ["fp64", "dfloat"])
def test_forward_2p20_elementwise_vs_oracle(cjt, precision):
    """The large workload's first item (forward, N = 2^20): 8192 sampled coefficients of the
    double-double oracle, both ends included."""
    N, a, b, d, c = big_item(0)
    idx, ref = checked(fixture("fwd_N%d" % N), c)
    prec = cjt.CJT_FP64 if precision == "fp64" else cjt.CJT_DFLOAT
    plan = cjt.Plan(N, a, b, precision=prec, M=16, seg_len=1024, directions=cjt.CJT_FWD)
    err = compare(run(cjt, plan, c, 1), idx, ref)
    assert err <= TOL * float(np.abs(c).sum()), err


def test_mixed_2p20_both_directions_vs_oracle(cjt):
    """The large mixed-precision workload's first two items (plan options of its benchmark):
    the forward item against the double-double oracle, the inverse item against the
    plain-double oracle, whose own error (stored in the fixture, measured against the
    double-double oracle at 2^14 and 2^16) is orders of magnitude below the bound."""
    for t in (0, 1):
        N, a, b, d, c = big_item(t)
        fx = fixture(("fwd_N%d" if d == 1 else "inv_N%d") % N)
        idx, ref = checked(fx, c)
        dirn = cjt.CJT_FWD if d == 1 else cjt.CJT_INV
        plan = cjt.Plan(N, a, b, precision=cjt.CJT_MIXED, M=16, seg_len=1024, directions=dirn)
        err = compare(run(cjt, plan, c, d), idx, ref)
        bound = cjt.error_bound(plan, dirn) * float(np.abs(c).sum())
        if d == -1:
            assert float(fx["f64_err_N65536"]) * float(np.abs(c).sum()) < 1e-3 * bound
        assert err <= bound, (t, err, bound)
