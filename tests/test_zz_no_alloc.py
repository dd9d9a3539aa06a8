"""The allocation-free entry point, cjt_cheb_coeffs_noalloc, called through the C ABI.

Some callers cannot call cudaMalloc (code under a host framework's pool
allocator, latency-critical paths, plug-ins in a nearly full device); this
entry point serves them with a fixed device array as its working memory.  It
computes the forward transform's last step, c = T_N^{-1} y, so on the Lobatto
values y of a Jacobi expansion (the double-double oracle's) its output must equal
the oracle's forward transform of that expansion within the parity tests'
tolerance; it must also agree with the library's forward transform.  Calls in a
row (different sizes, then a repeat) check that the shared array carries nothing
over, and the device's free memory is the same before and after calls at the
largest size.  This file is collected last.
"""
import ctypes
import hashlib
import os

import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def cjt():
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt as mod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mod


def oracle_forward(orc, N, a, b, c):
    """The oracle's forward transform: computed for small N, the stored oracle output
    (tests/golden, written by make_fullsize.py from the oracle) for the workload item at 2^16."""
    if N <= 4096:
        return orc.forward(c, a, b)
    fx = np.load(os.path.join(GOLDEN, "oracle_fwd_N%d.npz" % N))
    assert str(fx["input_sha256"]) == hashlib.sha256(np.ascontiguousarray(c).tobytes()).hexdigest()
    return fx["out"]


def test_noalloc_matches_oracle_on_consecutive_calls(cjt, orc):
    # the single-transform workload's N = 2^16 item, whose oracle output is stored
    big = [it for it in inputs.single_workload(seed=inputs.BASE_SEED) if it[0] == 1 << 16][0]
    cases = [(4096, 0.1, -0.3, inputs.decaying_coefficients(4096, 1.0, inputs.BASE_SEED + 4096)),
             (256, 0.45, 0.45, inputs.decaying_coefficients(256, 1.0, inputs.BASE_SEED + 256)),
             big,
             (4096, 0.1, -0.3, inputs.decaying_coefficients(4096, 1.0, inputs.BASE_SEED + 4096))]
    outputs = []
    for N, a, b, c in cases:
        want = oracle_forward(orc, N, a, b, c)
        plan = cjt.Plan(N, a, b)
        lib_fwd = cjt.cjt_forward(plan, torch.from_numpy(c).cuda()).cpu().numpy()
        y, _ = orc.forward_values(c, a, b)
        values = torch.from_numpy(y).cuda()
        out = torch.full_like(values, float("nan"))
        cjt.cjt_cheb_coeffs_noalloc(values, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        tol = TOL * np.abs(c).sum()
        assert np.max(np.abs(got - want)) <= tol, N
        assert np.max(np.abs(got - lib_fwd)) <= tol, N
        outputs.append(got)
    assert np.array_equal(outputs[0], outputs[3])


def test_noalloc_allocates_nothing(cjt):
    N = cjt.NOALLOC_MAX_N
    values = torch.from_numpy(inputs.decaying_coefficients(N, 1.0, 5)).cuda()
    out = torch.empty_like(values)
    cjt.cjt_cheb_coeffs_noalloc(values, out)      # first call on the device: the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(4):
        cjt.cjt_cheb_coeffs_noalloc(values, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_array(cjt):
    lib = cjt.load()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.cjt_cheb_coeffs_noalloc(cjt.NOALLOC_MAX_N * 2, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), None)
    assert rc == cjt.CJT_EUNSUPPORTED
    rc = lib.cjt_cheb_coeffs_noalloc(6, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None)
    assert rc == cjt.CJT_EUNSUPPORTED
