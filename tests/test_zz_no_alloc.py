"""The allocation-free entry point, cjt_cheb_coeffs_noalloc, called through the C ABI.

Some callers cannot call cudaMalloc (code under a host framework's pool
allocator, latency-critical paths, plug-ins in a nearly full device); this
entry point serves them with a fixed device array as its working memory.  It
computes the forward transform's last step, c = T_N^{-1} y, so its output on the
Lobatto values of a Jacobi expansion must agree with the library's forward
transform (cjt_forward) of that expansion, within the tolerance used by the
parity tests.  Two calls in a row (different sizes, then a repeat) check that
the shared array carries nothing over.  This file is collected last.
"""
import ctypes

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


def test_noalloc_matches_forward_on_consecutive_calls(cjt, orc):
    cases = [(4096, 0.1, -0.3), (256, 0.45, 0.45), (65536, -0.2, 0.3), (4096, 0.1, -0.3)]
    outputs = []
    for N, a, b in cases:
        c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + N)
        plan = cjt.Plan(N, a, b)
        ref = cjt.cjt_forward(plan, torch.from_numpy(c).cuda())
        y, _ = orc.forward_values(c, a, b)
        values = torch.from_numpy(y).cuda()
        out = torch.full_like(values, float("nan"))
        cjt.cjt_cheb_coeffs_noalloc(values, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref.cpu().numpy())) <= TOL * np.abs(c).sum(), N
        outputs.append(got)
    assert np.array_equal(outputs[0], outputs[3])


def test_noalloc_rejects_sizes_beyond_its_array(cjt):
    lib = cjt.load()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.cjt_cheb_coeffs_noalloc(cjt.NOALLOC_MAX_N * 2, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), None)
    assert rc == cjt.CJT_EUNSUPPORTED
    rc = lib.cjt_cheb_coeffs_noalloc(6, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None)
    assert rc == cjt.CJT_EUNSUPPORTED
