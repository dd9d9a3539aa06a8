"""Transform launch configurations (cjt_fft_set_config, set by the autotuner): the tile
occupancy target changes only the work split between CTAs, so results stay bit-identical;
the four-step splits (0, 1 and the narrower first pass 2) and the one-pass 8192-point
transform change the order of the arithmetic, and results stay within the library's tolerance
of the oracle.  The default configuration is
restored afterwards."""
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


def run(cjt, N, a, b, c, opts):
    p = cjt.Plan(N, a, b, **opts)
    x = torch.from_numpy(c).cuda()
    f = cjt.cjt_forward(p, x).cpu().numpy()
    i = cjt.cjt_inverse(p, x).cpu().numpy()
    p.close()
    return f, i


@pytest.mark.parametrize("precision", [0, 1])
def test_fft_configurations(cjt, orc, precision):
    N, a, b = 4096, 0.15, -0.25
    c = inputs.decaying_coefficients(N, 1.0, 321)
    opts = {"precision": precision, "M": 13}
    lens = range(1, 23)
    saved = {lg: cjt.fft_get_config(pr, lg) for pr in (0, precision) for lg in lens}
    try:
        ref = run(cjt, N, a, b, c, opts)
        for pr in {0, precision}:
            for lg in lens:
                cjt.fft_set_config(pr, lg, 2, saved[lg]["split"], saved[lg]["single_max_log2"])
        got = run(cjt, N, a, b, c, opts)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        for pr in {0, precision}:
            for lg in lens:
                cjt.fft_set_config(pr, lg, 8, 1, 13)
        got = run(cjt, N, a, b, c, opts)
        tol = TOL * np.abs(c).sum() if precision == 0 else None
        fwd, inv = orc.forward(c, a, b), orc.inverse(c, a, b)
        if precision == 0:
            assert np.max(np.abs(got[0] - fwd)) <= tol and np.max(np.abs(got[1] - inv)) <= tol
        else:
            p = cjt.Plan(N, a, b, **opts)
            bf, bi = cjt.error_bound(p, cjt.CJT_FWD), cjt.error_bound(p, cjt.CJT_INV)
            p.close()
            l1 = np.abs(c).sum()
            assert np.max(np.abs(got[0] - fwd)) <= bf * l1 and np.max(np.abs(got[1] - inv)) <= bi * l1
        # the narrower first pass (split 2), on power-of-two and radix-5 grids (N = 9000 plans
        # on 10240 = 5 2^11: rows of 4096 and 8192 points)
        for pr in {0, precision}:
            for lg in lens:
                cjt.fft_set_config(pr, lg, 4, 2, 12)
        for n, sd in ((N, 321), (9000, 322)):
            cn = c if n == N else inputs.decaying_coefficients(n, 1.0, sd)
            got = run(cjt, n, a, b, cn, opts)
            fwd, inv = orc.forward(cn, a, b), orc.inverse(cn, a, b)
            l1 = np.abs(cn).sum()
            if precision == 0:
                bf = bi = TOL
            else:
                p = cjt.Plan(n, a, b, **opts)
                bf, bi = cjt.error_bound(p, cjt.CJT_FWD), cjt.error_bound(p, cjt.CJT_INV)
                p.close()
            assert np.max(np.abs(got[0] - fwd)) <= bf * l1 and np.max(np.abs(got[1] - inv)) <= bi * l1, n
        assert cjt.fft_time(precision, 16, 64) > 0
    finally:
        for (pr, lg), v in ((k, v) for k, v in [((pr, lg), saved[lg]) for pr in (0, precision) for lg in lens]):
            cjt.fft_set_config(pr, lg, v["ctas_per_sm"], v["split"], v["single_max_log2"])
