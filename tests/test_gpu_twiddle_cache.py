"""Twiddle tables are shared by plans of the same transform lengths and precision (a
per-device cache).  A plan's results must not depend on whether its tables were built for
it, taken from a live plan, taken from the cache after the plan that built them was
destroyed, or rebuilt after the cache dropped them; plans built from many host threads at
once, which race for the same tables, must give the results of plans built one by one."""
import os
import threading

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
    assert torch.cuda.is_available()
    return mod


def run(cjt, plan, c, d, stream=None):
    x = torch.from_numpy(c).cuda()
    if stream is None:
        y = cjt.cjt_forward(plan, x) if d == cjt.CJT_FWD else cjt.cjt_inverse(plan, x)
        torch.cuda.synchronize()
        return y.cpu().numpy()
    with torch.cuda.stream(stream):
        x = torch.from_numpy(c).to("cuda", non_blocking=False)
        y = cjt.cjt_forward(plan, x, stream=stream) if d == cjt.CJT_FWD else cjt.cjt_inverse(plan, x, stream=stream)
    stream.synchronize()
    return y.cpu().numpy()


CASES = [(4096, 0.1, -0.3, 0), (3000, -0.2, 0.4, 0), (777, 0.3, 0.3, 0), (5000, 0.0, 0.25, 2), (1024, -0.4, 0.1, 1)]


def prec(cjt, k):
    return (cjt.CJT_FP64, cjt.CJT_MIXED, cjt.CJT_DFLOAT)[k]


def reference(cjt):
    out = {}
    for N, a, b, k in CASES:
        c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + N)
        p = cjt.Plan(N, a, b, precision=prec(cjt, k))
        out[(N, k)] = (c, run(cjt, p, c, cjt.CJT_FWD), run(cjt, p, c, cjt.CJT_INV))
        p.close()
    return out


def test_tables_from_a_live_plan_a_dead_plan_and_a_rebuild(cjt):
    ref = reference(cjt)
    for N, a, b, k in CASES:
        c, yf, yi = ref[(N, k)]
        first = cjt.Plan(N, -a, b, precision=prec(cjt, k))         # same lengths, other parameters
        live = cjt.Plan(N, a, b, precision=prec(cjt, k))           # tables of a live plan
        assert np.array_equal(run(cjt, live, c, cjt.CJT_FWD), yf)
        first.close()
        assert np.array_equal(run(cjt, live, c, cjt.CJT_INV), yi)  # its tables outlive the builder
        live.close()
        cached = cjt.Plan(N, a, b, precision=prec(cjt, k))         # tables from the cache, no plan alive
        assert np.array_equal(run(cjt, cached, c, cjt.CJT_FWD), yf)
        cached.close()
    old = os.environ.get("CJT_TWIDDLE_CACHE_MB")
    os.environ["CJT_TWIDDLE_CACHE_MB"] = "0"   # unused tables are freed on release
    try:
        for N, a, b, k in CASES:
            c, yf, yi = ref[(N, k)]
            p = cjt.Plan(N, a, b, precision=prec(cjt, k))
            assert np.array_equal(run(cjt, p, c, cjt.CJT_INV), yi)
            p.close()
            q = cjt.Plan(N, a, b, precision=prec(cjt, k))         # rebuilt
            assert np.array_equal(run(cjt, q, c, cjt.CJT_FWD), yf)
            q.close()
    finally:
        if old is None:
            os.environ.pop("CJT_TWIDDLE_CACHE_MB")
        else:
            os.environ["CJT_TWIDDLE_CACHE_MB"] = old


def test_plans_built_from_many_threads(cjt):
    old = os.environ.get("CJT_TWIDDLE_CACHE_MB")
    os.environ["CJT_TWIDDLE_CACHE_MB"] = "0"   # every thread races to build the tables anew
    try:
        ref = reference(cjt)
        errors, results = [], {}

        def worker(t):
            try:
                torch.cuda.set_device(0)
                s = torch.cuda.Stream()
                for r in range(3):
                    for N, a, b, k in CASES[t % 2::2] if t % 3 else CASES:
                        p = cjt.Plan(N, a, b, precision=prec(cjt, k), stream=s.cuda_stream)
                        c = ref[(N, k)][0]
                        results[(t, r, N, k)] = (run(cjt, p, c, cjt.CJT_FWD, s), run(cjt, p, c, cjt.CJT_INV, s))
                        p.close()
            except Exception as e:  # noqa: BLE001
                errors.append(repr(e))

        ths = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        assert not errors, errors
        assert len(results) > 8
        for (t, r, N, k), (yf, yi) in results.items():
            assert np.array_equal(yf, ref[(N, k)][1]) and np.array_equal(yi, ref[(N, k)][2]), (t, r, N, k)
    finally:
        if old is None:
            os.environ.pop("CJT_TWIDDLE_CACHE_MB")
        else:
            os.environ["CJT_TWIDDLE_CACHE_MB"] = old
