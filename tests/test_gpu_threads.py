"""One shared-workspace plan executed from two host threads at once, each on its own stream
with its own workspace: every execution takes its own side stream and fork/join events from
the library's per-device pool, so neither thread's asymptotic chain can be joined to the
other's.  Every result must equal, bit for bit, the plan run alone."""
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


@pytest.mark.parametrize("overlap", [1, 3])
def test_shared_plan_from_two_threads(cjt, overlap):
    N, a, b = 16384, 0.2, -0.35
    plan = cjt.Plan(N, a, b, shared_workspace=True, overlap=overlap)
    wsb = plan.info()["workspace_bytes"]
    xs = [torch.from_numpy(inputs.decaying_coefficients(N, 1.0, 900 + t)).cuda() for t in range(2)]
    # alone
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    ref = []
    for x in xs:
        f = cjt.cjt_forward_ws(plan, x, torch.empty_like(x), ws)
        i = cjt.cjt_inverse_ws(plan, x, torch.empty_like(x), ws)
        torch.cuda.synchronize()
        ref.append((f.cpu().numpy(), i.cpu().numpy()))
    reps = 30
    outs = [[None] * reps for _ in range(2)]
    errors = []

    def worker(t):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            w = torch.empty(wsb, dtype=torch.uint8, device="cuda")
            x = xs[t]
            res = []
            with torch.cuda.stream(st):
                for r in range(reps):
                    y = torch.empty_like(x)
                    if r % 2 == 0:
                        cjt.cjt_forward_ws(plan, x, y, w, stream=st)
                    else:
                        cjt.cjt_inverse_ws(plan, x, y, w, stream=st)
                    res.append(y)
            st.synchronize()
            outs[t] = [y.cpu().numpy() for y in res]
        except Exception as e:  # surfaced below
            errors.append(repr(e))

    th = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for t in range(2):
        for r in range(reps):
            assert np.array_equal(outs[t][r], ref[t][r % 2]), (t, r)
    plan.close()
