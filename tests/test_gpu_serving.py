"""Serving: continuous batching of transforms of different N, direction and
(alpha, beta) as they arrive.  Requests submitted while others run are admitted
into free slots and overlap with them on the device; every result must equal,
bit for bit, the same request run alone with a fresh plan of the same options."""
import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt, serve
    return cjt, serve


def make_requests(serve, n=40, seed=inputs.BASE_SEED + 4000):
    r = inputs.rng(seed)
    reqs = []
    for t in range(n):
        N = int(np.clip(np.rint(np.exp(r.uniform(np.log(128), np.log(20000)))), 128, 20000))
        a, b = (float(v) for v in r.uniform(-0.45, 0.45, 2))
        d = 1 if r.uniform() < 0.5 else 2
        reqs.append(serve.Request(N, a, b, d, inputs.decaying_coefficients(N, 1.0, seed + t)))
    # a repeated request reuses the resident plan
    N, a, b, d = reqs[0].N, reqs[0].alpha, reqs[0].beta, reqs[0].direction
    reqs.append(serve.Request(N, a, b, d, inputs.decaying_coefficients(N, 1.0, seed + 999)))
    return reqs


def test_results_in_the_mix_equal_alone(mods, orc):
    cjt, serve = mods
    server = serve.Server(slots=8, mem_budget=20e9, planners=3)
    reqs = make_requests(serve)
    serve.poisson_run(server, reqs, rate=5000.0, seed=1)
    st = server.stats()
    server.close()
    assert all(not r.error for r in reqs)
    assert st["requests"] == len(reqs)
    assert st["max_inflight"] > 1          # work from several requests overlapped on the device
    for r in reqs:
        p = cjt.Plan(r.N, r.alpha, r.beta, directions=r.direction, **server.plan_options(r.N))
        x = torch.from_numpy(r.x).cuda()
        y = cjt.cjt_forward(p, x) if r.direction == 1 else cjt.cjt_inverse(p, x)
        torch.cuda.synchronize()
        assert np.array_equal(r.out, y.cpu().numpy()), r.rid
        p.close()
    for r in reqs[:4]:
        want = orc.forward(r.x, r.alpha, r.beta) if r.direction == 1 else orc.inverse(r.x, r.alpha, r.beta)
        assert np.max(np.abs(r.out - want)) <= 1e-12 * np.abs(r.x).sum()


def test_memory_budget_evicts_idle_plans(mods):
    cjt, serve = mods
    server = serve.Server(slots=2, mem_budget=3e8, planners=1)
    reqs = make_requests(serve, n=12, seed=inputs.BASE_SEED + 4100)
    serve.poisson_run(server, reqs, rate=200.0, seed=2)
    st = server.stats()
    server.close()
    assert st["requests"] == len(reqs)
    assert st["resident_plan_bytes"] + st["slot_bytes"] <= 3e8 + 4000 * 20001


def test_bad_requests_fail_alone(mods):
    """A malformed request is refused at submit; one whose plan cannot be built (alpha
    outside [-1/2, 3/2]) comes back with an error; the requests around it are served."""
    cjt, serve = mods
    server = serve.Server(slots=2, mem_budget=5e9, planners=1)
    with pytest.raises(ValueError):
        server.submit(serve.Request(100, 0.1, 0.2, cjt.CJT_FWD, np.ones(100)))
    with pytest.raises(ValueError):
        server.submit(serve.Request(100, 0.1, 0.2, 3, np.ones(101)))
    good = make_requests(serve, n=3, seed=inputs.BASE_SEED + 4200)
    bad = serve.Request(300, 2.5, 0.0, cjt.CJT_FWD, np.ones(301))
    serve.poisson_run(server, [good[0], bad, good[1], good[2]], rate=2000.0, seed=3)
    server.close()
    assert bad.error and bad.out is None
    assert all(not r.error and r.out is not None for r in good[:3])
