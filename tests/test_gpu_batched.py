"""Batched forms: cjt_execute_batched over concurrent lanes, the graph-captured
cjt_batch (replayed twice), and the explicit-workspace entry points.  Every
batched result must equal, bit for bit, the same item run alone (same kernels,
deterministic reductions), for any mix of N, (alpha, beta), direction and precision."""
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


def mixed_items(count=24, seed=inputs.BASE_SEED + 500):
    r = inputs.rng(seed)
    Ns = np.clip(np.rint(np.exp(r.uniform(np.log(64), np.log(20000), count))).astype(int), 64, 20000)
    Ns[:4] = [1024, 4096, 3001, 64]
    items = []
    for t, N in enumerate(Ns):
        a, b = r.uniform(-0.45, 0.45, 2)
        d = 1 if (t % 2 == 0) else 2
        prec = 1 if (t % 5 == 3) else 0
        items.append((int(N), float(a), float(b), d, prec, inputs.decaying_coefficients(int(N), 1.0, seed + t)))
    return items


def run_alone(cjt, items):
    outs = []
    for N, a, b, d, prec, c in items:
        p = cjt.Plan(N, a, b, precision=prec)
        x = torch.from_numpy(c).cuda()
        y = cjt.cjt_forward(p, x) if d == 1 else cjt.cjt_inverse(p, x)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy())
        p.close()
    return outs


def pack(items):
    offs, pos = [], 0
    for N, *_ in items:
        offs.append(pos)
        pos += N + 1
    x = np.concatenate([it[5] for it in items])
    return offs, torch.from_numpy(x).cuda()


def test_execute_batched_equals_alone(cjt):
    items = mixed_items()
    ref = run_alone(cjt, items)
    plans = [cjt.Plan(N, a, b, precision=prec, shared_workspace=True) for N, a, b, d, prec, _ in items]
    offs, x = pack(items)
    out = torch.full_like(x, float("nan"))
    cjt.cjt_execute_batched(plans, [it[3] for it in items], offs, x, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    for (N, *_), off, r in zip(items, offs, ref):
        assert np.array_equal(o[off:off + N + 1], r), N


def test_batch_graph_equals_alone_and_replays(cjt, orc):
    items = mixed_items(count=16, seed=inputs.BASE_SEED + 900)
    ref = run_alone(cjt, items)
    plans = [cjt.Plan(N, a, b, precision=prec, shared_workspace=True) for N, a, b, d, prec, _ in items]
    offs, x = pack(items)
    out = torch.full_like(x, float("nan"))
    batch = cjt.Batch(plans, [it[3] for it in items], offs, x, out, nstreams=8)
    info = batch.info()
    assert info["kernels"] > 16 and info["arena_bytes"] > 0
    for rep in range(2):
        out.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        for (N, *_), off, r in zip(items, offs, ref):
            assert np.array_equal(o[off:off + N + 1], r), (rep, N)
    # and one item against the oracle, for good measure
    N, a, b, d, prec, c = items[0]
    want = orc.forward(c, a, b) if d == 1 else orc.inverse(c, a, b)
    tol = (1e-12 if prec == 0 else 1e-5) * np.abs(c).sum()
    assert np.max(np.abs(o[offs[0]:offs[0] + N + 1] - want)) <= tol
    batch.close()


@pytest.mark.parametrize("overlap", [2, 3])
def test_batch_graph_overlap_modes(cjt, overlap):
    """A captured batch of plans whose recurrence runs on its own side stream (or whose
    chains share one priority) replays to the items' results alone, bit for bit."""
    items = mixed_items(count=12, seed=inputs.BASE_SEED + 950)
    ref = run_alone(cjt, items)
    plans = [cjt.Plan(N, a, b, precision=prec, shared_workspace=True, overlap=overlap)
             for N, a, b, d, prec, _ in items]
    offs, x = pack(items)
    out = torch.full_like(x, float("nan"))
    batch = cjt.Batch(plans, [it[3] for it in items], offs, x, out, nstreams=4)
    for rep in range(2):
        out.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        for (N, *_), off, r in zip(items, offs, ref):
            assert np.array_equal(o[off:off + N + 1], r), (rep, N)
    batch.close()


def test_workspace_entry_points(cjt):
    N, a, b = 5000, 0.2, -0.1
    c = inputs.decaying_coefficients(N, 1.0, 17)
    own = cjt.Plan(N, a, b)
    shared = cjt.Plan(N, a, b, shared_workspace=True)
    assert shared.info()["device_bytes"] < own.info()["device_bytes"]
    ws = torch.empty(shared.info()["workspace_bytes"], dtype=torch.uint8, device="cuda")
    x = torch.from_numpy(c).cuda()
    y1 = cjt.cjt_forward(own, x)
    y2 = cjt.cjt_forward_ws(shared, x, torch.empty_like(x), ws)
    z1 = cjt.cjt_inverse(own, x)
    z2 = cjt.cjt_inverse_ws(shared, x, torch.empty_like(x), ws)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2) and torch.equal(z1, z2)
    with pytest.raises(cjt.CJTError) as e:
        cjt.cjt_forward(shared, x)
    assert e.value.code == cjt.CJT_EINVAL
