"""Grouped batched execution (cjt_batch_create): the stages of many transforms run in one
launch per stage and transform length class, in memory-bounded waves.  Every item of a
replayed batch must equal, bit for bit, the same plan run alone: the grouped kernels run the
single-transform kernels' per-element arithmetic.  The batches mix what runs grouped (FP64
and mixed precision, stored recurrence or not, parity fold, recurrence-only plans, N = 1)
with what the batch runs one chain per item (double-float form, shifted parameters,
Bluestein lengths on the paper's grid), and small arenas force many waves."""
import os

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


def diverse_items(cjt, seed):
    r = inputs.rng(seed)
    base = [(1, {}), (2, {}), (63, {}), (64, {"rec_store": 1}), (100, {"use_asy": -1}), (1000, {}),
            (3001, {"rec_store": 1}), (4096, {"M": 13, "ratio": 0.05}), (8191, {"precision": cjt.CJT_MIXED}),
            (20000, {"rec_store": 1, "seg_len": 256}), (65536, {"M": 10, "seg_len": 1024}),
            (5000, {"precision": cjt.CJT_DFLOAT}), (777, {"grid": -1}), (1500, {"shift": (1.2, 0.3)}),
            (2048, {"fold": True}), (12000, {"precision": cjt.CJT_MIXED, "rec_store": 1}), (300, {"M": 20}),
            (30000, {"M": 13, "seg_len": 256, "seg_whole": 8192}), (5000, {"seg_len": 256, "seg_whole": 2048})]
    items = []
    for t in range(3 * len(base)):
        N, opts = base[t % len(base)]
        opts = dict(opts)
        a, b = (float(v) for v in r.uniform(-0.45, 0.45, 2))
        if opts.pop("fold", False):
            b = a
            opts["rec_store"] = 1
        if "shift" in opts:
            a, b = opts.pop("shift")
        d = cjt.CJT_FWD if (t + t // len(base)) % 2 == 0 else cjt.CJT_INV
        items.append((N, a, b, d, opts, inputs.decaying_coefficients(N, 1.0, seed + t)))
    return items


def run_alone(cjt, items):
    outs = []
    for N, a, b, d, opts, c in items:
        p = cjt.Plan(N, a, b, directions=d, **opts)
        x = torch.from_numpy(c).cuda()
        y = cjt.cjt_forward(p, x) if d == cjt.CJT_FWD else cjt.cjt_inverse(p, x)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy())
        p.close()
    return outs


def run_batch(cjt, items, arena_mb, reps=2):
    plans = [cjt.Plan(N, a, b, directions=d, shared_workspace=True, **opts) for N, a, b, d, opts, _ in items]
    offs, pos = [], 0
    for N, *_ in items:
        offs.append(pos)
        pos += N + 1
    x = torch.from_numpy(np.concatenate([it[5] for it in items])).cuda()
    out = torch.empty_like(x)
    old = os.environ.get("CJT_BATCH_ARENA_MB")
    os.environ["CJT_BATCH_ARENA_MB"] = str(arena_mb)
    try:
        batch = cjt.Batch(plans, [it[3] for it in items], offs, x, out, nstreams=4)
    finally:
        if old is None:
            os.environ.pop("CJT_BATCH_ARENA_MB")
        else:
            os.environ["CJT_BATCH_ARENA_MB"] = old
    results = []
    for _ in range(reps):
        out.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    info = batch.info()
    batch.close()
    return offs, results, info


@pytest.mark.parametrize("arena_mb", [16, 4096])
def test_grouped_batch_equals_alone(cjt, arena_mb):
    items = diverse_items(cjt, inputs.BASE_SEED + 4200)
    ref = run_alone(cjt, items)
    offs, results, info = run_batch(cjt, items, arena_mb)
    for rep, o in enumerate(results):
        for (N, a, b, d, opts, _), off, r in zip(items, offs, ref):
            assert np.array_equal(o[off:off + N + 1], r), (rep, N, d, opts)


def test_grouped_batch_launch_count(cjt):
    """Hundreds of transforms of mixed lengths take a few launches per stage and length class,
    not a chain per transform."""
    items = []
    for t, (N, a, b, d, c) in enumerate(inputs.batch_workload(256, seed=inputs.BASE_SEED + 4300, nmax=8192)):
        items.append((N, a, b, cjt.CJT_FWD if d == 1 else cjt.CJT_INV, {}, c))
    per_item = 0
    for N, a, b, d, opts, c in items[:16]:
        p = cjt.Plan(N, a, b, directions=d)
        inf = p.info()
        per_item += inf["kernels_fwd"] if d == cjt.CJT_FWD else inf["kernels_inv"]
        p.close()
    ref = run_alone(cjt, items[:32])
    offs, results, info = run_batch(cjt, items, 4096, reps=1)
    # 256 items as chains would launch about 16 * per_item kernels (per_item: 16 items' chains)
    assert info["kernels"] < 4 * per_item, (info, per_item)
    for (N, *_), off, r in zip(items[:32], offs, ref):
        assert np.array_equal(results[0][off:off + N + 1], r), N
