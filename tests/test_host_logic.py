"""Host-side logic that needs no GPU: the seeded workload generators, the autotuner's
candidate sets, cache file and work model, the bench's grid choice and traffic gate, the
serving loop's memory admission, and the batch planner's memory budget (the last two with
fake plans), the bench's algorithmic-work count behind the roofline, and the
transform autotuner's choice (with a fake timer)."""
import json

import numpy as np
import pytest

from paper_1602_02618_gb300 import autotune, inputs


def test_batch_workload_shape_and_determinism():
    a = inputs.batch_workload(256)
    b = inputs.batch_workload(256)
    assert len(a) == 256
    Ns = np.array([it[0] for it in a])
    assert Ns.min() >= 64 and Ns.max() <= 65536
    # log-uniform: about half the items lie below the geometric midpoint 2048
    assert 0.35 < np.mean(Ns < 2048) < 0.65
    assert np.mean((Ns & (Ns - 1)) != 0) > 0.9          # mostly not powers of two
    dirs = np.array([it[3] for it in a])
    assert set(dirs) == {1, -1} and 0.35 < np.mean(dirs == 1) < 0.65
    for (N, al, be, d, c), (N2, al2, be2, d2, c2) in zip(a, b):
        assert (N, al, be, d) == (N2, al2, be2, d2) and np.array_equal(c, c2)
        assert -0.45 <= al <= 0.45 and -0.45 <= be <= 0.45
        assert c.shape == (N + 1,) and c.dtype == np.float64
    c = inputs.batch_workload(256, seed=inputs.BASE_SEED + 1)
    assert [it[0] for it in c] != [it[0] for it in a]


def test_coefficient_recipes():
    N = 4096
    g = inputs.rng(inputs.BASE_SEED).standard_normal(N + 1)
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED)
    n1 = np.arange(N + 1) + 1.0
    # (n+1)^1.5 as a product with the correctly rounded square root: the same bits on every
    # platform, and within an ulp or two of the power
    assert np.array_equal(c, g / (n1 * np.sqrt(n1)))
    assert np.max(np.abs(c - g / n1 ** 1.5) / np.abs(c)) < 1e-15
    assert np.array_equal(inputs.decaying_coefficients(N, 1.0, 7), inputs.rng(7).standard_normal(N + 1) / n1)
    u = inputs.irregular_coefficients(N)
    assert u.min() >= 0.0 and u.max() < 1.0
    v = inputs.continuous_coefficients(N)
    assert np.all(np.abs(v) <= 1.0 / (np.arange(N + 1) + 1.0) ** 2)
    items = inputs.single_workload()
    assert [it[0] for it in items] == [1 << 12, 1 << 14, 1 << 16, 1 << 18]
    big = inputs.mixed_large_workload(4, 1024)
    assert [it[3] for it in big] == [1, -1, 1, -1] and all(it[0] == 1024 for it in big)
    reqs = inputs.serving_requests(64)
    assert all(128 <= r[0] <= 1 << 18 and r[3] in (1, -1) for r in reqs)


def test_autotune_candidates():
    small = autotune.candidates(1000, 40e9)
    big = autotune.candidates(1 << 20, 40e9)
    for opts in small + big:
        assert opts["M"] >= 5 and opts["seg_len"] in (256, 1024) and opts["rec_store"] in (0, 1)
    # the recurrence-only candidate only when its stored matrix fits the cap
    assert any(o.get("use_asy") == -1 for o in small)
    assert not any(o.get("use_asy") == -1 for o in big)
    assert any(o["rec_store"] == 0 for o in big) and any(o.get("ratio") == 0.05 for o in big)
    assert len({json.dumps(o, sort_keys=True) for o in big}) == len(big)


def test_autotune_cache_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "cache.json"
    monkeypatch.setenv("CJT_AUTOTUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}
    entry = {"k": {"options": {"M": 10, "seg_len": 256, "rec_store": 1}, "ms": 1.5}}
    autotune._save(entry)
    assert autotune._load() == entry
    path.write_text("{not json")
    assert autotune._load() == {}
    # small N never times anything
    assert autotune.best_options(100, 0.1, -0.3) == {"M": 7, "seg_len": 256}


def test_bench_default_grid_and_traffic_gate(monkeypatch):
    """bench.default_grid is the least G >= N of the forms 2^a, 3 2^a, 5 2^a (brute force), and
    the recorded transform traffic is reported only for the captured workload, plan budget and
    sources: any other digest, budget or workload gives null."""
    import argparse
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    def smooth(g):
        while g % 2 == 0:
            g //= 2
        return g in (1, 3, 5)

    for N in list(range(1, 300)) + [3001, 40000, 45000, 65536, 65537]:
        G = bench.default_grid(N)
        assert G >= N and smooth(G) and all(not smooth(g) for g in range(N, G)), N

    class FakeCJT:
        CJT_FP64, CJT_MIXED = 0, 1

    args = argparse.Namespace(batch_count=4096, batch_fixed=False, batch_plan_gb=bench.FFT_TRAFFIC["plan_budget_gb"])
    ok = bench.measured_fft_traffic(args, FakeCJT.CJT_FP64, FakeCJT)
    assert ok is None or ok["bytes_per_step"] > 0
    assert bench.measured_fft_traffic(args, FakeCJT.CJT_MIXED, FakeCJT) is None
    assert bench.measured_fft_traffic(argparse.Namespace(**dict(vars(args), batch_count=48)), 0, FakeCJT) is None
    assert bench.measured_fft_traffic(argparse.Namespace(**dict(vars(args), batch_plan_gb=1.0)), 0, FakeCJT) is None
    monkeypatch.setitem(bench.FFT_TRAFFIC, "sources", {k: "0" * 64 for k in bench.FFT_TRAFFIC["sources"]})
    assert bench.measured_fft_traffic(args, FakeCJT.CJT_FP64, FakeCJT) is None


def test_mixed_work_model_discounts_fp32_transforms():
    """The batch autotuner's work model counts the mixed form's asymptotic transforms at a
    tenth of their FP64 cost and its final DCT-I / front end in full."""
    from paper_1602_02618_gb300 import cjt
    info = {"fft_len_fwd": 1 << 12, "fft_len_inv": 1 << 13, "nfft_fwd": 11, "nfft_inv": 13,
            "rec_steps_fwd": 1000, "rec_steps_inv": 2000}
    s64, f64 = autotune._work_model(info, 1, cjt.CJT_FP64)
    s32, f32 = autotune._work_model(info, 1, cjt.CJT_MIXED)
    assert s64 == s32 == 1000.0
    one = 5.0 * 4096 * 12 / autotune.ETA_FFT
    assert abs(f64 - 11 * one) < 1e-6 * f64 and abs(f32 - (10 * autotune.MIXED_ASY_FFT_FACTOR + 1) * one) < 1e-6 * f32


# --------------------------------------------------------------------------------------
# serving admission (serve.Server._make_room) on a server without threads or a device
# --------------------------------------------------------------------------------------
class _FakeServePlan:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def _bare_server(budget):
    import collections
    import threading
    from paper_1602_02618_gb300 import serve
    s = serve.Server.__new__(serve.Server)      # no planner/executor threads, no streams
    s.lock = threading.Lock()
    s.cv = threading.Condition(s.lock)
    s.plans = collections.OrderedDict()
    s.plan_bytes = 0
    s.slot_bytes = 0
    s.pending_bytes = 0.0
    s.mem_budget = float(budget)
    s._stop = False
    return s


def _add_plan(s, key, nbytes, users):
    p = _FakeServePlan()
    s.plans[key] = [p, nbytes, users]
    s.plan_bytes += nbytes
    return p


def test_serving_admission_evicts_idle_plans_lru_and_reserves():
    s = _bare_server(100)
    a = _add_plan(s, "a", 30, 0)     # least recently used
    b = _add_plan(s, "b", 30, 1)     # in use: never evicted
    c = _add_plan(s, "c", 30, 0)
    s._make_room(25)                 # 90 + 25 > 100: the idle LRU plan goes
    assert a.closed and not b.closed and not c.closed
    assert list(s.plans) == ["b", "c"] and s.plan_bytes == 60 and s.pending_bytes == 25
    s._make_room(30)                 # 60 + 25 + 30 > 100: the next idle plan goes
    assert c.closed and not b.closed and s.plan_bytes == 30 and s.pending_bytes == 55
    s._make_room(10)                 # 30 + 55 + 10 fits: nothing evicted
    assert list(s.plans) == ["b"] and s.pending_bytes == 65


def test_serving_admission_waits_for_plans_in_use():
    import threading
    import time
    s = _bare_server(100)
    b = _add_plan(s, "b", 50, 1)
    s.pending_bytes = 20.0
    t = threading.Thread(target=s._make_room, args=(40,), daemon=True)
    t.start()
    time.sleep(0.2)
    assert t.is_alive() and not b.closed          # 50 + 20 + 40 > 100 and b is in use
    with s.cv:
        s.plans["b"][2] = 0                        # the request using b completes
        s.cv.notify_all()
    t.join(timeout=5)
    assert not t.is_alive() and b.closed
    assert s.plan_bytes == 0 and s.pending_bytes == 60


# --------------------------------------------------------------------------------------
# batch planning under a device-memory budget (autotune.build_batch_plans) with fake plans
# --------------------------------------------------------------------------------------
class _FakeBatchPlan:
    """Plan tables of 64 bytes per coefficient; stored recurrence values of 8 bytes per
    recurrence step, which grow as N^2 (so stored values cost more per coefficient for
    larger N)."""
    made = []

    def __init__(self, N, alpha, beta, precision=0, directions=3, shared_workspace=False, **opts):
        self.N, self.opts, self.closed = int(N), dict(opts), False
        _FakeBatchPlan.made.append(self)

    def info(self):
        N, M = self.N, self.opts.get("M", 7)
        steps = int(0.05 * N * N / M)
        return {"fft_len_fwd": 2 * N, "fft_len_inv": 4 * N, "nfft_fwd": 1 + 2 * M, "nfft_inv": 1 + 2 * M,
                "rec_steps_fwd": steps, "rec_steps_inv": steps,
                "device_bytes": 64 * (N + 1) + (8 * steps if self.opts.get("rec_store") else 0)}

    def close(self):
        self.closed = True


def _plan_batch(monkeypatch, items, budget):
    from paper_1602_02618_gb300 import cjt
    monkeypatch.setattr(cjt, "Plan", _FakeBatchPlan)
    _FakeBatchPlan.made = []
    return autotune.build_batch_plans(items, plan_budget_bytes=budget)


def test_batch_plans_store_values_within_the_budget(monkeypatch):
    Ns = [100, 300, 1000, 3000, 10000, 30000, 70, 5000, 20000, 900]
    items = [(N, 0.1, -0.2, 1 if t % 2 else -1) for t, N in enumerate(Ns)]
    plain = sum(64 * (N + 1) for N in Ns)
    est = 1.25 * plain                         # the planner's reserve for the items to come

    plans, opts, rep = _plan_batch(monkeypatch, items, 1e15)
    assert all(o["rec_store"] == 1 for o in opts) and rep["stored_items"] == len(items)

    plans, opts, rep = _plan_batch(monkeypatch, items, plain)   # no room beyond the tables
    assert all(o["rec_store"] == 0 for o in opts) and rep["stored_items"] == 0
    assert [p.N for p in plans] == Ns and not any(p.closed for p in plans)

    budget = est + 8.0 * 0.05 * 3000 ** 2      # room for the stored values of a few small items
    plans, opts, rep = _plan_batch(monkeypatch, items, budget)
    stored = sorted(N for N, o in zip(Ns, opts) if o["rec_store"])
    assert 0 < len(stored) < len(items) and min(Ns) in stored and max(Ns) not in stored
    used = sum(p.info()["device_bytes"] for p in plans)
    assert used == rep["plan_bytes"] <= budget
    assert [p.N for p in plans] == Ns and not any(p.closed for p in plans)
    # every plan that was tried with stored values and did not fit was closed, not leaked
    kept = {id(p) for p in plans}
    assert all(p.closed for p in _FakeBatchPlan.made if id(p) not in kept)
    # segment length by size, as the grouped executor expects
    assert all(o["seg_len"] == (256 if N <= 16384 else 1024) for N, o in zip(Ns, opts))


def test_bench_oracle_errors_come_from_the_cpu_baseline_leg():
    """The batched form's error against the oracle is taken from the cpu_baseline leg's
    outputs of the items both ran (matched by N, parameters, direction and the input's
    digest); the form's kept GPU outputs never reach the JSON line."""
    import bench
    c1, c2 = np.arange(5.0), np.ones(9)
    it1, it2 = (4, 0.1, -0.2, 1, c1), (8, 0.3, 0.0, -1, c2)
    k1, k2 = bench.item_key(it1), bench.item_key(it2)
    assert k1 != bench.item_key((4, 0.1, -0.2, 1, c1 + 1.0)) and k1 != bench.item_key((4, 0.1, -0.2, -1, c1))
    ref1, ref2 = np.linspace(0, 1, 5), np.linspace(1, 2, 9)
    form = {"error": {"stated_bound": 1e-12},
            "_oracle_sample": {k1: (ref1 + 2e-3, float(np.abs(c1).sum())), k2: (ref2 - 9e-3, float(np.abs(c2).sum()))}}
    bench.oracle_errors(form, {k1: ref1, k2: ref2, ("other",): np.zeros(1)})
    assert "_oracle_sample" not in form
    assert form["error"]["items_checked"] == 2
    assert abs(form["error"]["max_abs_over_l1_vs_oracle"] - 1e-3) < 1e-12      # 9e-3 / 9 > 2e-3 / 10
    form = {"error": {}, "_oracle_sample": {k1: (ref1, 10.0)}}
    bench.oracle_errors(form, None)
    assert "_oracle_sample" not in form and "did not run" in form["error"]["vs_oracle"]
    form = {"error": {}, "_oracle_sample": {k1: (ref1, 10.0)}}
    bench.oracle_errors(form, {k2: ref2})
    assert "no item in common" in form["error"]["vs_oracle"]
    # the form picks its sample with the leg's own rule, so the same workload gives the same items
    items = bench.batch_items(64)
    assert [bench.item_key(it) for it in bench.batched_sample(items)] == \
        [bench.item_key(it) for it in bench.batched_sample(bench.batch_items(64))]


def test_bench_sample_outputs_match_the_legs_items():
    """The batched form keeps, at each sampled item's offset, exactly that item's output,
    under the keys of the cpu_baseline leg's own sample of the same workload."""
    import bench
    items = bench.batch_items(4096)
    offs, pos = [], 0
    for it in items:
        offs.append(pos)
        pos += it[0] + 1
    # a stand-in output: every item's own coefficients, so each slice identifies its item
    out = np.concatenate([it[4] for it in items])
    kept = bench.sample_outputs(items, offs, out)
    leg = bench.cpu_sample("batched")[0]
    assert list(kept) == [bench.item_key(it) for it in leg] and len(kept) > 10
    for it in leg:
        got, l1 = kept[bench.item_key(it)]
        assert np.array_equal(got, it[4]) and l1 == float(np.abs(it[4]).sum())


@pytest.mark.parametrize("config", ["all", "batched"])
def test_bench_main_line_carries_the_legs_oracle_error(monkeypatch, capsys, config):
    """bench.main with the GPU forms and the cpu_baseline leg replaced by fakes: the printed
    line carries the error against the leg's oracle outputs and none of the form's kept
    arrays."""
    import sys
    import torch
    import bench
    import __graft_entry__ as ge
    monkeypatch.setattr(ge, "build", lambda: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(bench, "Ctx", lambda *a, **k: object())
    for v in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(v, raising=False)
    key = (3, 0.1, -0.2, 1, "0" * 64)

    def form(value, kept=None):
        f = {"value": value, "unit": "coeffs/s", "ms_per_step": 1.0, "p50_ms": 1.0, "p99_ms": 1.0, "dtype": "f64",
             "workload": "w", "coefficients_per_step": 10, "plan_options": {}, "l2": "flushed",
             "error": {"stated_bound": 1e-12}, "roofline": {}, "e2e": {}, "gpu_launches": 1, "clocks": {}}
        if kept is not None:
            f["_oracle_sample"] = kept
        return f

    monkeypatch.setattr(bench, "run_batched", lambda ctx, big=False, steps=None:
                        form(2.0, None) if big else form(1.0, {key: (np.array([1.0, 2.0, 3.0, 4.0]), 4.0)}))
    monkeypatch.setattr(bench, "run_single", lambda ctx, precision_name=None: form(3.0))
    monkeypatch.setattr(bench, "run_serving", lambda ctx, precision_name: form(4.0))
    monkeypatch.setattr(bench, "cpu_baseline", lambda cfg, cores: ({"value": 5.0, "kind": "oracle", "cores": cores},
                                                                   {key: np.array([1.0, 2.2, 3.0, 4.0])}))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--config", config, "--steps", "3", "--warmup", "3"])
    bench.main()
    line = capsys.readouterr().out.strip().splitlines()[-1]
    assert "_oracle_sample" not in line
    d = json.loads(line)
    assert abs(d["error"]["max_abs_over_l1_vs_oracle"] - 0.05) < 1e-12 and d["error"]["items_checked"] == 1
    assert d["cpu_baseline"]["value"] == 5.0 and d["value"] == 1.0
    if config == "all":
        assert d["forms"]["batched_fp64"]["error"]["items_checked"] == 1
        assert "_oracle_sample" not in d["forms"]["batched_fp64"]


def test_bench_batch_work_counts_the_stated_units():
    """The roofline's algorithmic work, from plan summaries: 5 L log2 L per complex transform
    (the pairs of asymptotic items, plus one DCT-I / front-end transform per item), 8 flop per
    recurrence step at execution, 2 per stored value; points of all transforms for bytes."""
    import bench

    class P:
        def __init__(self, **kw):
            self.kw = kw

        def info(self):
            return self.kw

    fwd = P(fft_len_fwd=1024, nfft_fwd=4, rec_steps_fwd=1000, rec_store_bytes=8000,
            fft_len_inv=0, nfft_inv=0, rec_steps_inv=0)
    inv = P(fft_len_inv=2048, nfft_inv=1, rec_steps_inv=500, rec_store_bytes=0,
            fft_len_fwd=0, nfft_fwd=0, rec_steps_fwd=0)
    w = bench.batch_work([fwd, inv], [1, -1])
    assert w["fft_asy"] == 3 * 5.0 * 1024 * 10
    assert w["fft_dct"] == 5.0 * 1024 * 10 + 5.0 * 2048 * 11
    assert w["rec_stored"] == 2.0 * 1000 and w["rec"] == 8.0 * 500
    assert w["fft_points"] == 4 * 1024 + 1 * 2048


def test_tune_fft_keeps_the_fastest_configuration(monkeypatch):
    """tune_fft times every candidate of a length class, sets the fastest, reports the
    default's time, and restores the default when no candidate runs."""
    from paper_1602_02618_gb300 import cjt
    state = {}
    calls = []

    def set_config(prec, lg, ctas=4, split=0, single=12):
        state[(prec, lg)] = (ctas, split, single)
        calls.append((prec, lg, ctas, split, single))

    def fft_time(prec, lg, batch, reps):
        ctas, split, single = state[(prec, lg)]
        if lg == 20:
            raise cjt.CJTError(cjt.CJT_ENOMEM, "fft_time")
        return 1.0 + 0.1 * abs(ctas - 2) + 0.05 * split + (0.3 if single == 13 else 0.0)

    monkeypatch.setattr(cjt, "fft_set_config", set_config)
    monkeypatch.setattr(cjt, "fft_time", fft_time)
    out = autotune.tune_fft(0, [14, 13, 14, 20], points=1 << 20)
    assert sorted(out) == [13, 14]                       # 20: every candidate failed
    for lg in (13, 14):
        assert out[lg]["config"] == (2, 0, 12) and state[(0, lg)] == (2, 0, 12)
        assert abs(out[lg]["default_ms"] - 1.2) < 1e-12 and out[lg]["batch"] == max(1, (1 << 20) >> lg)
        assert len([c for c in calls if c[1] == lg]) == len(autotune.fft_candidates(lg)) + 1
    assert calls[-1] == (0, 20, 4, 0, 12)                # the default put back


def test_serving_submit_refuses_malformed_requests():
    """Requests whose coefficients are not N+1 long, or whose direction is unknown, are
    refused at submit and never reach the executor's queue; a good one is queued."""
    import queue
    from paper_1602_02618_gb300 import cjt, serve
    s = _bare_server(1e9)
    s.incoming = queue.Queue()
    s._next_id = 0
    for bad in (serve.Request(100, 0.1, 0.2, cjt.CJT_FWD, np.ones(100)),
                serve.Request(100, 0.1, 0.2, cjt.CJT_FWD, np.ones((101, 1))),
                serve.Request(100, 0.1, 0.2, 3, np.ones(101)),
                serve.Request(-1, 0.1, 0.2, cjt.CJT_INV, np.ones(0))):
        with pytest.raises(ValueError):
            s.submit(bad)
    assert s.incoming.empty()
    good = s.submit(serve.Request(100, 0.1, 0.2, cjt.CJT_INV, np.ones(101)))
    assert s.incoming.get_nowait() is good and good.rid == 0
