"""Plan autotuner: picks the number of Hahn terms M, the recurrence work
split (degree-segment length) and whether the recurrence values are stored in
the plan (rec_store) for a given N and precision by timing candidate plans on
the current GPU (forward + inverse, CUDA events), and caches the choice in a
JSON file.

Every candidate computes the same transform to within the stated tolerance
(the partition only moves work between the asymptotic blocks and the
recurrence, Sec. 2.2); only the time differs.  On GB300 the FP64 pipe is the
bottleneck of both parts, so the balance point differs from the paper's
CPU setting.
"""
from __future__ import annotations

import json
import os
import threading

CANDIDATES_M = (7, 10, 13, 16)
CANDIDATES_SEG = (256, 1024)


def candidates(N: int, max_store_bytes: float):
    """Options to time: the recurrence at execution over M and the segment length; the
    stored recurrence values over M, the segment length and a coarser block ratio (fewer
    transforms, more recurrence); and no asymptotic blocks at all when the stored matrix
    (8 (N+1)^2 bytes per direction) fits the memory cap."""
    out = []
    for M in CANDIDATES_M:
        for seg in CANDIDATES_SEG:
            out.append({"M": M, "seg_len": seg, "rec_store": 0})
    for M in (5, 7, 10, 13, 16):
        for seg in CANDIDATES_SEG:
            out.append({"M": M, "seg_len": seg, "rec_store": 1})
        out.append({"M": M, "seg_len": 1024, "rec_store": 1, "ratio": 0.05})
    if 3 * 8.0 * (N + 1) ** 2 <= max_store_bytes:
        out.append({"M": 7, "seg_len": 1024, "rec_store": 1, "use_asy": -1})
    return out


_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("CJT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cjt_gb300_autotune.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _key(N, precision, directions):
    import torch
    return "%s|N=%d|prec=%d|dir=%d" % (torch.cuda.get_device_name(), N, precision, directions)


def time_plan(plan, x, y, reps=3):
    """Average milliseconds of forward + inverse (CUDA events on the current stream)."""
    import torch
    from . import cjt
    info = plan.info()
    def run():
        if info["directions"] & cjt.CJT_FWD:
            cjt.cjt_forward(plan, x, y)
        if info["directions"] & cjt.CJT_INV:
            cjt.cjt_inverse(plan, x, y)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def best_options(N: int, alpha: float, beta: float, precision: int = 0, directions: int = 3,
                 refresh: bool = False) -> dict:
    """Options dict for cjt.Plan (M, seg_len, rec_store, ratio, use_asy), from the cache or by
    timing the candidates."""
    import numpy as np
    import torch
    from . import cjt
    if N < 256:
        return {"M": 7, "seg_len": 256}
    key = _key(N, precision, directions)
    with _lock:
        cache = _load()
        if not refresh and key in cache:
            return dict(cache[key]["options"])
    rng = np.random.default_rng(N)
    x = torch.from_numpy(rng.standard_normal(N + 1) / np.arange(1, N + 2)).cuda()
    y = torch.empty_like(x)
    max_store = float(os.environ.get("CJT_AUTOTUNE_MAX_STORE_GB", "40")) * 1e9
    results = []
    for opts in candidates(N, max_store):
        try:
            p = cjt.Plan(N, alpha, beta, precision=precision, directions=directions, **opts)
        except cjt.CJTError:
            continue
        if opts.get("rec_store") and p.info()["rec_store_bytes"] > max_store:
            p.close()
            continue
        results.append((time_plan(p, x, y), opts))
        p.close()
    if not results:
        raise RuntimeError("no candidate plan could be built for N=%d, alpha=%g, beta=%g" % (N, alpha, beta))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    with _lock:
        cache = _load()
        cache[key] = {"options": best, "ms": results[0][0],
                      "candidates": [{"options": o, "ms": t} for t, o in results]}
        _save(cache)
    return dict(best)


# ---------------------------------------------------------------------------
# Batches: options per size class under a device-memory budget
# ---------------------------------------------------------------------------
# Measured fractions of the FP64 pipe peak of the grouped stage kernels (grouped batch,
# serialised launches on GB300): recurrence at execution, stored values, transforms.
ETA_REC, ETA_STORED, ETA_FFT = 0.75, 0.85, 0.82
# The mixed form runs the asymptotic blocks' transforms on the FP32 pipe (64 times the FP64
# rate on GB300, but the transforms then wait on memory and latency): they are modelled at a
# tenth of their FP64 cost; its final DCT-I / inverse front end stay FP64.
MIXED_ASY_FFT_FACTOR = 0.1
BATCH_CANDIDATES = [{"M": M, "ratio": r} for M in (7, 10, 13, 16) for r in (0.0, 0.1, 0.05)]


def _work_model(info, direction, precision=0):
    """Modelled FP64-pipe seconds-at-peak factors of one execution: (recurrence steps,
    transform flop / ETA_FFT), from a plan's summary."""
    import math
    from . import cjt
    f = direction == 1
    L = info["fft_len_fwd"] if f else info["fft_len_inv"]
    nfft = info["nfft_fwd"] if f else info["nfft_inv"]
    steps = info["rec_steps_fwd"] if f else info["rec_steps_inv"]
    lg = max(math.log2(max(L, 2)), 1.0)
    asy = max(nfft - 1, 0) * (MIXED_ASY_FFT_FACTOR if precision == cjt.CJT_MIXED else 1.0)
    return float(steps), (asy + 1.0) * 5.0 * L * lg / ETA_FFT


def batch_class_options(items, precision: int = 0, samples: int = 2, seed: int = 0):
    """Per size class (floor log2 N) of a batch: the fastest candidate (M, block ratio) with
    the recurrence at execution and with stored values, by the modelled FP64-pipe work of
    `samples` planned items of the class (8 flop per recurrence step at ETA_REC, 2 flop per
    stored value at ETA_STORED, the transforms at ETA_FFT), and the measured plan-table
    bytes per coefficient of the first.  Returns {class: dict}."""
    import math
    import numpy as np
    from . import cjt
    classes = {}
    for t, it in enumerate(items):
        classes.setdefault(int(math.floor(math.log2(max(it[0], 1)))), []).append(t)
    rng = np.random.default_rng(seed)
    out = {}
    for k, members in sorted(classes.items()):
        pick = [members[i] for i in rng.choice(len(members), min(samples, len(members)), replace=False)]
        res = []
        for opts in BATCH_CANDIDATES:
            t_rec = t_sto = tab = n1 = 0.0
            ok = True
            for t in pick:
                N, a, b, d = items[t][:4]
                try:
                    p = cjt.Plan(N, a, b, precision=precision, directions=1 if d == 1 else 2,
                                 shared_workspace=True, **opts)
                except cjt.CJTError:
                    ok = False
                    break
                inf = p.info()
                p.close()
                steps, fft = _work_model(inf, d, precision)
                t_rec += 8.0 * steps / ETA_REC + fft
                t_sto += 2.0 * steps / ETA_STORED + fft
                tab += inf["device_bytes"]
                n1 += N + 1.0
            if ok:
                res.append((opts, t_rec / n1, t_sto / n1, tab / n1))
        if res:
            plain = min(res, key=lambda r: r[1])
            store = min(res, key=lambda r: r[2])
            out[k] = {"plain": dict(plain[0]), "store": dict(store[0]), "cost_plain": plain[1],
                      "cost_store": store[2], "store_better": store[2] < plain[1],
                      "table_bytes_per_coeff": max(plain[3], store[3]), "members": members}
    return out


def build_batch_plans(items, precision: int = 0, plan_budget_bytes: float = 200e9, samples: int = 2,
                      seed: int = 0):
    """Plans for every item of a batch (shared workspace, for the grouped executor), with the
    options of batch_class_options.  Items are planned in increasing N.  An item of a class
    whose stored-values option models faster gets stored recurrence values while the plans
    built so far, its own stored values and the modelled tables of the items still to come
    (1.25 x the sampled bytes per coefficient) fit plan_budget_bytes; every other item is
    planned with the recurrence at execution.  The time saved per stored byte is the same for
    every item (6 flop per 8 bytes), so the smaller items, which need fewer bytes per
    coefficient, come first.  Returns (plans in item order, options, report)."""
    import math
    from . import cjt
    cls = batch_class_options(items, precision, samples, seed)
    order = sorted(range(len(items)), key=lambda t: items[t][0])
    klass = [int(math.floor(math.log2(max(it[0], 1)))) for it in items]
    remaining = sum(1.25 * cls[klass[t]]["table_bytes_per_coeff"] * (items[t][0] + 1.0) for t in order
                    if klass[t] in cls)
    used = 0.0
    plans, opts = [None] * len(items), [None] * len(items)
    stored = 0
    for t in order:
        N, a, b, d = items[t][:4]
        c = cls.get(klass[t])
        est = 1.25 * c["table_bytes_per_coeff"] * (N + 1.0) if c else 0.0
        remaining -= est
        o = None
        p = None
        if c and c["store_better"]:
            o = dict(c["store"], seg_len=256 if N <= 16384 else 1024, rec_store=1)
            p = cjt.Plan(N, a, b, precision=precision, directions=1 if d == 1 else 2, shared_workspace=True, **o)
            if used + p.info()["device_bytes"] + remaining > plan_budget_bytes:
                p.close()
                p = None
            else:
                stored += 1
        if p is None:
            o = dict(c["plain"] if c else {}, seg_len=256 if N <= 16384 else 1024, rec_store=0)
            p = cjt.Plan(N, a, b, precision=precision, directions=1 if d == 1 else 2, shared_workspace=True, **o)
        used += p.info()["device_bytes"]
        plans[t], opts[t] = p, o
    report = {"classes": {str(k): {"plain": v["plain"], "store": v["store"], "store_better": v["store_better"],
                                   "stored_items": sum(1 for t in v["members"] if opts[t]["rec_store"]),
                                   "items": len(v["members"])} for k, v in cls.items()},
              "plan_bytes": used, "plan_budget_bytes": plan_budget_bytes, "stored_items": stored}
    return plans, opts, report


# ---------------------------------------------------------------------------
# Transforms: launch configuration per (precision, length)
# ---------------------------------------------------------------------------
FFT_CTAS = (2, 4, 8)


def fft_candidates(log2L: int):
    """(ctas_per_sm, split, single_max_log2) worth timing for transforms of length 2^log2L:
    the tile occupancy target always; the four-step splits above one pass (split 2, the
    narrower first pass, from 2^14); one pass or two at 2^13."""
    out = []
    for ctas in FFT_CTAS:
        if log2L <= 12:
            out.append((ctas, 0, 12))
        elif log2L == 13:
            out += [(ctas, 0, 12), (ctas, 1, 12), (ctas, 0, 13)]
        else:
            out += [(ctas, 0, 12), (ctas, 1, 12), (ctas, 2, 12)]
    return out


def tune_fft(precision: int, log2Ls, points: int = 1 << 24, reps: int = 3) -> dict:
    """For each length 2^log2L, time the candidates of fft_candidates on a batch of about
    `points` points (cjt_fft_time) and keep the fastest with cjt_fft_set_config.  Returns
    {log2L: {"config": (ctas_per_sm, split, single_max_log2), "ms": best, "default_ms": ...}}."""
    from . import cjt
    out = {}
    for lg in sorted(set(int(v) for v in log2Ls)):
        batch = max(1, points >> lg)
        res = []
        for ctas, split, single in fft_candidates(lg):
            cjt.fft_set_config(precision, lg, ctas, split, single)
            try:
                res.append((cjt.fft_time(precision, lg, batch, reps), (ctas, split, single)))
            except cjt.CJTError:
                continue
        if not res:
            cjt.fft_set_config(precision, lg)
            continue
        best = min(res)
        default = [t for t, c in res if c == (4, 0, 12)]
        cjt.fft_set_config(precision, lg, *best[1])
        out[lg] = {"config": best[1], "ms": best[0], "default_ms": default[0] if default else None, "batch": batch}
    return out
