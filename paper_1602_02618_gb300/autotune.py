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
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    with _lock:
        cache = _load()
        cache[key] = {"options": best, "ms": results[0][0],
                      "candidates": [{"options": o, "ms": t} for t, o in results]}
        _save(cache)
    return dict(best)
