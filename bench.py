#!/usr/bin/env python
"""Benchmark of the Chebyshev--Jacobi transform library on GB300.

Default (`--config all`): one JSON line whose `value` is the batched FP64 form, with the
other forms beside it under `forms`:

* batched_fp64 (the line's value): 4096 transforms per step, N log-uniform in
  [64, 65536] (integers, mostly not powers of two), (alpha, beta) ~ U[-0.45, 0.45]^2 and a
  random direction per transform, c_n = g_n/(n+1); one replay of a captured CUDA graph per
  step (grouped execution: one launch per stage and transform length class).
  `per_call_same_items` runs the same 4096 transforms one call per transform.
* plain_fp64: forward + inverse, one transform per call, of N in {2^12, 2^14, 2^16, 2^18}
  with their own (alpha, beta) and c_n = g_n/(n+1)^1.5; options autotuned per N.
* mixed64: 64 transforms at N = 2^20 in the mixed form (FP32 transforms), one graph
  replay per step; error against the FP64 GPU form and the oracle fixtures, and the
  plans' stated bounds.
* serving: Poisson arrivals at swept rates, N log-uniform in [128, 2^18], continuous
  batching with device-resident plans and a 40 GB budget; p50/p99 latency and coeffs/s,
  in the FP64 and the mixed form.

Plans are built (and autotuned) before the timed regions; inputs are resident in HBM when
they start.  The L2 cache is flushed (a 512 MiB write) between timed steps, outside the
timed events.  `--impl reference` times the CPU oracle (rank 0 only) on a bounded sample
of the same workload.  Under torchrun every rank runs its own seeded shard of the same
shape (rank 0: the one-GPU workload), with no collective on the data path; `value` is the
coefficients of all ranks over the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transform coeffs/sec (batched, mixed-precision vs plain FP64) at stated error; p50/p99"
LOGNS = (12, 14, 16, 18)
FP64_PEAK_DERIVED = 152 * 2070e6 * 4.0   # 152 SMs x 2.07 GHz x 2 FP64 FMA/clk/SM (1.2586 TFLOP/s)
P64_SOURCE = "derived FP64 pipe peak: 152 SMs x 2.07 GHz x 2 DFMA/clk/SM"
GOLDEN = os.path.join(ROOT, "tests", "golden")


def workload(rank=0):
    """Rank `rank`'s single-transform items (rank 0: the one-GPU workload)."""
    from paper_1602_02618_gb300 import inputs, multirank
    return inputs.single_workload(Ns=tuple(1 << k for k in LOGNS),
                                  seed=multirank.rank_seed(inputs.BASE_SEED, rank))


def batch_items(count, rank=0):
    from paper_1602_02618_gb300 import inputs, multirank
    return inputs.batch_workload(count, seed=multirank.rank_seed(inputs.BASE_SEED, rank))


PREC_NAMES = {"fp64": "FP64", "mixed": "mixed (FP32 ASY transforms)",
              "df": "double-float (f32x2 ASY transforms and stored recurrence, FP64 error bound)"}
DTYPES = {"fp64": "f64", "mixed": "f32 ASY transforms + f64",
          "df": "f32x2 double-float ASY transforms and stored recurrence + f64"}


def precision_code(cjt, name):
    return {"fp64": cjt.CJT_FP64, "mixed": cjt.CJT_MIXED, "df": cjt.CJT_DFLOAT}[name]


def default_grid(N):
    """The Lobatto grid a plan takes by default: the least G >= N of the forms 2^a, 3 2^a,
    5 2^a."""
    best = None
    for q in (1, 3, 5):
        g = q
        while g < N:
            g <<= 1
        best = g if best is None else min(best, g)
    return best


def lg2(v):
    return max(math.log2(max(v, 2)), 1.0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": float(np.median(power)) if power else None}


# ---------------------------------------------------------------------------
# CPU oracle samples (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_seconds_estimate(N, d):
    """Rough double-double oracle seconds of one item on 8 cores (measured at N = 4096:
    forward 0.09 s, inverse 0.29 s; O(N^2))."""
    return (N / 4096.0) ** 2 * (0.09 if d == 1 else 0.29) + 1e-3


def batched_sample_indices(items, budget_s=1.2):
    """Indices of the batch's transforms, in order, that fit about `budget_s` of oracle time
    on 8 cores (each item's estimate within what is left of the budget; the large items are
    skipped)."""
    out, t = [], 0.0
    for i, (N, a, b, d, c) in enumerate(items):
        e = oracle_seconds_estimate(N, d)
        if t + e > budget_s:
            continue
        out.append(i)
        t += e
        if budget_s - t < 0.01:
            break
    return out


def batched_sample(items, budget_s=1.2):
    """The items of batched_sample_indices, as (N, alpha, beta, direction, coefficients)."""
    return [tuple(items[i][:5]) for i in batched_sample_indices(items, budget_s)]


def sample_outputs(items, offs, out):
    """{item_key: (output, ||c_in||_1)} of the batch's items that the cpu_baseline leg's
    sampling rule picks, read from the batch's output array at the items' offsets."""
    kept = {}
    for i in batched_sample_indices(items):
        N, c = items[i][0], items[i][4]
        kept[item_key(items[i])] = (np.array(out[offs[i]:offs[i] + N + 1]), float(np.abs(c).sum()))
    return kept


def time_oracle_items(forward, inverse, items, nthreads):
    t0 = time.perf_counter()
    outs = [forward(c, a, b, nthreads=nthreads) if d == 1 else inverse(c, a, b, nthreads=nthreads)
            for N, a, b, d, c in items]
    return time.perf_counter() - t0, outs


def single_sample_items():
    """The single-transform workload's items the oracle runs in full: forward and inverse at
    N = 2^12 and 2^14, forward at 2^16 (the 2^16 inverse and the 2^18 items take minutes)."""
    out = []
    for N, a, b, c in workload():
        if N <= (1 << 14):
            out.append((N, a, b, 1, c))
            out.append((N, a, b, -1, c))
        elif N == (1 << 16):
            out.append((N, a, b, 1, c))
    return out


def cpu_sample(config):
    """(items, description) of the bounded oracle sample of a configuration's workload."""
    if config == "single":
        return single_sample_items(), ("forward and inverse at N = 2^12 and 2^14 and forward at 2^16 of the "
                                      "single-transform workload, in full")
    items = batch_sample_items()
    return items, ("%d transforms (N from %d to %d, %d coefficients) of the 4096-transform batch, the first in "
                   "order that fit the sample's time, in full"
                   % (len(items), min(it[0] for it in items), max(it[0] for it in items),
                      sum(it[0] + 1 for it in items)))


def batch_sample_items():
    return batched_sample(batch_items(4096))


def item_key(it):
    """Identity of a transform item (N, alpha, beta, direction, coefficients' digest)."""
    import hashlib
    N, a, b, d, c = it[:5]
    return (int(N), float(a), float(b), int(d), hashlib.sha256(np.ascontiguousarray(c).tobytes()).hexdigest())


def cpu_baseline(config, cores):
    """The cpu_baseline leg: the oracle as it stands (double-double) on the bounded sample, on
    all host cores, and the plain-double O(N^2) routines on all cores and on one core.
    Returns (the baseline's dict, {item_key: the oracle's output} of the sample's items); the
    outputs also serve the GPU forms' error against the oracle (oracle_errors)."""
    from oracle import oracle as orc
    orc.build()
    items, desc = cpu_sample(config)
    coeffs = sum(it[0] + 1 for it in items)
    t, outs = time_oracle_items(orc.forward, orc.inverse, items, cores)
    t64, _ = time_oracle_items(orc.forward_f64, orc.inverse_f64, items, cores)
    t64_1, _ = time_oracle_items(orc.forward_f64, orc.inverse_f64, items, 1)
    base = {"value": coeffs / t, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
            "sample": "oracle (double-double, O(N^2)): %s; %.1f s" % (desc, t),
            "fp64_naive": {"value_all_cores": coeffs / t64, "value_1_core": coeffs / t64_1, "unit": "coeffs/s",
                           "cores": cores, "sample": "plain-double O(N^2) forward/inverse, same sample"}}
    return base, {item_key(it): np.asarray(y) for it, y in zip(items, outs)}


def oracle_errors(form, oracle_out):
    """Fill the form's error against the oracle from the cpu_baseline leg's outputs: max
    |c_gpu - c_oracle| / ||c_in||_1 over the sample's items that the form also ran (the GPU
    outputs the form kept in "_oracle_sample"), then drop the kept outputs."""
    kept = form.pop("_oracle_sample", None)
    if kept is None:
        return
    err = form.setdefault("error", {})
    if oracle_out is None:
        err["vs_oracle"] = "not computed: the cpu_baseline leg did not run"
        return
    common = [k for k in kept if k in oracle_out]
    if not common:
        err["vs_oracle"] = "not computed: no item in common with the cpu_baseline leg's sample"
        return
    errs = [float(np.abs(kept[k][0] - oracle_out[k]).max() / kept[k][1]) for k in common]
    err["max_abs_over_l1_vs_oracle"] = max(errs)
    err["items_checked"] = len(common)
    err["vs_oracle"] = ("the cpu_baseline leg's double-double oracle outputs of %d items (N from %d to %d)"
                        % (len(common), min(k[0] for k in common), max(k[0] for k in common)))


def run_reference(args):
    """The CPU oracle on the host cores, each step a bounded sample of the workload of
    `--config` (default: the batched workload, the line's headline)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    config = "single" if args.config == "single" else "batched"
    items, desc = cpu_sample(config)
    coeffs = sum(it[0] + 1 for it in items)
    # every host core, whatever OMP_NUM_THREADS says (torchrun sets it to 1 for N > 1)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        time_oracle_items(orc.forward, orc.inverse, items, cores)
    times = [time_oracle_items(orc.forward, orc.inverse, items, cores)[0] for _ in range(args.steps)]
    total = float(np.sum(times))
    value = coeffs * len(times) / total
    t64, _ = time_oracle_items(orc.forward_f64, orc.inverse_f64, items, cores)
    t64_1, _ = time_oracle_items(orc.forward_f64, orc.inverse_f64, items, 1)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "coeffs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (double-double)",
        "data": "synthetic",
        "config": {"workload": BATCH_DESC % "FP64" if config == "batched" else single_desc("fp64"),
                   "sample": desc},
        "cpu_baseline": {"value": value, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
                         "sample": "oracle (double-double, O(N^2)): " + desc,
                         "fp64_naive": {"value_all_cores": coeffs / t64, "value_1_core": coeffs / t64_1,
                                        "unit": "coeffs/s", "cores": cores,
                                        "sample": "plain-double O(N^2) forward/inverse, same sample"}},
        "e2e": {"value": value, "unit": "coeffs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# GPU forms
# ---------------------------------------------------------------------------
BATCH_DESC = ("batched: 4096 transforms per step, N log-uniform in [64, 65536], alpha,beta~U[-0.45,0.45] "
              "each, random forward/inverse, c_n=g_n/(n+1); %s; one captured CUDA graph per step (grouped "
              "execution: one launch per stage and transform length class)")


def single_desc(precision, params=""):
    ab = ("(alpha,beta)=(%s) for every transform" % params) if params else \
        "alpha,beta~U[-0.45,0.45] per transform"
    return ("forward+inverse CJT singly, %s, N in {2^12,2^14,2^16,2^18}, %s, c_n=g_n/(n+1)^1.5, g~N(0,1)"
            % (PREC_NAMES[precision], ab))


class Ctx:
    def __init__(self, args, torch, cjt, dev, world, rank, dist):
        self.args, self.torch, self.cjt, self.dev = args, torch, cjt, dev
        self.world, self.rank, self.dist = world, rank, dist
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.local = int(os.environ.get("LOCAL_RANK", "0"))

    def events(self, n):
        t = self.torch
        return [(t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)) for _ in range(n)]


def batch_plan_options(N, big, precision, cjt):
    """Fixed plan options of the batched workloads (--batch-fixed; otherwise
    autotune.build_batch_plans chooses).  Batch of 4096: M = 13 and block ratio 0.1; stored
    recurrence values up to N = 16384.  Large mixed batch: M = 16, segment length 1024."""
    if big:
        return {"M": 16, "seg_len": 1024}
    o = {"M": 13, "seg_len": 256, "ratio": 0.1}
    if N <= 16384:
        o["rec_store"] = 1
    return o


# DRAM traffic of one replay of the 4096-item FP64 batch, summed over its transform launches
# (k_fft_sub, k_fft_rq) in the one-pass ncu capture summarised in
# profiles/traffic_batched_fp64_4096.md.  It stands for the code it was taken on: while the
# transform kernels' and the grouped executor's sources hash to the digests below.
FFT_TRAFFIC = {
    "read": 114.990e9, "write": 90.675e9, "bytes_per_step": 205.664e9, "plan_budget_gb": 260.0,
    "profile": "profiles/traffic_batched_fp64_4096.md",
    "sources": {"paper_1602_02618_gb300/csrc/cjt_fft.cu":
                "c6caedc1d33a40905e296ef093376fdfed8582969fe9c12e5381c585fa410e82",
                "paper_1602_02618_gb300/csrc/cjt_group.cu":
                "b6cca996de421e246f1361fb3eff42c54c6de599949f3175fa067cd808f93725"},
}


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return None


def measured_fft_traffic(args, precision, cjt):
    """FFT_TRAFFIC when this run is the captured workload on the captured code, else None."""
    import hashlib
    if (args.batch_count != 4096 or precision != cjt.CJT_FP64 or args.batch_fixed
            or args.batch_plan_gb != FFT_TRAFFIC["plan_budget_gb"]):
        return None
    for rel, digest in FFT_TRAFFIC["sources"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return FFT_TRAFFIC


def batch_work(plans, dirs):
    """Algorithmic FP64-pipe work of one batch replay per stage kind (flop) from the plans:
    transforms 5 L log2 L per complex transform of length L (2.5 L log2 L per real item);
    recurrence at execution 8 flop per step; stored values 2 flop (one multiply-add)."""
    w = {"fft_asy": 0.0, "fft_dct": 0.0, "rec": 0.0, "rec_stored": 0.0}
    points = 0.0   # complex points of all transforms (for their algorithmic bytes)
    for p, d in zip(plans, dirs):
        inf = p.info()
        f = d == 1
        L = inf["fft_len_fwd"] if f else inf["fft_len_inv"]
        npair = (inf["nfft_fwd"] if f else inf["nfft_inv"]) - 1
        steps = inf["rec_steps_fwd"] if f else inf["rec_steps_inv"]
        w["fft_asy"] += npair * 5.0 * L * lg2(L)
        w["fft_dct"] += 5.0 * L * lg2(L)
        points += (npair + 1) * L
        if inf["rec_store_bytes"] > 0:
            w["rec_stored"] += 2.0 * steps
        else:
            w["rec"] += 8.0 * steps
    w["fft_points"] = points
    return w


def oracle_fixture(name):
    path = os.path.join(GOLDEN, "oracle_%s.npz" % name)
    return np.load(path) if os.path.exists(path) else None


def run_batched(ctx, big=False, steps=None):
    """The batched FP64 form (4096 transforms) or, big=True, the large mixed batch
    (64 x N = 2^20).  Returns the form's dict."""
    args, torch, cjt, dev = ctx.args, ctx.torch, ctx.cjt, ctx.dev
    from paper_1602_02618_gb300 import inputs, multirank
    seed = multirank.rank_seed(inputs.BASE_SEED, ctx.rank)
    steps = steps or args.steps
    if big:
        items = inputs.mixed_large_workload(64, 1 << 20, seed=seed)
        precision = cjt.CJT_DFLOAT if args.precision == "df" else cjt.CJT_MIXED
    else:
        items = inputs.batch_workload(args.batch_count, seed=seed)
        precision = precision_code(cjt, args.precision)
    # transform launch configuration: tuned per length class the batch uses (process-wide,
    # before the graph is captured)
    fft_tune = None
    if not args.no_autotune:
        from paper_1602_02618_gb300 import autotune
        t0 = time.perf_counter()
        # the power-of-two transform lengths the plans run: 2G and 4G, or their power-of-two
        # factors when G = 3 2^a or 5 2^a (the default grid: the least of 2^a, 3 2^a, 5 2^a >= N)
        lens = set()
        for N, *_ in items:
            G = default_grid(N)
            q = 3 if G % 3 == 0 else 5 if G % 5 == 0 else 1
            for L in (2 * G, 4 * G):
                lens.add(int(math.log2(L // q)))
        lens = sorted(lens)
        fft_tune = {"precision": args.precision if not big else "mixed",
                    "lengths": autotune.tune_fft(precision, lens), "tune_s": None}
        if precision != cjt.CJT_FP64:   # the DCT-I and the front end stay in FP64
            fft_tune["fp64_lengths"] = autotune.tune_fft(cjt.CJT_FP64, lens)
        fft_tune["tune_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    tune = None
    if args.batch_fixed:
        plans = []
        for N, a, b, d, c in items:
            plans.append(cjt.Plan(N, a, b, precision=precision, directions=cjt.CJT_FWD if d == 1 else cjt.CJT_INV,
                                  shared_workspace=True, **batch_plan_options(N, big, precision, cjt)))
    else:
        from paper_1602_02618_gb300 import autotune
        # the plans may take the budget, within the device memory free now less 20 GB for the
        # arenas (about 9 GB), the I/O buffers, the per-call comparison and the runtime
        free, _ = torch.cuda.mem_get_info(dev)
        budget = min(args.batch_plan_gb * 1e9, free - 20e9)
        plans, _, tune = autotune.build_batch_plans(items, precision, plan_budget_bytes=budget)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    dirs = [1 if d == 1 else 2 for _, _, _, d, _ in items]
    offs, pos = [], 0
    for N, *_ in items:
        offs.append(pos)
        pos += N + 1
    coeffs = pos
    host_in = torch.from_numpy(np.concatenate([it[4] for it in items])).pin_memory()
    x = host_in.to(dev)
    out = torch.empty_like(x)
    t0 = time.perf_counter()
    batch = cjt.Batch(plans, dirs, offs, x, out, nstreams=args.lanes)
    graph_s = time.perf_counter() - t0
    binfo = batch.info()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.launch()
    torch.cuda.synchronize()
    multirank.barrier(ctx.dist)
    sampler = ClockSampler(ctx.local).start()
    time.sleep(0.3)
    evs = ctx.events(steps)
    for k in range(steps):
        ctx.flush.zero_()
        evs[k][0].record(stream)
        torch.cuda.nvtx.range_push("timed_batch")
        batch.launch()
        torch.cuda.nvtx.range_pop()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    multirank.barrier(ctx.dist)
    clocks = sampler.stop()
    step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    total_s = multirank.max_over_ranks(float(step_ms.sum()) / 1e3, ctx.dist, dev)
    coeffs_all = multirank.sum_over_ranks(coeffs, ctx.dist, dev)
    value = multirank.job_rate(coeffs_all * steps, total_s)
    o = out.cpu().numpy()

    # stage kinds timed alone (profiled replays after the timed region: the same launches
    # issued directly, one after another on one stream, with an event pair around each)
    batch.set_profiling(True)
    batch.profile()
    nprof = 2
    for _ in range(nprof):
        ctx.flush.zero_()
        batch.launch()
    torch.cuda.synchronize()
    prof = batch.profile()
    batch.set_profiling(False)
    work = batch_work(plans, dirs)
    live = {k: prof[k][0] / nprof for k in prof if prof[k][1]}
    step_s = total_s / steps
    peak = FP64_PEAK_DERIVED
    if precision != cjt.CJT_FP64:
        asy_peak = cjt.microbench_fma(0 if precision == cjt.CJT_MIXED else 2)
    else:
        asy_peak = peak
    t_peak = {"fft_asy": work["fft_asy"] / asy_peak, "fft_dct": work["fft_dct"] / peak,
              "rec": work["rec"] / peak, "rec_stored": work["rec_stored"] / peak}
    dom = max(live, key=lambda k: live[k])
    roof = {"kernel": {"fft_asy": "k_fft_sub (grouped asymptotic-block transforms)",
                       "fft_dct": "k_fft_sub (grouped final DCT-I / front end)",
                       "rec": "k_g_rec_fwd / k_g_rec_inv (recurrences at execution)",
                       "rec_stored": "k_g_rec_fwd_stored / k_g_rec_inv_stored"}.get(dom, dom),
            "stage": dom, "bound": "alu", "unit": "TFLOP/s", "traffic": None,
            "serialised_ms_per_step": live, "time_share": live[dom] / sum(live.values()), "work_tflop_per_step": {k: v / 1e12 for k, v in work.items() if k != "fft_points"}}
    if dom in t_peak and live[dom] > 0:
        pk = asy_peak if dom == "fft_asy" else peak
        ach = (t_peak[dom] * pk) / (live[dom] * 1e-3)
        roof.update({"achieved": ach / 1e12, "peak": pk / 1e12, "frac": ach / pk,
                     "peak_source": P64_SOURCE if pk == peak else "measured multiply-add rate of the ASY form"})
    # DRAM traffic of the transform launches, from the one-pass capture of this workload
    tr = measured_fft_traffic(args, precision, cjt)
    if tr is not None:
        tsec = 1e-3 * (live.get("fft_asy", 0.0) + live.get("fft_dct", 0.0))
        roof["traffic"] = tr["bytes_per_step"]
        roof["traffic_detail"] = {
            "kernels": "all transform launches of one replay (k_fft_sub, k_fft_rq; asymptotic blocks, DCT-I and "
                       "front end together): dram__bytes_read.sum + dram__bytes_write.sum",
            "read": tr["read"], "write": tr["write"], "profile": tr["profile"],
            "algorithmic_bytes": 32.0 * work["fft_points"],
            "note": "algorithmic bytes: every complex point read once and written once (16 B each way)",
            "traffic_over_algorithmic": tr["bytes_per_step"] / (32.0 * work["fft_points"]),
            "achieved_gbs": tr["bytes_per_step"] / tsec / 1e9 if tsec > 0 else None,
            "hbm_gbs": measured_hbm_gbs()}
    roof["step"] = {"frac": sum(t_peak.values()) / step_s, "ms_at_peak": 1e3 * sum(t_peak.values()),
                    "ms_per_step": 1e3 * step_s,
                    "note": "all stage kinds at their pipe's peak, summed (they share the FP64 pipe)"}

    # accuracy: the mixed batch against the stored oracle fixtures (tests/golden); the FP64
    # batch keeps its outputs of the cpu_baseline leg's sample items, compared with the
    # oracle's by oracle_errors once that leg has run
    err = {}
    kept = None
    if big:
        err64 = []
        for (N, a, b, d, c), off in zip(items, offs):      # every item of the batch
            p64 = cjt.Plan(N, a, b, M=16, seg_len=1024, directions=cjt.CJT_FWD if d == 1 else cjt.CJT_INV)
            xt = torch.from_numpy(c).to(dev)
            ref = (cjt.cjt_forward(p64, xt) if d == 1 else cjt.cjt_inverse(p64, xt)).cpu().numpy()
            p64.close()
            err64.append(float(np.abs(o[off:off + N + 1] - ref).max() / np.abs(c).sum()))
        err["vs_fp64_gpu_max_abs_over_l1"] = max(err64)
        err["vs_fp64_gpu_items"] = len(err64)
        for t in (0, 1):
            N, a, b, d, c = items[t]
            fx = oracle_fixture(("fwd_N%d" if d == 1 else "inv_N%d") % N) if ctx.rank == 0 else None
            got = o[offs[t]:offs[t] + N + 1]
            dirn = cjt.CJT_FWD if d == 1 else cjt.CJT_INV
            key = "forward" if d == 1 else "inverse"
            err["stated_bound_" + key] = cjt.error_bound(plans[t], dirn)
            if fx is not None and str(fx["input_sha256"]) == item_key(items[t])[4]:   # same input
                err["vs_oracle_%s_max_abs_over_l1" % key] = float(
                    np.abs(got[fx["idx"]] - fx["out"]).max() / np.abs(c).sum())
                err["oracle_%s" % key] = "%s, %d sampled coefficients" % (str(fx["oracle"]), fx["idx"].size)
    else:
        kept = sample_outputs(items, offs, o)
        err = {"stated_bound": max(cjt.error_bound(p, d) for p, d in zip(plans, dirs))}

    # end to end through the C ABI: pinned host input -> device -> replay -> host output
    host_out = torch.empty_like(host_in).pin_memory()
    ksteps = max(3, min(steps, 10))
    batch.launch_host(host_in.numpy(), host_out.numpy())
    multirank.barrier(ctx.dist)
    t0 = time.perf_counter()
    for _ in range(ksteps):
        batch.launch_host(host_in.numpy(), host_out.numpy())
    e2e_s = multirank.max_over_ranks(time.perf_counter() - t0, ctx.dist, dev)

    form = {
        "value": value, "unit": "coeffs/s", "steps": steps, "warmup": args.warmup,
        "ms_per_step": float(step_ms.mean()), "p50_ms": float(np.percentile(step_ms, 50)),
        "p99_ms": float(np.percentile(step_ms, 99)),
        "dtype": DTYPES["df" if precision == cjt.CJT_DFLOAT else ("mixed" if precision == cjt.CJT_MIXED else "fp64")],
        "workload": ("64 transforms at N=2^20, alpha,beta~U[-0.45,0.45] each, forward/inverse alternating, "
                     "c_n=g_n/(n+1); %s ASY transforms, FP64 recurrences, scalings and accumulation; one captured "
                     "CUDA graph per step" % ("double-float" if precision == cjt.CJT_DFLOAT else "FP32"))
        if big else BATCH_DESC % PREC_NAMES[args.precision],
        "coefficients_per_step": coeffs,
        "plan_options": (
            ("M=16, seg_len=1024" if big else "M=13, seg_len=256, ratio=0.1, rec_store for N <= 16384")
            if args.batch_fixed else
            {"autotuner": "autotune.build_batch_plans: per size class (M, ratio) by the modelled FP64-pipe work "
                          "of candidate plans; stored recurrence values in increasing N while the plans fit %.0f GB"
                          % ((tune["plan_budget_bytes"] if tune else 0) / 1e9), "classes": tune["classes"] if tune else None,
             "stored_items": tune["stored_items"] if tune else None}),
        "l2": "inputs (%.0f MB) exceed L2; flushed between steps" % (coeffs * 8 / 1e6),
        "error": err, "roofline": roof,
        "e2e": {"value": multirank.job_rate(coeffs_all * ksteps, e2e_s), "unit": "coeffs/s",
                "h2d_bytes_per_step": coeffs * 8, "d2h_bytes_per_step": coeffs * 8,
                "via": "cjt_batch_launch_host (C ABI, pinned host buffers)"},
        "kernels_per_step": int(binfo["kernels"]), "gpu_launches": int(binfo["kernels"]) * steps,
        "fft_autotune": fft_tune,
        "setup": {"plan_s": plan_s, "graph_create_s": graph_s,
                  "plan_bytes": sum(p.info()["device_bytes"] for p in plans),
                  "rec_store_bytes": sum(p.info()["rec_store_bytes"] for p in plans),
                  "arena_bytes": binfo["arena_bytes"]},
        "clocks": clocks,
    }
    if kept is not None:
        form["_oracle_sample"] = kept

    if not big:
        # the same transforms one call per transform (the plain form on this workload)
        ws = torch.empty(max(p.info()["workspace_bytes"] for p in plans) // 8 + 64, dtype=torch.float64, device=dev)
        y = torch.empty_like(x)

        def per_call():
            for p, (N, a, b, d, c), off in zip(plans, items, offs):
                xi, yi = x[off:off + N + 1], y[off:off + N + 1]
                (cjt.cjt_forward_ws if d == 1 else cjt.cjt_inverse_ws)(p, xi, yi, ws)

        per_call()
        torch.cuda.synchronize()
        pc = []
        for _ in range(3):
            ctx.flush.zero_()
            e0, e1 = ctx.events(1)[0]
            e0.record(stream)
            per_call()
            e1.record(stream)
            torch.cuda.synchronize()
            pc.append(e0.elapsed_time(e1))
        same = bool(torch.equal(y, out))
        pc_s = multirank.max_over_ranks(float(np.median(pc)) / 1e3, ctx.dist, dev)
        form["per_call_same_items"] = {
            "value": multirank.job_rate(coeffs_all, pc_s), "unit": "coeffs/s", "ms_per_step": 1e3 * pc_s,
            "steps": 3, "bit_identical_to_batched": same,
            "note": "the same 4096 transforms, one cjt_forward_ws / cjt_inverse_ws call each on one stream"}
        form["batched_over_per_call"] = value / form["per_call_same_items"]["value"]
    batch.close()
    for p in plans:
        p.close()
    torch.cuda.empty_cache()
    return form


def run_single(ctx, precision_name=None):
    """The plain form: forward + inverse of each single-transform item, one call each."""
    args, torch, cjt, dev = ctx.args, ctx.torch, ctx.cjt, ctx.dev
    from paper_1602_02618_gb300 import autotune, multirank
    precision_name = precision_name or args.precision
    precision = precision_code(cjt, precision_name)
    items = workload(ctx.rank)
    if args.only_logn:
        items = [it for it in items if it[0] == (1 << args.only_logn)]
    if args.params:
        pa, pb = (float(v) for v in args.params.split(","))
        items = [(N, pa, pb, c) for N, _, _, c in items]
    expansion = {"auto": cjt.CJT_EXPANSION_AUTO, "hahn": cjt.CJT_EXPANSION_HAHN,
                 "ultra": cjt.CJT_EXPANSION_ULTRASPHERICAL}[args.expansion]
    fixed = {}
    for kv in filter(None, args.fixed_options.split(",")):
        k, v = kv.split("=")
        fixed[k.strip()] = float(v) if k.strip() in ("ratio", "eps") else int(v)
    plans, xs, ys, zs, ws, chosen = [], [], [], [], [], []
    for N, a, b, c in items:
        opts = dict(fixed) if (fixed or args.no_autotune) else autotune.best_options(N, a, b, precision)
        if expansion != cjt.CJT_EXPANSION_AUTO:
            opts["expansion"] = expansion
        plans.append(cjt.Plan(N, a, b, precision=precision, **opts))
        chosen.append(opts)
        xs.append(torch.from_numpy(c).to(dev))
        ys.append(torch.empty_like(xs[-1]))
        zs.append(torch.empty_like(xs[-1]))
        ws.append(torch.empty_like(xs[-1]))
    coeffs_per_step = 2 * sum(N + 1 for N, _, _, _ in items)
    stream = torch.cuda.current_stream()

    def step():
        for p, x, y, z in zip(plans, xs, ys, zs):
            cjt.cjt_forward(p, x, y)
            cjt.cjt_inverse(p, y, z)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    multirank.barrier(ctx.dist)
    torch.cuda.synchronize()
    sampler = ClockSampler(ctx.local).start()
    time.sleep(0.3)
    evs = ctx.events(args.steps)
    for k in range(args.steps):
        ctx.flush.zero_()
        evs[k][0].record(stream)
        torch.cuda.nvtx.range_push("timed")
        step()
        torch.cuda.nvtx.range_pop()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    multirank.barrier(ctx.dist)
    clocks = sampler.stop()
    step_ms = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
    total_s = multirank.max_over_ranks(float(step_ms.sum()) / 1e3, ctx.dist, dev)
    coeffs_all = multirank.sum_over_ranks(coeffs_per_step, ctx.dist, dev)
    value = multirank.job_rate(coeffs_all * args.steps, total_s)

    # stage times: profiled steps after the timed region, each stage timed alone by an event
    # pair on the launching stream (profiled executions run their two chains one after the
    # other); per step
    prof = {}
    launches = 0
    infos = [p.info() for p in plans]
    nprof = 2
    for p in plans:
        p.set_profiling(True)
        p.profile()
    for _ in range(nprof):
        ctx.flush.zero_()
        step()
    torch.cuda.synchronize()
    for p, inf in zip(plans, infos):
        for st, (ms, cnt) in p.profile().items():
            a = prof.setdefault(st, [0.0, 0])
            a[0] += ms / nprof
            a[1] += cnt
        launches += (inf["kernels_fwd"] + inf["kernels_inv"]) * args.steps
    for p in plans:
        p.set_profiling(False)
    # Roofline per stage.  Algorithmic work of one plan per step, and the peak it is held to:
    #   recurrence at execution: 8 flop per step (sum_i J(i)), FP64 pipe;
    #   stored recurrence values (rec_store): one multiply-add per value, 2 flop on the FP64
    #   pipe, or, in the double-float form, 8 bytes read per value against HBM bandwidth;
    #   asymptotic blocks: 2.5 L log2 L flop per (block, m) item, L = 2G forward, 4G inverse,
    #   on the FP64 pipe, the FP32 pipe (mixed form) or at the measured double-float rate;
    #   final DCT-I / inverse front end: 5 L log2 L flop (one complex transform), FP64 pipe.
    try:
        fp64_meas = cjt.microbench_fma(1)
    except Exception:
        fp64_meas = None
    try:
        fp32_meas = cjt.microbench_fma(0)
    except Exception:
        fp32_meas = None
    try:
        df_meas = cjt.microbench_fma(2) if precision == cjt.CJT_DFLOAT else None
    except Exception:
        df_meas = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_gbs, hbm_src = float(json.load(f)["hbm_gbs"]), "measured HBM copy bandwidth (MEASURED_PEAKS.json)"
    except Exception:
        hbm_gbs, hbm_src = 6800.0, "fallback HBM bandwidth 6.8 TB/s"
    P64 = ("alu", "TFLOP/s", FP64_PEAK_DERIVED, P64_SOURCE)
    P32 = ("alu", "TFLOP/s", fp32_meas or 77e12, "measured FP32 FMA rate (cjt_microbench_fma)")
    PDF = ("alu", "TFLOP/s", df_meas or 4.5e12, "measured double-float multiply-add rate (cjt_microbench_fma kind 2)")
    PHBM = ("hbm", "GB/s", hbm_gbs * 1e9, hbm_src)
    ideal = {k: 0.0 for k in cjt.STAGES}
    model = {}
    for inf, opt in zip(infos, chosen):
        store = opt.get("rec_store", 0)
        Lf, Li, M = inf["fft_len_fwd"], inf["fft_len_inv"], inf["M"]
        work = {}
        for st, steps_ in (("fwd_rec", inf["rec_steps_fwd"]), ("inv_rec", inf["rec_steps_inv"])):
            if store and precision == cjt.CJT_DFLOAT:
                work[st] = (8.0 * steps_, PHBM)
            else:
                work[st] = ((2.0 if store else 8.0) * steps_, P64)
        asy = PDF if precision == cjt.CJT_DFLOAT else (P32 if precision == cjt.CJT_MIXED else P64)
        work["fwd_fft"] = (inf["nblk_fwd"] * M * 2.5 * Lf * lg2(Lf), asy)
        work["inv_fft"] = (inf["nblk_inv"] * M * 2.5 * Li * lg2(Li), asy)
        work["fwd_dct"] = (5.0 * Lf * lg2(Lf), P64)
        work["inv_front"] = (5.0 * Li * lg2(Li), P64)
        for st, (w, pk) in work.items():
            ideal[st] += w / pk[2]
            if w > 0:
                model[st] = pk
    # The dominant stage is the one with the largest (serialised) time.
    measured = [st for st in prof if prof[st][0] > 0 and ideal.get(st, 0.0) > 0]
    dom = max(measured, key=lambda st: prof[st][0]) if measured else None
    kernel_of = {"fwd_rec": "k_rec_fwd_stored(_df) / k_rec_fwd", "inv_rec": "k_rec_inv_stored(_df) / k_rec_inv",
                 "fwd_fft": "k_fft_sub (forward ASY transforms)", "inv_fft": "k_fft_sub (transposed ASY transforms)",
                 "fwd_dct": "k_fft_sub (final DCT-I)", "inv_front": "k_fft_sub (front end)"}

    def frac_of(st):
        t = prof.get(st, (0.0, 0))[0] * 1e-3
        return ideal[st] / t if t > 0 and ideal[st] > 0 else None
    roof = {"kernel": kernel_of.get(dom, dom), "stage": dom, "traffic": None,
            "time_share": prof[dom][0] / sum(v[0] for v in prof.values()) if dom else None,
            "fp64_fma_measured_tflops": fp64_meas / 1e12 if fp64_meas else None,
            "fp32_fma_measured_tflops": fp32_meas / 1e12 if fp32_meas else None,
            "df_fma_measured_tflops": df_meas / 1e12 if df_meas else None}
    f = frac_of(dom) if dom else None
    if f is not None and dom in model:
        bound, unit, pk, src = model[dom]
        scale = 1e9 if unit == "GB/s" else 1e12
        roof.update({"bound": bound, "unit": unit, "peak": pk / scale, "achieved": f * pk / scale, "frac": f,
                     "peak_source": src})
    roof["stages_frac_of_peak"] = {k: frac_of(k) for k in cjt.STAGES if frac_of(k) is not None}
    by_res = {}
    for st, pk in model.items():
        by_res[pk[3]] = by_res.get(pk[3], 0.0) + ideal[st]
    step_s = total_s / args.steps
    if by_res and step_s > 0:
        res, t_res = max(by_res.items(), key=lambda kv: kv[1])
        roof["step"] = {"frac": t_res / step_s, "bound_ms": 1e3 * t_res, "ms_per_step": 1e3 * step_s,
                        "bound_by": res}

    # accuracy: the round trip of one step, and each transform against the oracle's outputs
    # stored in tests/golden (written by tests/golden/make_fullsize.py, for these very inputs)
    err = {"round_trip_max_abs_over_l1": max(float((z - x).abs().max()) / float(x.abs().sum())
                                              for x, z in zip(xs, zs))}
    if ctx.rank == 0 and not args.params:
        import hashlib
        vs = {}
        for (N, a, b, c), p, x in zip(items, plans, xs):
            dg = hashlib.sha256(np.ascontiguousarray(c).tobytes()).hexdigest()
            inv_of_c = cjt.cjt_inverse(p, x).cpu().numpy()
            fwd_of_c = cjt.cjt_forward(p, x).cpu().numpy()
            for name, got in (("forward", fwd_of_c), ("inverse", inv_of_c)):
                fx = oracle_fixture(("fwd_N%d" if name == "forward" else "inv_N%d") % N)
                if fx is None or str(fx["input_sha256"]) != dg:
                    continue                    # no stored oracle output for this input
                vs["%s_N%d" % (name, N)] = float(np.abs(got - fx["out"]).max() / np.abs(c).sum())
        err["max_abs_over_l1_vs_oracle"] = vs
        err["stated_bound"] = max(cjt.error_bound(p, cjt.CJT_INV) for p in plans)

    # end to end through the C ABI from pinned host memory
    hx = [torch.from_numpy(c).pin_memory() for _, _, _, c in items]
    hy = [torch.empty_like(h).pin_memory() for h in hx]
    hz = [torch.empty_like(h).pin_memory() for h in hx]

    def e2e_step():
        for p, xh, yh, zh in zip(plans, hx, hy, hz):
            cjt.cjt_execute_host(p, cjt.CJT_FWD, xh.numpy(), yh.numpy())
            cjt.cjt_execute_host(p, cjt.CJT_INV, yh.numpy(), zh.numpy())
    ksteps = max(3, min(args.steps, 20))
    e2e_step()
    multirank.barrier(ctx.dist)
    t0 = time.perf_counter()
    for _ in range(ksteps):
        e2e_step()
    e2e_s = multirank.max_over_ranks(time.perf_counter() - t0, ctx.dist, dev)
    bytes_io = 2 * sum(8 * (N + 1) for N, _, _, _ in items)
    form = {
        "value": value, "unit": "coeffs/s", "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(step_ms.mean()), "p50_ms": float(np.percentile(step_ms, 50)),
        "p99_ms": float(np.percentile(step_ms, 99)), "dtype": DTYPES[precision_name],
        "workload": single_desc(precision_name, args.params), "N": [it[0] for it in items],
        "options": chosen, "l2": "flushed between steps (512 MiB write, outside timed events)",
        "plans": [{"plan_ms": round(inf["plan_ms"], 2), "device_bytes": inf["device_bytes"],
                   "rec_store_bytes": inf["rec_store_bytes"], "workspace_bytes": inf["workspace_bytes"]}
                  for inf in infos],
        "error": err, "stages_ms_per_step_serialised": {k: v[0] for k, v in prof.items() if v[1]},
        "roofline": roof,
        "e2e": {"value": multirank.job_rate(coeffs_all * ksteps, e2e_s), "unit": "coeffs/s",
                "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
                "via": "cjt_execute_host (C ABI, pinned host buffers)"},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    for p in plans:
        p.close()
    torch.cuda.empty_cache()
    return form


def run_serving(ctx, precision_name):
    """Poisson arrivals at swept rates, continuous batching, 40 GB budget."""
    args, torch, cjt, dev = ctx.args, ctx.torch, ctx.cjt, ctx.dev
    from paper_1602_02618_gb300 import inputs, multirank, serve
    precision = precision_code(cjt, precision_name)
    rates = [float(r) for r in args.rates.split(",")]
    results = []
    for k, rate in enumerate(rates):
        reqs = [serve.Request(N, a, b, cjt.CJT_FWD if d == 1 else cjt.CJT_INV, c)
                for N, a, b, d, c in inputs.serving_requests(
                    args.requests, seed=multirank.rank_seed(inputs.BASE_SEED, ctx.rank) + 100 * k)]
        sampler = ClockSampler(ctx.local).start()
        server = serve.Server(slots=args.slots, mem_budget=40e9, precision=precision, planners=args.planners)
        serve.poisson_run(server, reqs, rate=rate, seed=k)
        st = server.stats()
        server.close()
        st["rate_req_per_s"] = rate
        st["errors"] = sum(1 for r in reqs if r.error)
        st["clocks"] = sampler.stop()
        st["coeffs_per_s"] = multirank.sum_over_ranks(st["coeffs_per_s"], ctx.dist, dev)
        results.append(st)
        torch.cuda.empty_cache()
    kbest = int(np.argmax([r["coeffs_per_s"] for r in results]))
    best = results[kbest]
    return {"value": best["coeffs_per_s"], "unit": "coeffs/s", "requests_per_rate": args.requests,
            "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "dtype": DTYPES[precision_name],
            "workload": "serving: Poisson arrivals, %d requests per rate, N log-uniform in [128, 2^18], "
                        "alpha,beta~U[-0.45,0.45], random direction, c_n=g_n/(n+1); plan built per request "
                        "(device-resident, reused on repeats); %d slots, 40 GB budget" % (args.requests, args.slots),
            "per_rate": results}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "df"], default="fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--fixed-options", default="", help="e.g. M=13,seg_len=1024 (applied to every N; no autotune)")
    ap.add_argument("--only-logn", type=int, default=0, help="profile runs: one size of the single workload only")
    ap.add_argument("--config", choices=["all", "single", "batched", "mixed64", "serving"], default="all")
    ap.add_argument("--rates", default="50,200,800,3200")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--planners", type=int, default=8)
    ap.add_argument("--slots", type=int, default=16, help="serving: concurrent requests on the device")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--lanes", type=int, default=16)
    ap.add_argument("--batch-plan-gb", type=float, default=260.0,
                    help="device memory the batched workload's plans may take (autotuned options)")
    ap.add_argument("--batch-fixed", action="store_true",
                    help="batched workload with fixed options (M=13, ratio=0.1, stored values for N <= 16384)")
    ap.add_argument("--params", default="",
                    help="fixed (alpha, beta) for every transform of the single workload, e.g. 0,0 (Legendre)")
    ap.add_argument("--expansion", choices=["auto", "hahn", "ultra"], default="auto",
                    help="asymptotic formula of the plans (ultra: App. B.1, needs alpha = beta)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_1602_02618_gb300 import multirank
    world, rank, local = multirank.env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt
    ctx = Ctx(args, torch, cjt, dev, world, rank, dist)
    cores = os.cpu_count() or 1
    common = {"metric": METRIC, "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "data": "synthetic"}

    if args.config == "all":
        forms = {}
        forms["batched_fp64"] = run_batched(ctx)
        forms["plain_fp64"] = run_single(ctx, "fp64")
        forms["mixed64"] = run_batched(ctx, big=True, steps=min(args.steps, 5))
        forms["serving_fp64"] = run_serving(ctx, "fp64")
        forms["serving_mixed"] = run_serving(ctx, "mixed")
        head = forms["batched_fp64"]
        for k in ("plain_fp64", "mixed64", "serving_fp64", "serving_mixed"):
            forms[k]["ratio_to_batched_fp64"] = forms[k]["value"] / head["value"]
        out = dict(common)
        out.update({"value": head["value"], "unit": "coeffs/s", "steps": args.steps, "warmup": args.warmup,
                    "ms_per_step": head["ms_per_step"], "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
                    "dtype": head["dtype"],
                    "config": {"workload": head["workload"], "coefficients_per_step": head["coefficients_per_step"],
                               "plan_options": head["plan_options"], "l2": head["l2"],
                               "parallelism": ("%d independent shards (one per rank, no collective on the data "
                                               "path)" % world) if world > 1 else "single GPU"},
                    "error": head["error"], "roofline": head["roofline"], "e2e": head["e2e"],
                    "gpu_launches": head["gpu_launches"], "clocks": head["clocks"], "forms": forms})
        oracle_out = None
        if rank == 0 and not args.no_cpu_baseline:
            out["cpu_baseline"], oracle_out = cpu_baseline("batched", cores)
        elif rank == 0:
            out["cpu_baseline"] = None
        oracle_errors(forms["batched_fp64"], oracle_out)
        out["error"] = forms["batched_fp64"]["error"]
        if rank == 0:
            print(json.dumps(out))
    else:
        if args.config == "single":
            f = run_single(ctx)
        elif args.config == "batched":
            f = run_batched(ctx)
        elif args.config == "mixed64":
            f = run_batched(ctx, big=True)
        else:
            f = run_serving(ctx, args.precision)
        out = dict(common)
        out.update({k: v for k, v in f.items() if k not in ("workload",)})
        out["config"] = {"workload": f["workload"]}
        out.setdefault("steps", args.steps)
        out.setdefault("warmup", args.warmup)
        oracle_out = None
        if rank == 0 and args.config in ("single", "batched") and not args.no_cpu_baseline:
            out["cpu_baseline"], oracle_out = cpu_baseline(args.config, cores)
        oracle_errors(f, oracle_out)
        out.pop("_oracle_sample", None)
        out["error"] = f.get("error")
        if rank == 0:
            print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
