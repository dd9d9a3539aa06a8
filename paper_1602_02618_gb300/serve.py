"""Continuous-batching request loop for Chebyshev--Jacobi transforms (one GPU).

Requests (N, alpha, beta, direction, coefficients on the host) arrive at any
time.  Planner threads build each request's plan as soon as it arrives (plans
stay device-resident, keyed by (N, alpha, beta, precision, direction), and are
reused by later requests with the same key).  The executor admits planned
requests into free slots -- one CUDA stream, one workspace arena and one pair of
device/pinned I/O buffers per slot -- as soon as a slot and the memory budget
allow, so requests that arrive while others run overlap with them on the
device.  Completion is detected by a CUDA event per slot; the latency of a
request runs from its arrival to its result being on the host.

Every transform runs in the library's kernels through the C ABI
(cjt_plan, cjt_forward_ws / cjt_inverse_ws); this module only schedules.
Admission by memory: before a planner builds a new plan, plans not in use are
evicted least-recently-used until the resident plans, the slot arenas and I/O
buffers, the estimates of the plans other planners are building and the new
plan's estimate fit in `mem_budget`; the estimate stays reserved until the plan is
registered (or its build fails); while plans in use fill the budget, the planner
waits for them to be released.  Slot arenas grow to the largest
workspace their slot has served; they count against the budget but are not
gated themselves (at most slots x the largest workspace).
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import cjt


@dataclass
class Request:
    N: int
    alpha: float
    beta: float
    direction: int          # cjt.CJT_FWD or cjt.CJT_INV
    x: np.ndarray           # N+1 coefficients (host)
    rid: int = 0
    t_arrival: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    out: np.ndarray = None
    done: threading.Event = field(default_factory=threading.Event)
    error: str = ""


class _Slot:
    def __init__(self, torch, dev):
        self.torch = torch
        self.stream = torch.cuda.Stream(device=dev)
        self.event = torch.cuda.Event()
        self.arena = None
        self.arena_bytes = 0
        self.io_cap = 0
        self.d_in = self.d_out = self.h_in = self.h_out = None
        self.req = None
        self.plan_key = None

    def ensure(self, ws_bytes, n, dev):
        t = self.torch
        grown = 0
        if ws_bytes > self.arena_bytes:
            grown += ws_bytes - self.arena_bytes
            self.arena = t.empty(max(ws_bytes, 256), dtype=t.uint8, device=dev)
            self.arena_bytes = ws_bytes
        if n > self.io_cap:
            grown += 16 * (n - self.io_cap)
            self.d_in = t.empty(n, dtype=t.float64, device=dev)
            self.d_out = t.empty(n, dtype=t.float64, device=dev)
            self.h_in = t.empty(n, dtype=t.float64).pin_memory()
            self.h_out = t.empty(n, dtype=t.float64).pin_memory()
            self.io_cap = n
        return grown


class Server:
    def __init__(self, slots: int = 16, mem_budget: float = 40e9, precision: int = cjt.CJT_FP64,
                 planners: int = 4, plan_options=None, device: int = 0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.precision = precision
        self.mem_budget = float(mem_budget)
        # one-shot plans: rows whose recurrence spans at most 8192 degrees run as one item, so
        # the plan computes no segment states for them (planning bounds the loop's throughput)
        self.plan_options = plan_options or (lambda N: {"M": 13 if N >= 16384 else 10, "seg_len": 256,
                                                        "seg_whole": 8192})
        self.slots = [_Slot(torch, self.dev) for _ in range(slots)]
        self.incoming = queue.Queue()
        self.ready = collections.deque()
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.plans = collections.OrderedDict()   # key -> [Plan, bytes, users]
        self.plan_bytes = 0
        self.slot_bytes = 0
        self.pending_bytes = 0.0   # estimates of the plans being built
        self.completed = []
        self.max_inflight = 0
        self._stop = False
        self._next_id = 0
        self.threads = [threading.Thread(target=self._planner, daemon=True) for _ in range(planners)]
        self.threads.append(threading.Thread(target=self._executor, daemon=True))
        for th in self.threads:
            th.start()

    # ---------------------------------------------------------------- public
    def submit(self, req: Request) -> Request:
        """Queue a request; a malformed one (coefficients not of length N+1, an unknown
        direction) raises ValueError here instead of reaching the executor."""
        if req.direction not in (cjt.CJT_FWD, cjt.CJT_INV):
            raise ValueError("direction must be CJT_FWD or CJT_INV")
        if int(req.N) < 0 or np.shape(req.x) != (int(req.N) + 1,):
            raise ValueError("x must hold N+1 = %d coefficients, got shape %s" % (int(req.N) + 1, np.shape(req.x)))
        with self.lock:
            req.rid = self._next_id
            self._next_id += 1
        req.t_arrival = time.perf_counter()
        self.incoming.put(req)
        return req

    def close(self):
        self._stop = True
        for _ in self.threads:
            self.incoming.put(None)
        with self.cv:
            self.cv.notify_all()
        for th in self.threads:
            th.join(timeout=30)
        # requests still queued or planned get an error instead of waiting for ever
        left = list(self.ready)
        self.ready.clear()
        while True:
            try:
                r = self.incoming.get_nowait()
            except queue.Empty:
                break
            if r is not None:
                left.append(r)
        for r in left:
            self._fail(r, "server closed before the request ran")
        with self.lock:
            for p, _, _ in self.plans.values():
                p.close()
            self.plans.clear()

    @staticmethod
    def _fail(r, msg):
        r.error = msg
        r.t_done = time.perf_counter()
        r.done.set()

    def stats(self):
        lat = np.array([r.t_done - r.t_arrival for r in self.completed])
        if not len(lat):
            return {}
        t0 = min(r.t_arrival for r in self.completed)
        t1 = max(r.t_done for r in self.completed)
        coeffs = sum(r.N + 1 for r in self.completed)
        return {"requests": len(lat), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
                "coeffs_per_s": coeffs / (t1 - t0), "wall_s": t1 - t0, "max_inflight": self.max_inflight,
                "resident_plan_bytes": self.plan_bytes, "slot_bytes": self.slot_bytes}

    # --------------------------------------------------------------- planner
    def _key(self, r):
        return (r.N, r.alpha, r.beta, self.precision, r.direction)

    def _planner(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        # plan kernels are small and each plan waits for them several times (its partition
        # and work lists come back to the host): the highest priority lets them take SMs as
        # the executing transforms' CTAs retire instead of queueing behind them
        stream = torch.cuda.Stream(device=self.dev, priority=-100)
        while not self._stop:
            r = self.incoming.get()
            if r is None:
                return
            key = self._key(r)
            try:
                with self.lock:
                    ent = self.plans.get(key)
                    if ent is not None:
                        ent[2] += 1
                        self.plans.move_to_end(key)
                if ent is None:
                    est = 4000.0 * (r.N + 1)   # conservative device bytes of one plan's tables
                    self._make_room(est)       # reserves est as pending bytes
                    try:
                        p = cjt.Plan(r.N, r.alpha, r.beta, precision=self.precision, directions=r.direction,
                                     shared_workspace=True, stream=stream.cuda_stream, **self.plan_options(r.N))
                    except Exception:
                        with self.cv:
                            self.pending_bytes -= est
                            self.cv.notify_all()
                        raise
                    nbytes = p.info()["device_bytes"]
                    with self.cv:
                        self.pending_bytes -= est
                        if key in self.plans:           # another planner made it meanwhile
                            self.plans[key][2] += 1
                            p.close()
                        else:
                            self.plans[key] = [p, nbytes, 1]
                            self.plan_bytes += nbytes
                        self.cv.notify_all()
            except Exception as e:  # bad request: report it on the request, keep serving
                self._fail(r, str(e))
                continue
            with self.cv:
                self.ready.append(r)
                self.cv.notify_all()

    def _make_room(self, need):
        """Evict unused plans until the resident plans, the slots, the plans being built by
        other planners (their reserved estimates) and `need` fit the budget, then reserve
        `need` as pending bytes until the caller registers its plan."""
        with self.cv:
            while (self.plan_bytes + self.slot_bytes + self.pending_bytes + need > self.mem_budget
                   and not self._stop):
                victim = next((k for k, v in self.plans.items() if v[2] == 0), None)
                if victim is None:
                    self.cv.wait(timeout=0.05)
                    continue
                p, nbytes, _ = self.plans.pop(victim)
                p.close()
                self.plan_bytes -= nbytes
            self.pending_bytes += need

    # -------------------------------------------------------------- executor
    def _executor(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        busy = []
        while not (self._stop and not busy):
            progressed = False
            # retire finished work
            for s in list(busy):
                if s.event.query():
                    r = s.req
                    r.out = s.h_out[: r.N + 1].numpy().copy()
                    r.t_done = time.perf_counter()
                    with self.cv:
                        self.plans[s.plan_key][2] -= 1
                        self.completed.append(r)
                        self.cv.notify_all()
                    s.req = None
                    busy.remove(s)
                    r.done.set()
                    progressed = True
            # admit ready requests into free slots
            free = [s for s in self.slots if s.req is None]
            while free:
                with self.cv:
                    if not self.ready:
                        break
                    r = self.ready.popleft()
                    key = self._key(r)
                    plan = self.plans[key][0]
                s = free.pop()
                n = r.N + 1
                try:
                    grown = s.ensure(plan.info()["workspace_bytes"], n, self.dev)
                    with self.cv:
                        self.slot_bytes += grown
                    r.t_admit = time.perf_counter()
                    s.h_in[:n].copy_(torch.from_numpy(np.ascontiguousarray(r.x, dtype=np.float64)))
                    with torch.cuda.stream(s.stream):
                        s.d_in[:n].copy_(s.h_in[:n], non_blocking=True)
                        fn = cjt.cjt_forward_ws if r.direction == cjt.CJT_FWD else cjt.cjt_inverse_ws
                        fn(plan, s.d_in, s.d_out, s.arena, stream=s.stream)
                        s.h_out[:n].copy_(s.d_out[:n], non_blocking=True)
                        s.event.record(s.stream)
                except Exception as e:   # the request fails; the slot and the loop go on
                    s.stream.synchronize()
                    with self.cv:
                        self.plans[key][2] -= 1
                        self.cv.notify_all()
                    self._fail(r, str(e))
                    free.append(s)
                    progressed = True
                    continue
                s.req, s.plan_key = r, key
                busy.append(s)
                self.max_inflight = max(self.max_inflight, len(busy))
                progressed = True
            if not progressed:
                with self.cv:
                    if not self.ready or not any(s.req is None for s in self.slots):
                        self.cv.wait(timeout=0.0005)


def poisson_run(server: Server, requests, rate: float, seed: int = 0):
    """Submit `requests` with exponential inter-arrival times of mean 1/rate; wait for all."""
    rng = np.random.default_rng(seed)
    t = time.perf_counter()
    for r in requests:
        t += rng.exponential(1.0 / rate)
        delay = t - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        server.submit(r)
    for r in requests:
        r.done.wait()
    return requests
