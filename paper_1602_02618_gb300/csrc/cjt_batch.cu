// Batched execution: many transforms (any mix of N, (alpha, beta), precision and
// direction) issued over a set of concurrent streams, and the same sequence
// captured once into a CUDA graph so that a whole batch is one graph launch.
//
// Items are assigned longest-first to the lane (stream) with the least
// estimated work.  Each lane has a workspace arena sized for the largest
// shared-workspace item it runs; items on one lane run in order, so they can
// share the lane's arena.  The lanes fork from the caller's stream with an
// event and join back with one event per lane.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <numeric>
#include <vector>

#include "cjt_group.cuh"
#include "cjt_internal.cuh"

namespace {

// estimated FP64 work of one execution (the recurrence steps and transform points)
double item_cost(const cjt_plan_s *p, int dir) {
    const double N = (double)p->N;
    if (dir == CJT_FWD) {
        const Dft &d = p->dft_f;
        double L = (double)d.fft_len();
        return 4.0 * (double)p->fw.rec_steps + 3.5 * p->npair_f * L * std::log2(std::max(L, 2.0)) * (d.P ? 2.0 : 1.0) +
               40.0 * N;
    }
    const Dft &d = p->dft_i;
    double L = (double)d.fft_len();
    return 5.0 * (double)p->iv.rec_steps + 3.5 * p->npair_i * L * std::log2(std::max(L, 2.0)) * (d.P ? 2.0 : 1.0) +
           80.0 * N;
}

struct Assignment {
    std::vector<int> lane;            // lane of each item
    std::vector<std::vector<int>> order;  // items per lane, longest first
    std::vector<int64_t> need;        // arena bytes per lane
};

Assignment assign(int count, const cjt_plan_t *plans, const int8_t *dir, int nlanes) {
    Assignment a;
    std::vector<double> cost(count);
    for (int t = 0; t < count; ++t) cost[t] = item_cost(plans[t], dir[t]);
    std::vector<int> idx(count);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<double> load(nlanes, 0.0);
    a.lane.assign(count, 0);
    a.order.assign(nlanes, {});
    a.need.assign(nlanes, 0);
    for (int t : idx) {
        int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += cost[t];
        a.lane[t] = l;
        a.order[l].push_back(t);
        if (plans[t]->shared_ws) a.need[l] = std::max(a.need[l], plans[t]->ws_bytes);
    }
    return a;
}

struct Lanes {
    int dev = -1;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};

int make_lanes(Lanes &L, int n) {
    CJT_CUDA_TRY(cudaGetDevice(&L.dev));
    while ((int)L.streams.size() < n) {
        cudaStream_t s;
        cudaEvent_t e;
        CJT_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        CJT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        L.streams.push_back(s);
        L.join.push_back(e);
    }
    if (!L.fork) CJT_CUDA_TRY(cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming));
    return CJT_OK;
}

// Issues the items over the lanes; arenas[l] (>= a.need[l] bytes) is lane l's workspace.
int issue(int /*count: a.order holds the items*/, const cjt_plan_t *plans, const int8_t *dir,
          const int64_t *offsets, const double *in, double *out, const Assignment &a, Lanes &L,
          const std::vector<void *> &arenas, cudaStream_t st) {
    const int nl = (int)a.order.size();
    CJT_CUDA_TRY(cudaEventRecord(L.fork, st));
    for (int l = 0; l < nl; ++l) {
        if (a.order[l].empty()) continue;
        CJT_CUDA_TRY(cudaStreamWaitEvent(L.streams[l], L.fork, 0));
        for (int t : a.order[l]) {
            cjt_plan_s *p = plans[t];
            const Workspace ws = p->shared_ws ? cjt_carve(p, arenas[l]) : p->ws;
            int rc = dir[t] == CJT_FWD
                         ? cjt_exec_forward_shifted(p, ws, in + offsets[t], out + offsets[t], L.streams[l])
                         : cjt_exec_inverse_shifted(p, ws, in + offsets[t], out + offsets[t], L.streams[l]);
            if (rc) return rc;
        }
        CJT_CUDA_TRY(cudaEventRecord(L.join[l], L.streams[l]));
        CJT_CUDA_TRY(cudaStreamWaitEvent(st, L.join[l], 0));
    }
    return CJT_OK;
}

int validate(int count, const cjt_plan_t *plans, const int8_t *dir, const int64_t *offsets, const double *in,
             double *out) {
    if (count < 0) return CJT_EINVAL;
    if (count == 0) return CJT_OK;
    if (!plans || !dir || !offsets || !in || !out) return CJT_EINVAL;
    int dev = -1;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    for (int t = 0; t < count; ++t) {
        if (!plans[t] || offsets[t] < 0) return CJT_EINVAL;
        if (plans[t]->dev != dev) return CJT_EINVAL;   // every plan on the current device
        if (dir[t] != CJT_FWD && dir[t] != CJT_INV) return CJT_EINVAL;
        if (!(plans[t]->opts.directions & dir[t])) return CJT_EDIRECTION;
    }
    std::vector<const cjt_plan_s *> seen(plans, plans + count);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return CJT_EINVAL;
    return CJT_OK;
}

int default_lanes() {
    const char *e = getenv("CJT_BATCH_STREAMS");
    int n = e ? atoi(e) : 16;
    return std::min(std::max(n, 1), 64);
}

// the library's lanes and growable arenas for cjt_execute_batched, per device.  An arena
// that is outgrown is retired, not freed: a graph captured from an earlier call may still
// hold its address, and a replay of that graph must not write into freed memory.  Retired
// arenas stay allocated until the process exits.
struct Context {
    Lanes lanes;
    std::vector<void *> arena;
    std::vector<int64_t> bytes;
    std::vector<void *> retired;
};
std::mutex g_mu;
Context g_ctx[64];

}  // namespace

struct cjt_batch_s {
    int dev = -1;   // the device of its plans (current at creation)
    Lanes lanes;
    std::vector<void *> arenas;
    int64_t arena_bytes = 0;
    cjt_group_t group = nullptr;   // the grouped items (cjt_group.cu)
    // the items that run one chain each, for direct (profiled) launches
    std::vector<cjt_plan_t> rp;
    std::vector<int8_t> rd;
    std::vector<int64_t> ro;
    Assignment ra;
    const double *in = nullptr;
    double *out = nullptr;
    int64_t total = 0;             // doubles of the input and of the output buffer
    bool prof = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
};

namespace {
// workspace of one wave of the grouped items: CJT_BATCH_ARENA_MB, default 4096 MiB (two
// such arenas alternate between consecutive waves)
int64_t group_arena_budget() {
    const char *e = getenv("CJT_BATCH_ARENA_MB");
    const long long mb = e ? atoll(e) : 4096;
    return (int64_t)std::max(16LL, mb) << 20;
}
}  // namespace

extern "C" {

int cjt_execute_batched(int count, const cjt_plan_t *plans, const int8_t *dir, const int64_t *offsets,
                        const double *in_dev, double *out_dev, void *stream) {
    int rc = validate(count, plans, dir, offsets, in_dev, out_dev);
    if (rc || count == 0) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CJT_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (!capturing) {
        for (int t = 0; t < count; ++t) {
            rc = cjt_internal_begin_use(plans[t], st);
            if (rc) return rc;
        }
    }
    int dev = 0;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CJT_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    Context &C = g_ctx[dev];
    const int nl = std::min(default_lanes(), count);
    Assignment a = assign(count, plans, dir, nl);
    rc = make_lanes(C.lanes, nl);
    if (rc) return rc;
    C.arena.resize(std::max<size_t>(C.arena.size(), nl), nullptr);
    C.bytes.resize(std::max<size_t>(C.bytes.size(), nl), 0);
    for (int l = 0; l < nl; ++l) {
        if (a.need[l] > C.bytes[l]) {
            if (capturing) return CJT_EBUSY;   // arenas cannot grow under capture
            if (C.arena[l]) C.retired.push_back(C.arena[l]);
            C.arena[l] = nullptr;
            C.bytes[l] = 0;
            cudaError_t e = cudaMalloc(&C.arena[l], a.need[l]);
            if (e != cudaSuccess) {
                cjt_internal_set_cuda_error(e, "cudaMalloc");
                return CJT_ENOMEM;
            }
            C.bytes[l] = a.need[l];
        }
    }
    rc = issue(count, plans, dir, offsets, in_dev, out_dev, a, C.lanes, C.arena, st);
    if (rc) return rc;
    if (!capturing)
        for (int t = 0; t < count; ++t) {
            rc = cjt_internal_end_use(plans[t], st);
            if (rc) return rc;
        }
    return CJT_OK;
}

int cjt_batch_create(cjt_batch_t *out, int count, const cjt_plan_t *plans, const int8_t *dir, const int64_t *offsets,
                     const double *in_dev, double *out_dev, int nstreams) {
    if (!out) return CJT_EINVAL;
    *out = nullptr;
    int rc = validate(count, plans, dir, offsets, in_dev, out_dev);
    if (rc) return rc;
    if (count == 0) return CJT_EINVAL;
    cjt_batch_s *b = new cjt_batch_s();
    auto fail = [&](int code) {
        cjt_batch_destroy(b);
        return code;
    };
    b->dev = plans[0]->dev;   // validate: every plan's device is the current one
    // the grouped items, and the rest (one chain of launches per item on the lanes)
    std::vector<int> grouped, rest;
    const bool no_group = getenv("CJT_BATCH_NO_GROUP") != nullptr;
    for (int t = 0; t < count; ++t)
        (!no_group && cjt_group_eligible(plans[t], dir[t]) ? grouped : rest).push_back(t);
    rc = cjt_group_create(&b->group, grouped, plans, dir, offsets, in_dev, out_dev, group_arena_budget());
    if (rc) return fail(rc);
    b->arena_bytes += cjt_group_arena_bytes(b->group);
    b->kernels += cjt_group_kernels(b->group);
    std::vector<cjt_plan_t> &rp = b->rp;
    std::vector<int8_t> &rd = b->rd;
    std::vector<int64_t> &ro = b->ro;
    for (int t : rest) {
        rp.push_back(plans[t]);
        rd.push_back(dir[t]);
        ro.push_back(offsets[t]);
    }
    b->in = in_dev;
    b->out = out_dev;
    for (int t = 0; t < count; ++t) b->total = std::max(b->total, offsets[t] + plans[t]->N + 1);
    const int nrest = (int)rest.size();
    const int nl = nrest ? std::min(nstreams > 0 ? std::min(nstreams, 64) : default_lanes(), nrest) : 0;
    Assignment &a = b->ra;
    if (nrest) {
        a = assign(nrest, rp.data(), rd.data(), nl);
        rc = make_lanes(b->lanes, nl);
        if (rc) return fail(rc);
        b->arenas.assign(nl, nullptr);
        for (int l = 0; l < nl; ++l) {
            if (!a.need[l]) continue;
            cudaError_t e = cudaMalloc(&b->arenas[l], a.need[l]);
            if (e != cudaSuccess) {
                cjt_internal_set_cuda_error(e, "cudaMalloc");
                return fail(CJT_ENOMEM);
            }
            b->arena_bytes += a.need[l];
        }
        for (int t : rest) {
            cjt_plan_info inf;
            cjt_get_info(plans[t], &inf);
            b->kernels += dir[t] == CJT_FWD ? inf.kernels_fwd : inf.kernels_inv;
        }
    }
    // capture on a private stream: the graph has no tie to any stream once instantiated
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail(CJT_ECUDA);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = cjt_group_issue(b->group, cs);
        if (!rc && nrest) rc = issue(nrest, rp.data(), rd.data(), ro.data(), in_dev, out_dev, a, b->lanes, b->arenas, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
        if (!rc && e2 != cudaSuccess) {
            cjt_internal_set_cuda_error(e2, "cudaStreamEndCapture");
            rc = CJT_ECUDA;
        }
    } else {
        cjt_internal_set_cuda_error(e, "cudaStreamBeginCapture");
        rc = CJT_ECUDA;
    }
    cudaStreamDestroy(cs);
    if (rc) return fail(rc);
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        cjt_internal_set_cuda_error(e, "cudaGraphInstantiate");
        return fail(CJT_ECUDA);
    }
    *out = b;
    return CJT_OK;
}

int cjt_batch_launch(cjt_batch_t b, void *stream) {
    if (!b || !b->exec) return CJT_EINVAL;
    int dev = -1;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->dev) return CJT_EINVAL;   // launched with another device current
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->prof) {
        CJT_CUDA_TRY(cudaGraphLaunch(b->exec, st));
        return CJT_OK;
    }
    // profiled: the graph's launches issued directly, with events around the grouped ones
    int rc = cjt_group_issue(b->group, st, true);
    if (!rc && !b->rp.empty())
        rc = issue((int)b->rp.size(), b->rp.data(), b->rd.data(), b->ro.data(), b->in, b->out, b->ra, b->lanes,
                   b->arenas, st);
    return rc;
}

int cjt_batch_launch_host(cjt_batch_t b, const double *in_host, double *out_host, void *stream) {
    if (!b || !b->exec || !in_host || !out_host) return CJT_EINVAL;
    int dev = -1;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->dev) return CJT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)b->total;
    CJT_CUDA_TRY(cudaMemcpyAsync((void *)b->in, in_host, bytes, cudaMemcpyHostToDevice, st));
    int rc = cjt_batch_launch(b, stream);
    if (rc) return rc;
    CJT_CUDA_TRY(cudaMemcpyAsync(out_host, b->out, bytes, cudaMemcpyDeviceToHost, st));
    CJT_CUDA_TRY(cudaStreamSynchronize(st));
    return CJT_OK;
}

int cjt_batch_set_profiling(cjt_batch_t b, int on) {
    if (!b) return CJT_EINVAL;
    b->prof = on != 0;
    return CJT_OK;
}

int cjt_batch_get_profile(cjt_batch_t b, double *ms, int64_t *counts, int n) {
    if (!b || n < 0) return CJT_EINVAL;
    for (int s = 0; s < n; ++s) {
        if (ms) ms[s] = 0.0;
        if (counts) counts[s] = 0;
    }
    return cjt_group_profile(b->group, ms, counts, n);
}

int cjt_batch_info(cjt_batch_t b, int64_t *kernels, int64_t *arena_bytes) {
    if (!b) return CJT_EINVAL;
    if (kernels) *kernels = b->kernels;
    if (arena_bytes) *arena_bytes = b->arena_bytes;
    return CJT_OK;
}

void cjt_batch_destroy(cjt_batch_t b) {
    if (!b) return;
    // on the batch's device: the synchronisation below must cover its replays
    int cur = -1;
    const bool other = b->dev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != b->dev &&
                       cudaSetDevice(b->dev) == cudaSuccess;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaDeviceSynchronize();
    cjt_group_destroy(b->group);
    for (void *v : b->arenas)
        if (v) cudaFree(v);
    for (auto s : b->lanes.streams) cudaStreamDestroy(s);
    for (auto e : b->lanes.join) cudaEventDestroy(e);
    if (b->lanes.fork) cudaEventDestroy(b->lanes.fork);
    if (other) cudaSetDevice(cur);
    delete b;
}

}  // extern "C"
