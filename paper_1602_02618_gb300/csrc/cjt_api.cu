// C ABI entry points (include/cjt.h): argument checks, plan lifetime, the
// one-stream-at-a-time guard, host-buffer execution and error reporting.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "cjt_internal.cuh"

namespace {
thread_local char g_cuda_err[256] = "";

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

int cjt_internal_check_device(const cjt_plan_s *p) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cjt_internal_set_cuda_error(e, "cudaGetDevice");
        return CJT_ECUDA;
    }
    return dev == p->dev ? CJT_OK : CJT_EINVAL;
}

int cjt_internal_begin_use(cjt_plan_s *p, cudaStream_t st) {
    // a shared-workspace plan holds only read-only tables: any number of streams may use
    // it at once, each with its own workspace
    if (p->shared_ws) return CJT_OK;
    if (p->has_pending && p->last_stream != st) {
        cudaError_t q = cudaEventQuery(p->done);
        if (q == cudaErrorNotReady) return CJT_EBUSY;
        if (q != cudaSuccess) {
            cjt_internal_set_cuda_error(q, "cudaEventQuery");
            return CJT_ECUDA;
        }
    }
    return CJT_OK;
}

namespace {
// Per device and overlap mode: every context ever made (kept until exit) and the free ones
// in the order they were given back.  A chain on a stream of the highest priority is served
// first by the CTA scheduler: at equal priority it hands freed SMs to the kernel launched
// first, so a chain whose head kernel waits behind the thousands of CTAs of the other
// chain's kernel effectively runs after it.
constexpr int kOvPoolMin = 32;   // contexts made before any is reused
std::mutex g_ov_mu;
std::vector<OvCtx *> g_ov_all[64][4];
std::vector<OvCtx *> g_ov_free[64][4];

int make_ovctx(int dev, int mode, OvCtx **out) {
    int least = 0, greatest = 0;
    CJT_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    OvCtx *c = new (std::nothrow) OvCtx();
    if (!c) return CJT_ENOMEM;
    c->dev = dev;
    c->mode = mode;
    const int prio_side = mode == CJT_OVERLAP_ASY_FIRST ? greatest : least;
    CJT_CUDA_TRY(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_side));
    CJT_CUDA_TRY(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    CJT_CUDA_TRY(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming));
    if (mode == CJT_OVERLAP_REC_FIRST) {
        CJT_CUDA_TRY(cudaStreamCreateWithPriority(&c->side_rec, cudaStreamNonBlocking, greatest));
        CJT_CUDA_TRY(cudaEventCreateWithFlags(&c->join_rec, cudaEventDisableTiming));
    }
    g_ov_all[dev][mode].push_back(c);
    *out = c;
    return CJT_OK;
}

// id of the stream capture `s` belongs to (0 when it is not being captured)
unsigned long long capture_id(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    unsigned long long id = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, &id) != cudaSuccess) return ~0ULL;
    return cs == cudaStreamCaptureStatusNone ? 0 : id;
}
}  // namespace

int cjt_internal_ovctx_acquire(int overlap, cudaStream_t origin, OvCtx **out) {
    int dev = 0;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || overlap < 1 || overlap > 3) return CJT_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_ov_mu);
    auto &fr = g_ov_free[dev][overlap];
    if ((int)g_ov_all[dev][overlap].size() >= kOvPoolMin) {
        const unsigned long long mine = capture_id(origin);
        for (size_t k = 0; k < fr.size(); ++k) {
            OvCtx *c = fr[k];
            const unsigned long long cs = capture_id(c->side);
            const unsigned long long cr = c->side_rec ? capture_id(c->side_rec) : 0;
            if ((cs == 0 || cs == mine) && (cr == 0 || cr == mine)) {
                fr.erase(fr.begin() + (long)k);
                *out = c;
                return CJT_OK;
            }
        }
    }
    return make_ovctx(dev, overlap, out);
}

void cjt_internal_ovctx_release(OvCtx *c) {
    if (!c) return;
    std::lock_guard<std::mutex> lk(g_ov_mu);
    g_ov_free[c->dev][c->mode].push_back(c);
}

int cjt_internal_end_use(cjt_plan_s *p, cudaStream_t st) {
    CJT_CUDA_TRY(cudaEventRecord(p->done, st));
    p->last_stream = st;
    p->has_pending = true;
    return CJT_OK;
}

namespace {

int fft_launches(int64_t L) { return L <= 1 ? 0 : (L <= 4096 ? 1 : 2); }
int dft_launches(const Dft &d) { return d.L <= 1 ? 0 : (d.P ? 3 + 2 * fft_launches(d.P) : fft_launches(d.L)); }

// frees a plan's events and memory on the plan's device (the caller's device is restored)
void free_plan(cjt_plan_s *p) {
    int cur = -1;
    const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != p->dev && cudaSetDevice(p->dev) == cudaSuccess;
    for (auto &r : p->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : p->prof_pool) cudaEventDestroy(e);
    for (void *v : p->allocs) cudaFree(v);
    p->allocs.clear();
    cjt_release_twiddles(p);
    if (p->done) cudaEventDestroy(p->done);
    if (other) cudaSetDevice(cur);
    delete p;
}
}  // namespace

void cjt_internal_set_cuda_error(cudaError_t e, const char *what) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

extern "C" {

const char *cjt_version(void) { return "cjt-gb300 0.1 (sm_103a)"; }

const char *cjt_last_cuda_error(void) { return g_cuda_err; }

const char *cjt_strerror(int code) {
    switch (code) {
        case CJT_OK: return "success";
        case CJT_EINVAL: return "invalid argument";
        case CJT_EDOMAIN: return "alpha or beta outside [-1/2, 3/2]";
        case CJT_ENOMEM: return "out of memory";
        case CJT_ECUDA: return "CUDA runtime error";
        case CJT_ETIMEOUT: return "device-side wait timed out";
        case CJT_EBUSY: return "plan in use on another stream";
        case CJT_EUNSUPPORTED: return "unsupported request";
        case CJT_EDIRECTION: return "plan not built for this direction";
        default: return "unknown error";
    }
}

int cjt_plan_opts_default(cjt_plan_opts *o) {
    if (!o) return CJT_EINVAL;
    memset(o, 0, sizeof(*o));
    o->M = 7;
    o->eps = 0x1p-52;
    o->precision = CJT_FP64;
    o->directions = CJT_FWD | CJT_INV;
    o->ratio = 0.0;
    o->seg_len = 2048;
    o->use_asy = 1;
    return CJT_OK;
}

int cjt_plan(cjt_plan_t *out, int64_t N, double alpha, double beta, const cjt_plan_opts *opts, void *stream) {
    if (!out) return CJT_EINVAL;
    *out = nullptr;
    if (N < 0) return CJT_EINVAL;
    if (N > (1LL << 22)) return CJT_EUNSUPPORTED;
    if (!(alpha >= -0.5 && alpha <= 1.5) || !(beta >= -0.5 && beta <= 1.5)) return CJT_EDOMAIN;
    cjt_plan_opts o;
    cjt_plan_opts_default(&o);
    if (opts) {
        if (opts->M) o.M = opts->M;
        if (opts->eps != 0.0) o.eps = opts->eps;
        o.precision = opts->precision;
        if (opts->directions) o.directions = opts->directions;
        o.ratio = opts->ratio;
        if (opts->seg_len) o.seg_len = opts->seg_len;
        if (opts->use_asy) o.use_asy = opts->use_asy;
        o.shared_workspace = opts->shared_workspace;
        o.rec_store = opts->rec_store;
        o.expansion = opts->expansion;
        o.grid = opts->grid;
        o.overlap = opts->overlap;
        o.seg_whole = opts->seg_whole;
    }
    if (o.M < 1 || o.M > 20) return CJT_EINVAL;
    if (!(o.eps > 0.0 && o.eps < 1.0)) return CJT_EINVAL;
    if (o.precision != CJT_FP64 && o.precision != CJT_MIXED && o.precision != CJT_DFLOAT) return CJT_EINVAL;
    if (o.directions < 1 || o.directions > 3) return CJT_EINVAL;
    if (!(o.ratio == 0.0 || (o.ratio > 0.0 && o.ratio < 1.0))) return CJT_EINVAL;
    if (o.use_asy != 1 && o.use_asy != -1) return CJT_EINVAL;
    if (o.rec_store != 0 && o.rec_store != 1) return CJT_EINVAL;
    if (o.expansion < CJT_EXPANSION_AUTO || o.expansion > CJT_EXPANSION_ULTRASPHERICAL) return CJT_EINVAL;
    if (o.expansion == CJT_EXPANSION_ULTRASPHERICAL && alpha != beta) return CJT_EINVAL;
    if (o.grid < -1 || o.grid > 1) return CJT_EINVAL;
    if (o.overlap < CJT_OVERLAP_AUTO || o.overlap > CJT_OVERLAP_REC_FIRST) return CJT_EINVAL;
    if (o.overlap == CJT_OVERLAP_AUTO) o.overlap = CJT_OVERLAP_ASY_FIRST;
    if (o.seg_len < 32 || o.seg_len > (1 << 20) || (o.seg_len % 32) != 0) return CJT_EINVAL;
    if (o.seg_whole < 0 || o.seg_whole > (1 << 23)) return CJT_EINVAL;
    if (N > (1LL << 21) && !is_pow2(N) && !cjt_is_3pow2(N) && !cjt_is_5pow2(N) && o.grid == -1)
        return CJT_EUNSUPPORTED;   // Bluestein lengths <= 2^24

    cjt_plan_s *p = new (std::nothrow) cjt_plan_s();
    if (!p) return CJT_ENOMEM;
    p->N = N;
    {
        cudaError_t e = cudaGetDevice(&p->dev);
        if (e != cudaSuccess) {
            cjt_internal_set_cuda_error(e, "cudaGetDevice");
            delete p;
            return CJT_ECUDA;
        }
    }
    // one unit step down into the square [-1/2, 1/2]^2 for a parameter in (1/2, 3/2]
    // (Sec. 1.2; alpha - 1 is exact there)
    auto shift_of = [](double v) { return v > 0.5 ? 1 : 0; };
    p->alpha_user = alpha;
    p->beta_user = beta;
    p->shift_a = shift_of(alpha);
    p->shift_b = shift_of(beta);
    p->alpha = alpha - p->shift_a;
    p->beta = beta - p->shift_b;
    p->opts = o;
    p->seg_len = o.seg_len;
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    int rc;
    if (N == 0) {
        rc = CJT_OK;
        cudaError_t e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
        if (e != cudaSuccess) { cjt_internal_set_cuda_error(e, "cudaEventCreate"); rc = CJT_ECUDA; }
        if (!rc) {
            e = cudaMalloc((void **)&p->d_in, 2 * sizeof(double));
            if (e != cudaSuccess) { cjt_internal_set_cuda_error(e, "cudaMalloc"); rc = CJT_ENOMEM; }
            else { p->allocs.push_back(p->d_in); p->d_out = p->d_in + 1; }
        }
    } else {
        rc = cjt_plan_build(p, st);
    }
    if (rc) {
        cudaStreamSynchronize(st);
        free_plan(p);
        return rc;
    }
    p->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return CJT_OK;
}

void cjt_destroy(cjt_plan_t p) {
    if (!p) return;
    if (p->has_pending && p->done) cudaEventSynchronize(p->done);
    free_plan(p);
}

int cjt_get_info(cjt_plan_t p, cjt_plan_info *info) {
    if (!p || !info) return CJT_EINVAL;
    memset(info, 0, sizeof(*info));
    info->N = p->N;
    info->alpha = p->alpha_user;
    info->beta = p->beta_user;
    info->shift_alpha = p->shift_a;
    info->shift_beta = p->shift_b;
    info->expansion = p->expansion_used;
    info->parity_fold = (p->fw.fold || p->iv.fold) ? 1 : 0;
    info->overlap = p->opts.overlap;
    info->grid_fwd = (p->opts.directions & CJT_FWD) ? p->Gf : 0;
    info->grid_inv = (p->opts.directions & CJT_INV) ? 2 * p->Gi : 0;
    info->M = p->M;
    info->precision = p->opts.precision;
    info->directions = p->opts.directions;
    info->n_M = p->n_M;
    info->ratio = p->ratio;
    info->nblk_fwd = p->fw.nblk;
    info->nblk_inv = p->iv.nblk;
    info->rec_steps_fwd = p->fw.rec_steps;
    info->rec_steps_inv = p->iv.rec_steps;
    info->fft_len_fwd = p->Lf;
    info->fft_len_inv = p->Li;
    info->nfft_fwd = p->npair_f + (p->N > 0 ? 1 : 0);
    info->nfft_inv = p->npair_i + (p->N > 0 ? 1 : 0);
    info->rec_items_fwd = p->fw.nitems;
    info->rec_items_inv = p->iv.nitems;
    info->device_bytes = p->device_bytes;
    info->plan_ms = p->plan_ms;
    info->workspace_bytes = p->ws_bytes;
    info->rec_store_bytes = 8 * ((p->fw.d_E ? p->fw.nE : 0) + (p->iv.d_E ? p->iv.nE : 0));
    if (p->N == 0) {
        info->kernels_fwd = info->kernels_inv = 1;
    } else {
        const int nqf = p->fw.nblk * p->M, nqi = p->iv.nblk * p->M;
        info->kernels_fwd = (p->fw.nitems > 0) + (nqf > 0 ? 1 + dft_launches(p->dft_f) : 0) + 1 +
                            dft_launches(p->dft_dct) + 1 +
                            (p->prec_asy == PREC_DF ? 2 : 0);   // input scaling to double-float
        info->kernels_inv = 1 + dft_launches(p->dft_front) + 1 + (nqi > 0 ? 1 + dft_launches(p->dft_i) : 0) +
                            (p->iv.nitems > 0) + 2 + (p->prec_asy == PREC_DF ? 2 : 0);
        info->kernels_fwd += cjt_conv_kernels(p);
        info->kernels_inv += cjt_conv_kernels(p);
        if (!(p->opts.directions & CJT_FWD)) info->kernels_fwd = 0;
        if (!(p->opts.directions & CJT_INV)) info->kernels_inv = 0;
    }
    return CJT_OK;
}

// ---------------------------------------------------------------------------
// the plan's asymptotic expansion on the host
// ---------------------------------------------------------------------------
namespace {
int asy_host(double alpha, double beta, int expansion, AsyExp *e) {
    if (!(alpha >= -0.5 && alpha <= 0.5) || !(beta >= -0.5 && beta <= 0.5)) return CJT_EDOMAIN;
    if (expansion < CJT_EXPANSION_AUTO || expansion > CJT_EXPANSION_ULTRASPHERICAL) return CJT_EINVAL;
    const bool corner = std::fabs(alpha) == 0.5 && std::fabs(beta) == 0.5;
    return cjt_asy_make(alpha, beta, corner && alpha != beta ? CJT_EXPANSION_HAHN : expansion, e);
}
}  // namespace

int cjt_asy_coefficient(double alpha, double beta, int expansion, int64_t n, int m, double *C) {
    if (!C || n < 0 || m < 0 || m > 20) return CJT_EINVAL;
    AsyExp e;
    int rc = asy_host(alpha, beta, expansion, &e);
    if (rc) return rc;
    *C = cjt_asy_C(e, n, m);
    return CJT_OK;
}

int cjt_rec_coefficients(double alpha, double beta, int64_t n, double *out) {
    if (!out || n < 0 || n > (1LL << 40)) return CJT_EINVAL;
    if (!(alpha >= -0.5 && alpha <= 0.5) || !(beta >= -0.5 && beta <= 0.5)) return CJT_EDOMAIN;
    const RecRow r = cjt_rec_row(n, alpha, beta);
    const double v[CJT_REC_COEFFS] = {r.A, r.B, r.C, r.rf_p, r.rf_m, r.rb_p, r.rb_m, r.Ce_p, r.Ce_m, r.Cr_p, r.Cr_m};
    for (int k = 0; k < CJT_REC_COEFFS; ++k) out[k] = v[k];
    return CJT_OK;
}

int cjt_asy_eval(double alpha, double beta, int expansion, int M, int64_t n, int64_t i, int64_t Ng, double *value,
                 double *bound) {
    if (!value || !bound || M < 1 || M > 20 || n < 0 || Ng < 2 || Ng > (1LL << 30) || i <= 0 || i >= Ng)
        return CJT_EINVAL;
    AsyExp e;
    int rc = asy_host(alpha, beta, expansion, &e);
    if (rc) return rc;
    // cos(n theta), sin(n theta) with the argument reduced exactly: n i mod 2 Ng
    const int64_t r = ((n % (2 * Ng)) * i) % (2 * Ng);
    const double cn = cjt_host_cospi((double)r / (double)Ng), sn = cjt_host_sinpi((double)r / (double)Ng);
    double s = 0.0;
    for (int m = 0; m < M; ++m) {
        double u, v;
        cjt_asy_uv(e, m, i, Ng, &u, &v);
        s += cjt_asy_C(e, n, m) * (u * cn + v * sn);
    }
    *value = s;
    *bound = 2.0 * cjt_asy_C(e, n, M) * cjt_asy_env(e, M, i, Ng);
    return CJT_OK;
}

int cjt_get_partition(cjt_plan_t p, int direction, int cap, int64_t *boxes, int *nblk) {
    if (!p || !nblk || cap < 0 || (cap > 0 && !boxes)) return CJT_EINVAL;
    if (direction != CJT_FWD && direction != CJT_INV) return CJT_EINVAL;
    if (!(p->opts.directions & direction)) return CJT_EDIRECTION;
    const GridWork &gw = direction == CJT_FWD ? p->fw : p->iv;
    *nblk = gw.nblk;
    if (gw.nblk > cap) return CJT_EINVAL;
    for (int k = 0; k < gw.nblk; ++k) {
        boxes[3 * k] = gw.jk[k];
        boxes[3 * k + 1] = gw.i1[k];
        boxes[3 * k + 2] = gw.i2[k];
    }
    return CJT_OK;
}

int cjt_error_bound(cjt_plan_t p, int direction, double *bound) {
    if (!p || !bound) return CJT_EINVAL;
    if (direction != CJT_FWD && direction != CJT_INV) return CJT_EINVAL;
    if (!(p->opts.directions & direction)) return CJT_EDIRECTION;
    const double fp64 = 1e-12;   // the FP64 form's stated bound (all forms' FP64 parts)
    *bound = fp64 + (p->opts.precision == CJT_MIXED ? (direction == CJT_FWD ? p->err_mixed_fwd : p->err_mixed_inv) : 0.0);
    return CJT_OK;
}

int cjt_set_profiling(cjt_plan_t p, int on) {
    if (!p) return CJT_EINVAL;
    p->prof = on != 0;
    return CJT_OK;
}

int cjt_get_profile(cjt_plan_t p, double *ms, int64_t *counts, int n) {
    if (!p || n < 0) return CJT_EINVAL;
    for (int s = 0; s < n; ++s) {
        if (ms) ms[s] = 0.0;
        if (counts) counts[s] = 0;
    }
    int rc = CJT_OK;
    for (auto &r : p->prof_pending) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) {
            cjt_internal_set_cuda_error(e, "cudaEventElapsedTime");
            rc = CJT_ECUDA;
        }
        if (r.stage < n) {
            if (ms) ms[r.stage] += t;
            if (counts) counts[r.stage] += 1;
        }
        p->prof_pool.push_back(r.a);
        p->prof_pool.push_back(r.b);
    }
    p->prof_pending.clear();
    return rc;
}

static int run_one(cjt_plan_t p, int direction, const double *in, double *out, const Workspace &ws, void *stream) {
    if (!p || !in || !out) return CJT_EINVAL;
    if (!(p->opts.directions & direction)) return CJT_EDIRECTION;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cjt_internal_check_device(p);
    if (rc) return rc;
    rc = cjt_internal_begin_use(p, st);
    if (rc) return rc;
    rc = direction == CJT_FWD ? cjt_exec_forward_shifted(p, ws, in, out, st)
                              : cjt_exec_inverse_shifted(p, ws, in, out, st);
    if (rc) return rc;
    return cjt_internal_end_use(p, st);
}

int cjt_forward(cjt_plan_t p, const double *in, double *out, void *stream) {
    if (p && p->shared_ws && p->N > 0) return CJT_EINVAL;
    return p ? run_one(p, CJT_FWD, in, out, p->ws, stream) : CJT_EINVAL;
}

int cjt_inverse(cjt_plan_t p, const double *in, double *out, void *stream) {
    if (p && p->shared_ws && p->N > 0) return CJT_EINVAL;
    return p ? run_one(p, CJT_INV, in, out, p->ws, stream) : CJT_EINVAL;
}

int cjt_jacobi_to_jacobi(cjt_plan_t from, cjt_plan_t to, const double *in, double *out, void *stream) {
    if (!from || !to || !in || !out || from->N != to->N) return CJT_EINVAL;
    if (!(from->opts.directions & CJT_FWD) || !(to->opts.directions & CJT_INV)) return CJT_EDIRECTION;
    int rc = cjt_forward(from, in, out, stream);
    if (rc) return rc;
    return cjt_inverse(to, out, out, stream);
}

int cjt_forward_ws(cjt_plan_t p, const double *in, double *out, void *ws, size_t bytes, void *stream) {
    if (!p || (!ws && p->ws_bytes > 0) || (int64_t)bytes < p->ws_bytes) return CJT_EINVAL;
    return run_one(p, CJT_FWD, in, out, cjt_carve(p, ws), stream);
}

int cjt_inverse_ws(cjt_plan_t p, const double *in, double *out, void *ws, size_t bytes, void *stream) {
    if (!p || (!ws && p->ws_bytes > 0) || (int64_t)bytes < p->ws_bytes) return CJT_EINVAL;
    return run_one(p, CJT_INV, in, out, cjt_carve(p, ws), stream);
}

int cjt_execute_host(cjt_plan_t p, int direction, const double *in_host, double *out_host, void *stream) {
    if (!p || !in_host || !out_host) return CJT_EINVAL;
    if (direction != CJT_FWD && direction != CJT_INV) return CJT_EINVAL;
    if (!(p->opts.directions & direction)) return CJT_EDIRECTION;
    if (p->shared_ws && p->N > 0) return CJT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cjt_internal_check_device(p);
    if (rc) return rc;
    rc = cjt_internal_begin_use(p, st);
    if (rc) return rc;
    const size_t bytes = sizeof(double) * (size_t)(p->N + 1);
    CJT_CUDA_TRY(cudaMemcpyAsync(p->d_in, in_host, bytes, cudaMemcpyHostToDevice, st));
    rc = direction == CJT_FWD ? cjt_exec_forward_shifted(p, p->ws, p->d_in, p->d_out, st)
                              : cjt_exec_inverse_shifted(p, p->ws, p->d_in, p->d_out, st);
    if (rc) return rc;
    CJT_CUDA_TRY(cudaMemcpyAsync(out_host, p->d_out, bytes, cudaMemcpyDeviceToHost, st));
    rc = cjt_internal_end_use(p, st);
    if (rc) return rc;
    CJT_CUDA_TRY(cudaStreamSynchronize(st));
    return CJT_OK;
}

int cjt_sync(void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        cjt_internal_set_cuda_error(e, "cudaStreamSynchronize");
        return CJT_ECUDA;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cjt_internal_set_cuda_error(e, "cudaGetLastError");
        return CJT_ECUDA;
    }
    return CJT_OK;
}

}  // extern "C"
