// Grouped batched execution: the transforms of a batch run stage by stage, one launch per
// stage over many transforms at once, instead of one chain of launches per transform
// (Sec. 4: one plan machinery applied to many sets of coefficients).
//
// Items are taken in order of decreasing cost and packed into waves whose workspace fits
// an arena of a given size; waves alternate between two arenas and two stream pairs, so
// that one wave's last stages overlap the next wave's first.  In a wave:
//   main stream   inverse front end: [c; 0] packing, DCT-I of length 4G per length class,
//                 g = w o p_N
//   side stream   forward ASY packs, their DCT-I/DST-I per (length, precision) class, then
//   (priority)    (after the front end) the inverse ASY packs and transforms
//   main stream   recurrences (forward and transposed, at execution or stored), the fixed-
//                 order reduction over items, then (after the side stream) the combines,
//                 the final DCT-I per length class and its scaling
// Each elementwise launch walks a table of (transform, chunk) pairs, one per CTA; each
// recurrence launch finds a warp's (or CTA's) transform by binary search over the prefix
// sums of the transforms' work items.  All transforms of a length class share one batched
// FFT launch over a contiguous region of the arena, with the twiddle tables of one member
// plan: a plan's tables hold omega_{Ltab}^k = exp(-2 pi i k / Ltab) from the same
// sincospi call at the same (exactly scaled) angle whatever Ltab, so every member would
// read the same values.  The per-element arithmetic is that of the single-transform
// kernels (cjt_kern.cuh), so each result is bit-identical to the transform run alone.
//
// Eligible items: N >= 1, FP64 or mixed (FP32 transforms) precision, no parameter shift,
// transform lengths 2^b, 3 2^b or 5 2^b (the default grids).  The batch runs the others (double-
// float form, shifted parameters, Bluestein lengths) one chain per item on its lanes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "cjt_group.cuh"
#include "cjt_kern.cuh"

namespace {

inline int ilog2_exact(int64_t v) {
    int r = 0;
    while ((1LL << r) < v) ++r;
    return r;
}

// Everything one transform's stage kernels read or write.
struct __align__(16) GDesc {
    int64_t N, G, Ng, L;      // degree; forward grid G; grid of this direction (G or 2G); ASY length
    int logL, M, nblk, nq, npair, seg_len, q, pad1;   // L = q 2^logL, q = 1, 3 or 5
    RecTables rt;
    const RecItem *items;
    int64_t nitems;
    const double *states, *E;
    const int *rowk;
    const int64_t *row_base;
    const int *row_nseg;
    const double *scale, *u, *v, *Cnm, *w, *s_n;
    const int *box;
    const int64_t *seg_ptr, *seg_out;
    const int *seg_b;
    const double *in;
    double *out;
    void *fft;        // npair x L transform inputs (FP64 or FP32 complex)
    double2 *dct;     // forward: even extension of y, length 2G; inverse: front end, length 4G
    double *y, *g, *part;
};
static_assert(sizeof(GDesc) % 8 == 0 && sizeof(GDesc) <= 256 * 8, "descriptor copy");

struct GTab {
    int item;   // descriptor index
    int blk;    // chunk of the transform's index space
};

constexpr int GE_THREADS = 256;
constexpr int GE_CHUNK = 8 * GE_THREADS;   // elements per CTA of the elementwise launches

// ---------------------------------------------------------------------------
// elementwise stages: index space and element of one transform
// ---------------------------------------------------------------------------
enum { OP_PACK_FWD, OP_PACK_INV, OP_COMBINE_FWD, OP_DCT_FINISH, OP_FRONT_PACK, OP_INV_G, OP_COMBINE_INV, OP_NELEM };

template <int OP> struct Elem;
// packs: the pair's scales are formed once per thread and pair (PairCache)
struct PairCache {
    int p = -1;
    cjt_kern::PairScale ps;
    __device__ const cjt_kern::PairScale &of(int pp, const GDesc &d) {
        if (pp != p) {
            p = pp;
            ps = cjt_kern::pair_scale(pp, d.M, d.nq, d.scale);
        }
        return ps;
    }
};
template <> struct Elem<OP_FRONT_PACK> {
    static __host__ __device__ int64_t size(const GDesc &d) { return d.L; }   // 4G
    template <typename V, typename R> static __device__ void apply(const GDesc &d, int64_t k, PairCache &) {
        cjt_kern::inv_front_pack_elem(k, d.N, d.in, d.dct);
    }
};
template <> struct Elem<OP_INV_G> {
    static __host__ __device__ int64_t size(const GDesc &d) { return d.Ng + 1; }
    template <typename V, typename R> static __device__ void apply(const GDesc &d, int64_t i, PairCache &) {
        cjt_kern::inv_g_elem(i, d.dct, d.w, d.g);
    }
};
// the transform (pair) of element idx of a pack's index space, and the element within it
__device__ __forceinline__ int pair_of(const GDesc &d, int64_t idx) {
    return d.q > 1 ? (int)((idx >> d.logL) / d.q) : (int)(idx >> d.logL);
}
template <> struct Elem<OP_PACK_FWD> {
    static __host__ __device__ int64_t size(const GDesc &d) { return (int64_t)d.npair * d.L; }
    template <typename V, typename R> static __device__ void apply(const GDesc &d, int64_t idx, PairCache &pc) {
        const int p = pair_of(d, idx);
        cjt_kern::asy_pack_fwd_elem<V, R>(idx - (int64_t)p * d.L, p, pc.of(p, d), d.N, d.L, d.box, d.Cnm, d.in,
                                          (V *)d.fft);
    }
};
// one element per row i < Ng = L / 2 of each pair (the row's two transform inputs)
template <> struct Elem<OP_PACK_INV> {
    static __host__ __device__ int64_t size(const GDesc &d) { return (int64_t)d.npair * d.Ng; }
    template <typename V, typename R> static __device__ void apply(const GDesc &d, int64_t idx, PairCache &pc) {
        const int p = d.q > 1 ? (int)((idx >> (d.logL - 1)) / d.q) : (int)(idx >> (d.logL - 1));
        cjt_kern::asy_pack_inv_elem<V, R>(idx - (int64_t)p * d.Ng, p, pc.of(p, d), d.Ng, d.L, d.box, d.u, d.v, d.g,
                                          (V *)d.fft);
    }
};
template <> struct Elem<OP_COMBINE_FWD> {
    static __host__ __device__ int64_t size(const GDesc &d) { return d.G + 1; }
    template <typename V, typename R> static __device__ void apply(const GDesc &d, int64_t i, PairCache &) {
        cjt_kern::combine_fwd_elem<V>(i, d.G, d.L, d.M, d.rowk, d.scale, d.u, d.v, (const V *)d.fft, d.row_base,
                                      d.row_nseg, d.part, d.dct);
    }
};
template <> struct Elem<OP_DCT_FINISH> {
    static __host__ __device__ int64_t size(const GDesc &d) { return d.N + 1; }
    template <typename V, typename R> static __device__ void apply(const GDesc &d, int64_t k, PairCache &) {
        cjt_kern::dct_finish_elem(k, d.G, d.dct, d.out);
    }
};
template <> struct Elem<OP_COMBINE_INV> {
    static __host__ __device__ int64_t size(const GDesc &d) { return d.N + 1; }
    template <typename V, typename R> static __device__ void apply(const GDesc &d, int64_t n, PairCache &) {
        cjt_kern::combine_inv_elem<V>(n, d.N, d.L, d.M, d.nblk, d.box, d.scale, d.Cnm, (const V *)d.fft, d.y, d.s_n,
                                      nullptr, 0, d.out);
    }
};

// one CTA per table entry: the transform's descriptor goes to shared memory once
template <int OP, typename V, typename R>
__global__ void __launch_bounds__(GE_THREADS) k_g_elem(const GDesc *__restrict__ D, const GTab *__restrict__ tab) {
    __shared__ GDesc sd;
    const GTab e = tab[blockIdx.x];
    {
        const long long *src = reinterpret_cast<const long long *>(D + e.item);
        long long *dst = reinterpret_cast<long long *>(&sd);
        for (int k = threadIdx.x; k < (int)(sizeof(GDesc) / 8); k += GE_THREADS) dst[k] = src[k];
    }
    __syncthreads();
    const int64_t n = Elem<OP>::size(sd);
    const int64_t i0 = (int64_t)e.blk * GE_CHUNK, i1 = min(n, i0 + GE_CHUNK);
    PairCache pc;
    // a fixed trip count, unrolled, so that the loads of several elements are in flight
#pragma unroll
    for (int u = 0; u < GE_CHUNK / GE_THREADS; ++u) {
        const int64_t i = i0 + threadIdx.x + (int64_t)u * GE_THREADS;
        if (i < i1) Elem<OP>::template apply<V, R>(sd, i, pc);
    }
}

// ---------------------------------------------------------------------------
// recurrences and the reduction over items
// ---------------------------------------------------------------------------
// index of the selected transform whose work items contain global item x: the largest s
// with pre[s] <= x (pre[0] = 0, pre[nsel] = total)
__device__ __forceinline__ int g_find(const int64_t *__restrict__ pre, int nsel, int64_t x) {
    int lo = 0, hi = nsel;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(128) k_g_rec_fwd(const GDesc *__restrict__ D, const int *__restrict__ sel,
                                                   const int64_t *__restrict__ pre, int nsel, int64_t total) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= total) return;
    const int s = g_find(pre, nsel, w);
    const GDesc &d = D[sel[s]];
    const RecItem it = d.items[w - pre[s]];
    const RecTables t = d.rt;
    cjt_kern::rec_fwd_warp(it, threadIdx.x & 31, d.Ng, t, d.in, d.states, d.part);
}

constexpr int GRI_WARPS = 4;
__global__ void __launch_bounds__(32 * GRI_WARPS) k_g_rec_inv(const GDesc *__restrict__ D, const int *__restrict__ sel,
                                                              const int64_t *__restrict__ pre, int nsel, int64_t total) {
    __shared__ double tile[GRI_WARPS][32][33];
    const int wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * GRI_WARPS + wib;
    if (w >= total) return;
    const int s = g_find(pre, nsel, w);
    const GDesc &d = D[sel[s]];
    const RecItem it = d.items[w - pre[s]];
    const RecTables t = d.rt;
    cjt_kern::rec_inv_warp(it, threadIdx.x & 31, tile[wib], d.Ng, t, d.g, d.states, d.part);
}

__global__ void __launch_bounds__(32 * cjt_kern::SW) k_g_rec_fwd_stored(const GDesc *__restrict__ D,
                                                                        const int *__restrict__ sel,
                                                                        const int64_t *__restrict__ pre, int nsel) {
    const int s = g_find(pre, nsel, blockIdx.x);
    const GDesc &d = D[sel[s]];
    const RecItem it = d.items[blockIdx.x - pre[s]];
    cjt_kern::rec_fwd_stored_cta(it, d.in, d.E, d.part);
}

__global__ void __launch_bounds__(32 * cjt_kern::SW) k_g_rec_inv_stored(const GDesc *__restrict__ D,
                                                                        const int *__restrict__ sel,
                                                                        const int64_t *__restrict__ pre, int nsel) {
    const int s = g_find(pre, nsel, blockIdx.x);
    const GDesc &d = D[sel[s]];
    const RecItem it = d.items[blockIdx.x - pre[s]];
    cjt_kern::rec_inv_stored_cta(it, d.Ng, d.g, d.E, d.part);
}

// W warps per block: 8 for small transforms (more blocks resident per SM), 32 for large ones,
// whose heavy low-degree segments have few blocks (the bits are the same for every W)
template <int W>
__global__ void __launch_bounds__(32 * W) k_g_inv_reduce(const GDesc *__restrict__ D, const GTab *__restrict__ tab) {
    const GTab e = tab[blockIdx.x];
    const GDesc &d = D[e.item];
    cjt_kern::inv_reduce_block<W>(e.blk, d.N, d.seg_len, d.seg_ptr, d.seg_out, d.seg_b, d.part, d.y);
}
constexpr int64_t kReduceWideRows = 1 << 19;   // inverse grids of at least this many rows: W = 32

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
enum { ST_ELEM, ST_REC, ST_REDUCE, ST_FFT, ST_RECORD, ST_WAIT };
enum { REC_K_FWD, REC_K_INV, REC_K_FWD_STORED, REC_K_INV_STORED };
enum { EV_FORK, EV_FRONT, EV_SIDE, EV_N };

struct Step {
    int type = 0;
    int cat = -1;                     // CJT_BSTAGE_* of the launch (profiling)
    int op = 0, prec = PREC_F64;      // ST_ELEM: Elem op and transform precision; ST_REC: REC_K_*
    size_t tab = 0;                   // ST_ELEM / ST_REDUCE: GTab offset; ST_REC: sel offset
    size_t pre = 0;                   // ST_REC: prefix offset
    int64_t grid = 0, total = 0;      // CTAs; ST_REC: work items
    int nsel = 0;
    // ST_FFT
    size_t data = 0, scratch = 0;     // arena offsets
    int64_t L = 0, count = 0;
    Twiddles tw{};
    int event = 0;                    // ST_RECORD / ST_WAIT
};

struct WavePlan {
    int pair = 0;
    std::vector<Step> main_front, side, main_rec, main_post;
};

double item_cost(const cjt_plan_s *p, int dir) {
    const bool f = dir == CJT_FWD;
    const GridWork &gw = f ? p->fw : p->iv;
    const double L = (double)(f ? p->Lf : p->Li);
    const double npair = f ? p->npair_f : p->npair_i;
    const double lg = std::log2(std::max(L, 2.0));
    const double rec = (gw.d_E ? 2.0 : 8.0) * (double)gw.rec_steps;
    return rec + 2.5 * (npair + 1.0) * L * lg + 50.0 * (double)gw.Ng;
}

int64_t align256(int64_t v) { return (v + 255) / 256 * 256; }

}  // namespace

struct cjt_group_s {
    int dev = 0;
    std::vector<GDesc> desc;                 // host copy
    std::vector<unsigned char> tables;       // host copy of the launch tables
    unsigned char *d_tables = nullptr;       // descriptors first, then tables
    size_t desc_bytes = 0;
    void *arena[2] = {nullptr, nullptr};
    int64_t arena_bytes[2] = {0, 0};
    std::vector<WavePlan> waves;
    cudaStream_t main[2] = {nullptr, nullptr}, side[2] = {nullptr, nullptr};
    cudaEvent_t ev[2][EV_N] = {{nullptr}};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    int64_t kernels = 0;
    // profiling: an event pair around every launch step of a direct (not captured) issue
    struct Rec { int cat; cudaEvent_t a, b; };
    std::vector<Rec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
};

bool cjt_group_eligible(const cjt_plan_s *p, int dir) {
    if (p->N < 1 || p->shift_a || p->shift_b) return false;
    if (p->prec_asy != PREC_F64 && p->prec_asy != PREC_F32) return false;
    if (dir == CJT_FWD) {
        if (p->fw.nblk > 0 && p->dft_f.P) return false;
        if (p->dft_dct.P) return false;
    } else {
        if (p->iv.nblk > 0 && p->dft_i.P) return false;
        if (p->dft_front.P) return false;
    }
    return true;
}

namespace {

template <typename T> size_t push_table(std::vector<unsigned char> &buf, const std::vector<T> &v) {
    size_t off = (buf.size() + 15) / 16 * 16;
    buf.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

// an elementwise launch over the selected descriptors (those with a non-empty index space)
template <int OP> void add_elem(cjt_group_s *g, std::vector<Step> &out, const std::vector<int> &sel, int prec) {
    std::vector<GTab> tab;
    for (int t : sel) {
        const int64_t n = Elem<OP>::size(g->desc[t]);
        for (int64_t b = 0; b * GE_CHUNK < n; ++b) tab.push_back({t, (int)b});
    }
    if (tab.empty()) return;
    Step s;
    s.type = ST_ELEM;
    s.op = OP;
    s.prec = prec;
    s.cat = (OP == OP_PACK_FWD || OP == OP_PACK_INV) ? CJT_BSTAGE_PACK
            : (OP == OP_COMBINE_FWD || OP == OP_COMBINE_INV) ? CJT_BSTAGE_COMBINE : CJT_BSTAGE_OTHER;
    s.tab = push_table(g->tables, tab);
    s.grid = (int64_t)tab.size();
    out.push_back(s);
}

void add_rec(cjt_group_s *g, std::vector<Step> &out, const std::vector<int> &sel, int kind) {
    std::vector<int> s2;
    std::vector<int64_t> pre(1, 0);
    for (int t : sel) {
        if (g->desc[t].nitems <= 0) continue;
        s2.push_back(t);
        pre.push_back(pre.back() + g->desc[t].nitems);
    }
    if (s2.empty()) return;
    Step s;
    s.type = ST_REC;
    s.op = kind;
    s.cat = (kind == REC_K_FWD_STORED || kind == REC_K_INV_STORED) ? CJT_BSTAGE_REC_STORED : CJT_BSTAGE_REC;
    s.tab = push_table(g->tables, s2);
    s.pre = push_table(g->tables, pre);
    s.nsel = (int)s2.size();
    s.total = pre.back();
    out.push_back(s);
}

void add_reduce(cjt_group_s *g, std::vector<Step> &out, const std::vector<int> &sel) {
    for (int wide = 0; wide < 2; ++wide) {
        std::vector<GTab> tab;
        for (int t : sel) {
            if ((g->desc[t].Ng >= kReduceWideRows) != (wide == 1)) continue;
            for (int64_t b = 0; b * 32 < g->desc[t].N + 1; ++b) tab.push_back({t, (int)b});
        }
        if (tab.empty()) continue;
        Step s;
        s.type = ST_REDUCE;
        s.op = wide ? 32 : 8;
        s.cat = CJT_BSTAGE_REDUCE;
        s.tab = push_table(g->tables, tab);
        s.grid = (int64_t)tab.size();
        out.push_back(s);
    }
}

Step ev_step(int type, int e) {
    Step s;
    s.type = type;
    s.event = e;
    return s;
}

// kernel launches of one transform of length L batched over `count` sequences
int fft_launches(int64_t L) { return L <= 1 ? 0 : (L <= 4096 ? 1 : 2); }

template <int OP, typename V, typename R>
int launch_elem(const GDesc *D, const GTab *tab, int64_t grid, cudaStream_t st) {
    k_g_elem<OP, V, R><<<(unsigned)grid, GE_THREADS, 0, st>>>(D, tab);
    CJT_CUDA_TRY(cudaGetLastError());
    return CJT_OK;
}

template <int OP> int launch_elem_prec(int prec, const GDesc *D, const GTab *tab, int64_t grid, cudaStream_t st) {
    return prec == PREC_F32 ? launch_elem<OP, float2, float>(D, tab, grid, st)
                            : launch_elem<OP, double2, double>(D, tab, grid, st);
}

int run_step(cjt_group_s *g, const Step &s, int pair, cudaStream_t st) {
    const GDesc *D = reinterpret_cast<const GDesc *>(g->d_tables);
    const unsigned char *T = g->d_tables + g->desc_bytes;
    switch (s.type) {
        case ST_ELEM: {
            const GTab *tab = reinterpret_cast<const GTab *>(T + s.tab);
            switch (s.op) {
                case OP_PACK_FWD: return launch_elem_prec<OP_PACK_FWD>(s.prec, D, tab, s.grid, st);
                case OP_PACK_INV: return launch_elem_prec<OP_PACK_INV>(s.prec, D, tab, s.grid, st);
                case OP_COMBINE_FWD: return launch_elem_prec<OP_COMBINE_FWD>(s.prec, D, tab, s.grid, st);
                case OP_COMBINE_INV: return launch_elem_prec<OP_COMBINE_INV>(s.prec, D, tab, s.grid, st);
                case OP_DCT_FINISH: return launch_elem<OP_DCT_FINISH, double2, double>(D, tab, s.grid, st);
                case OP_FRONT_PACK: return launch_elem<OP_FRONT_PACK, double2, double>(D, tab, s.grid, st);
                case OP_INV_G: return launch_elem<OP_INV_G, double2, double>(D, tab, s.grid, st);
            }
            return CJT_EINVAL;
        }
        case ST_REC: {
            const int *sel = reinterpret_cast<const int *>(T + s.tab);
            const int64_t *pre = reinterpret_cast<const int64_t *>(T + s.pre);
            switch (s.op) {
                case REC_K_FWD:
                    k_g_rec_fwd<<<(unsigned)((s.total * 32 + 127) / 128), 128, 0, st>>>(D, sel, pre, s.nsel, s.total);
                    break;
                case REC_K_INV:
                    k_g_rec_inv<<<(unsigned)((s.total + GRI_WARPS - 1) / GRI_WARPS), 32 * GRI_WARPS, 0, st>>>(
                        D, sel, pre, s.nsel, s.total);
                    break;
                case REC_K_FWD_STORED:
                    k_g_rec_fwd_stored<<<(unsigned)s.total, 32 * cjt_kern::SW, 0, st>>>(D, sel, pre, s.nsel);
                    break;
                case REC_K_INV_STORED:
                    k_g_rec_inv_stored<<<(unsigned)s.total, 32 * cjt_kern::SW, 0, st>>>(D, sel, pre, s.nsel);
                    break;
                default:
                    return CJT_EINVAL;
            }
            CJT_CUDA_TRY(cudaGetLastError());
            return CJT_OK;
        }
        case ST_REDUCE:
            if (s.op == 32)
                k_g_inv_reduce<32><<<(unsigned)s.grid, 32 * 32, 0, st>>>(D, reinterpret_cast<const GTab *>(T + s.tab));
            else
                k_g_inv_reduce<8><<<(unsigned)s.grid, 32 * 8, 0, st>>>(D, reinterpret_cast<const GTab *>(T + s.tab));
            CJT_CUDA_TRY(cudaGetLastError());
            return CJT_OK;
        case ST_FFT: {
            unsigned char *base = (unsigned char *)g->arena[pair];
            return cjt_fft_any(base + s.data, cjt_fft_scratch_elems(s.L, 1) ? base + s.scratch : nullptr, s.L, s.count,
                               s.tw, s.prec, st);
        }
        case ST_RECORD:
            CJT_CUDA_TRY(cudaEventRecord(g->ev[pair][s.event], st));
            return CJT_OK;
        case ST_WAIT:
            CJT_CUDA_TRY(cudaStreamWaitEvent(st, g->ev[pair][s.event], 0));
            return CJT_OK;
    }
    return CJT_EINVAL;
}

cudaEvent_t prof_event(cjt_group_s *g) {
    if (!g->prof_pool.empty()) {
        cudaEvent_t e = g->prof_pool.back();
        g->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// run_step, with an event pair around a launch step when `prof`
int run_step_p(cjt_group_s *g, const Step &s, int pair, cudaStream_t st, bool prof) {
    if (!prof || s.cat < 0) return run_step(g, s, pair, st);
    cudaEvent_t a = prof_event(g), b = prof_event(g);
    if (!a || !b) return CJT_ECUDA;
    CJT_CUDA_TRY(cudaEventRecord(a, st));
    int rc = run_step(g, s, pair, st);
    if (rc) return rc;
    CJT_CUDA_TRY(cudaEventRecord(b, st));
    g->prof_pending.push_back({s.cat, a, b});
    return CJT_OK;
}

int64_t step_kernels(const Step &s) {
    if (s.type == ST_ELEM || s.type == ST_REC || s.type == ST_REDUCE) return 1;
    if (s.type == ST_FFT) return fft_launches(s.L);
    return 0;
}

// A transform length class inside one wave: the member transforms' sequences, contiguous.
struct Cls {
    int64_t L = 0;
    int prec = 0;
    std::vector<int> members;   // descriptor indices
    std::vector<int64_t> seqs;  // sequences per member
    int64_t total = 0;          // sequences
    size_t off = 0;             // arena offset of the region
    const cjt_plan_s *tw_of = nullptr;
};

// Lays out one wave (descriptor indices `items`, plans `owner`) in an arena and appends
// its steps.  Returns the arena bytes it needs.
int64_t plan_wave(cjt_group_s *g, const std::vector<int> &items, const std::vector<const cjt_plan_s *> &owner,
                  const std::vector<int> &dirs, WavePlan &wv, bool emit) {
    // classes: forward ASY (L, prec), inverse ASY (L, prec), forward DCT (2G), inverse front (4G)
    std::vector<Cls> asy_f, asy_i, dct, front;
    auto add = [](std::vector<Cls> &v, int64_t L, int prec, int t, int64_t seqs, const cjt_plan_s *p) {
        for (auto &c : v)
            if (c.L == L && c.prec == prec) {
                c.members.push_back(t);
                c.seqs.push_back(seqs);
                c.total += seqs;
                return;
            }
        Cls c;
        c.L = L;
        c.prec = prec;
        c.members.push_back(t);
        c.seqs.push_back(seqs);
        c.total = seqs;
        c.tw_of = p;
        v.push_back(c);
    };
    for (int t : items) {
        const GDesc &d = g->desc[t];
        const cjt_plan_s *p = owner[t];
        if (dirs[t] == CJT_FWD) {
            if (d.npair > 0) add(asy_f, d.L, p->prec_asy, t, d.npair, p);
            add(dct, 2 * d.G, PREC_F64, t, 1, p);
        } else {
            if (d.npair > 0) add(asy_i, d.L, p->prec_asy, t, d.npair, p);
            add(front, 2 * d.Ng, PREC_F64, t, 1, p);
        }
    }
    int64_t off = 0;
    int64_t scr_side = 0, scr_main = 0;
    auto place = [&](std::vector<Cls> &v, int64_t &scr) {
        for (auto &c : v) {
            const int64_t bytes = c.total * c.L * prec_cbytes(c.prec);
            c.off = (size_t)off;
            off = align256(off + bytes);
            if (cjt_fft_scratch_elems(c.L, 1)) scr = std::max(scr, bytes);
        }
    };
    place(asy_f, scr_side);
    place(asy_i, scr_side);
    place(dct, scr_main);
    place(front, scr_main);
    const size_t off_scr_side = (size_t)off;
    off = align256(off + scr_side);
    const size_t off_scr_main = (size_t)off;
    off = align256(off + scr_main);
    // per-transform buffers: recurrence partials, y and g (inverse)
    std::vector<size_t> off_part(items.size()), off_y(items.size()), off_g(items.size());
    for (size_t k = 0; k < items.size(); ++k) {
        const cjt_plan_s *p = owner[items[k]];
        const bool f = dirs[items[k]] == CJT_FWD;
        const GridWork &gw = f ? p->fw : p->iv;
        off_part[k] = (size_t)off;
        off = align256(off + 8 * std::max<int64_t>(gw.npartials, 1));
        if (!f) {
            off_y[k] = (size_t)off;
            off = align256(off + 8 * (p->N + 1));
            off_g[k] = (size_t)off;
            off = align256(off + 8 * (gw.Ng + 1));
        }
    }
    if (!emit) return off;

    // workspace pointers of the descriptors
    unsigned char *base = (unsigned char *)g->arena[wv.pair];
    auto seq_ptrs = [&](std::vector<Cls> &v, bool to_fft) {
        for (auto &c : v) {
            int64_t pos = 0;
            for (size_t k = 0; k < c.members.size(); ++k) {
                GDesc &d = g->desc[c.members[k]];
                unsigned char *at = base + c.off + pos * c.L * prec_cbytes(c.prec);
                if (to_fft) d.fft = at;
                else d.dct = reinterpret_cast<double2 *>(at);
                pos += c.seqs[k];
            }
        }
    };
    seq_ptrs(asy_f, true);
    seq_ptrs(asy_i, true);
    seq_ptrs(dct, false);
    seq_ptrs(front, false);
    for (size_t k = 0; k < items.size(); ++k) {
        GDesc &d = g->desc[items[k]];
        d.part = reinterpret_cast<double *>(base + off_part[k]);
        if (dirs[items[k]] != CJT_FWD) {
            d.y = reinterpret_cast<double *>(base + off_y[k]);
            d.g = reinterpret_cast<double *>(base + off_g[k]);
        }
    }
    auto ffts = [&](std::vector<Step> &out, const std::vector<Cls> &v, size_t scr, int cat) {
        for (auto &c : v) {
            Step s;
            s.type = ST_FFT;
            s.cat = cat;
            s.data = c.off;
            s.scratch = scr;
            s.L = c.L;
            s.count = c.total;
            s.prec = c.prec;
            s.tw = c.tw_of->twiddles(c.prec);
            out.push_back(s);
        }
    };
    // selections
    std::vector<int> fwd, inv, fwd64, fwd32, inv64, inv32, fwd_rec, fwd_sto, inv_rec, inv_sto;
    for (int t : items) {
        const cjt_plan_s *p = owner[t];
        const bool f = dirs[t] == CJT_FWD;
        const bool f32 = p->prec_asy == PREC_F32;
        const bool stored = (f ? p->fw.d_E : p->iv.d_E) != nullptr;
        (f ? fwd : inv).push_back(t);
        if (f) (f32 ? fwd32 : fwd64).push_back(t);
        else (f32 ? inv32 : inv64).push_back(t);
        if (f) (stored ? fwd_sto : fwd_rec).push_back(t);
        else (stored ? inv_sto : inv_rec).push_back(t);
    }
    // main: inverse front end
    add_elem<OP_FRONT_PACK>(g, wv.main_front, inv, PREC_F64);
    ffts(wv.main_front, front, off_scr_main, CJT_BSTAGE_FFT_DCT);
    add_elem<OP_INV_G>(g, wv.main_front, inv, PREC_F64);
    wv.main_front.push_back(ev_step(ST_RECORD, EV_FRONT));
    // side: forward ASY, then (after the front end) inverse ASY
    add_elem<OP_PACK_FWD>(g, wv.side, fwd64, PREC_F64);
    add_elem<OP_PACK_FWD>(g, wv.side, fwd32, PREC_F32);
    ffts(wv.side, asy_f, off_scr_side, CJT_BSTAGE_FFT_ASY);
    if (!inv.empty()) wv.side.push_back(ev_step(ST_WAIT, EV_FRONT));
    add_elem<OP_PACK_INV>(g, wv.side, inv64, PREC_F64);
    add_elem<OP_PACK_INV>(g, wv.side, inv32, PREC_F32);
    ffts(wv.side, asy_i, off_scr_side, CJT_BSTAGE_FFT_ASY);
    wv.side.push_back(ev_step(ST_RECORD, EV_SIDE));
    // main: recurrences and the reduction
    add_rec(g, wv.main_rec, fwd_sto, REC_K_FWD_STORED);
    add_rec(g, wv.main_rec, fwd_rec, REC_K_FWD);
    add_rec(g, wv.main_rec, inv_sto, REC_K_INV_STORED);
    add_rec(g, wv.main_rec, inv_rec, REC_K_INV);
    add_reduce(g, wv.main_rec, inv);
    // main: combines and the final DCT-I
    wv.main_post.push_back(ev_step(ST_WAIT, EV_SIDE));
    add_elem<OP_COMBINE_FWD>(g, wv.main_post, fwd64, PREC_F64);
    add_elem<OP_COMBINE_FWD>(g, wv.main_post, fwd32, PREC_F32);
    ffts(wv.main_post, dct, off_scr_main, CJT_BSTAGE_FFT_DCT);
    add_elem<OP_DCT_FINISH>(g, wv.main_post, fwd, PREC_F64);
    add_elem<OP_COMBINE_INV>(g, wv.main_post, inv64, PREC_F64);
    add_elem<OP_COMBINE_INV>(g, wv.main_post, inv32, PREC_F32);
    return off;
}

GDesc make_desc(const cjt_plan_s *p, int dir, const double *in, double *out) {
    GDesc d;
    memset(&d, 0, sizeof(d));
    const bool f = dir == CJT_FWD;
    const GridWork &gw = f ? p->fw : p->iv;
    d.N = p->N;
    d.G = p->Gf;
    d.Ng = gw.Ng;
    d.L = f ? p->Lf : p->Li;
    d.q = std::max(cjt_odd_radix(d.L), 1);
    d.logL = ilog2_exact(std::max<int64_t>(d.L / d.q, 1));
    d.M = p->M;
    d.nblk = gw.nblk;
    d.nq = gw.nblk * p->M;
    d.npair = f ? p->npair_f : p->npair_i;
    d.seg_len = p->seg_len;
    d.rt = p->rt;
    d.items = gw.d_items;
    d.nitems = gw.nitems;
    d.states = gw.d_states;
    d.E = gw.d_E;
    d.rowk = gw.d_rowk;
    d.row_base = gw.d_row_base;
    d.row_nseg = gw.d_row_nseg;
    d.scale = gw.d_scale;
    d.u = gw.d_u;
    d.v = gw.d_v;
    d.Cnm = p->d_Cnm;
    d.w = p->d_w;
    d.s_n = p->d_s;
    d.box = gw.d_box;
    d.seg_ptr = gw.d_seg_ptr;
    d.seg_out = gw.d_seg_out;
    d.seg_b = gw.d_seg_b;
    d.in = in;
    d.out = out;
    return d;
}

}  // namespace

int cjt_group_create(cjt_group_t *out, const std::vector<int> &idx, const cjt_plan_t *plans, const int8_t *dir,
                     const int64_t *offsets, const double *in, double *outp, int64_t arena_budget) {
    *out = nullptr;
    if (idx.empty()) return CJT_OK;
    cjt_group_s *g = new cjt_group_s();
    auto fail = [&](int rc) {
        cjt_group_destroy(g);
        return rc;
    };
    CJT_CUDA_TRY(cudaGetDevice(&g->dev));
    const int n = (int)idx.size();
    std::vector<const cjt_plan_s *> owner(n);
    std::vector<int> dirs(n);
    std::vector<double> cost(n);
    for (int k = 0; k < n; ++k) {
        const int t = idx[k];
        owner[k] = plans[t];
        dirs[k] = dir[t];
        g->desc.push_back(make_desc(plans[t], dir[t], in + offsets[t], outp + offsets[t]));
        cost[k] = item_cost(plans[t], dir[t]);
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // waves: items by decreasing cost, each wave's workspace within the budget.  The running
    // estimate bounds the exact layout of plan_wave from above: every buffer with its
    // alignment, and the four-step scratch of each stream as large as its largest class.
    std::vector<std::vector<int>> waves;
    {
        struct Acc { int kind; int64_t L; int prec; int64_t bytes; };
        std::vector<int> cur;
        std::vector<Acc> cls;
        int64_t sum = 0;
        auto est = [&]() {
            int64_t scr[2] = {0, 0};
            for (auto &c : cls)
                if (cjt_fft_scratch_elems(c.L, 1)) scr[c.kind >> 1] = std::max(scr[c.kind >> 1], c.bytes);
            return sum + 256 * (int64_t)cls.size() + scr[0] + scr[1] + 1024;
        };
        auto add_cls = [&](std::vector<Acc> &v, int kind, int64_t L, int prec, int64_t bytes) {
            for (auto &c : v)
                if (c.kind == kind && c.L == L && c.prec == prec) { c.bytes += bytes; return; }
            v.push_back({kind, L, prec, bytes});
        };
        for (int k : order) {
            const cjt_plan_s *p = owner[k];
            const GDesc &d = g->desc[k];
            const bool f = dirs[k] == CJT_FWD;
            const GridWork &gw = f ? p->fw : p->iv;
            const int64_t asy = (int64_t)d.npair * d.L * prec_cbytes(p->prec_asy);
            const int64_t dl = f ? 2 * d.G : d.L;
            const int64_t own = align256(8 * std::max<int64_t>(gw.npartials, 1)) +
                                (f ? 0 : align256(8 * (p->N + 1)) + align256(8 * (gw.Ng + 1)));
            const int64_t add = asy + 16 * dl + own + 512;
            std::vector<Acc> trial = cls;
            if (d.npair > 0) add_cls(trial, f ? 0 : 1, d.L, p->prec_asy, asy);
            add_cls(trial, f ? 2 : 3, dl, PREC_F64, 16 * dl);
            std::swap(trial, cls);
            sum += add;
            if (!cur.empty() && est() > arena_budget) {
                waves.push_back(cur);
                cur.clear();
                cls.clear();
                sum = add;
                if (d.npair > 0) add_cls(cls, f ? 0 : 1, d.L, p->prec_asy, asy);
                add_cls(cls, f ? 2 : 3, dl, PREC_F64, 16 * dl);
            }
            cur.push_back(k);
        }
        if (!cur.empty()) waves.push_back(cur);
    }
    // arenas: wave w uses arena w % 2, sized for the largest of its waves
    for (size_t w = 0; w < waves.size(); ++w) {
        WavePlan tmp;
        const int64_t need = plan_wave(g, waves[w], owner, dirs, tmp, false);
        g->arena_bytes[w & 1] = std::max(g->arena_bytes[w & 1], need);
    }
    for (int a = 0; a < 2; ++a) {
        if (!g->arena_bytes[a]) continue;
        cudaError_t e = cudaMalloc(&g->arena[a], (size_t)g->arena_bytes[a]);
        if (e != cudaSuccess) {
            cjt_internal_set_cuda_error(e, "cudaMalloc");
            return fail(CJT_ENOMEM);
        }
    }
    for (size_t w = 0; w < waves.size(); ++w) {
        WavePlan wv;
        wv.pair = (int)(w & 1);
        plan_wave(g, waves[w], owner, dirs, wv, true);
        g->waves.push_back(std::move(wv));
    }
    // descriptors and tables in one device buffer
    g->desc_bytes = (size_t)align256((int64_t)(g->desc.size() * sizeof(GDesc)));
    const size_t total = g->desc_bytes + g->tables.size();
    cudaError_t e = cudaMalloc((void **)&g->d_tables, total);
    if (e != cudaSuccess) {
        cjt_internal_set_cuda_error(e, "cudaMalloc");
        return fail(CJT_ENOMEM);
    }
    if (cudaMemcpy(g->d_tables, g->desc.data(), g->desc.size() * sizeof(GDesc), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        (!g->tables.empty() && cudaMemcpy(g->d_tables + g->desc_bytes, g->tables.data(), g->tables.size(),
                                          cudaMemcpyHostToDevice) != cudaSuccess))
        return fail(CJT_ECUDA);
    // streams (side: the highest priority, as the single-transform path's asymptotic chain)
    int least = 0, greatest = 0;
    CJT_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (int a = 0; a < 2; ++a) {
        if (cudaStreamCreateWithPriority(&g->main[a], cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaStreamCreateWithPriority(&g->side[a], cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&g->join[a], cudaEventDisableTiming) != cudaSuccess)
            return fail(CJT_ECUDA);
        for (int k = 0; k < EV_N; ++k)
            if (cudaEventCreateWithFlags(&g->ev[a][k], cudaEventDisableTiming) != cudaSuccess) return fail(CJT_ECUDA);
    }
    if (cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) return fail(CJT_ECUDA);
    for (auto &wv : g->waves)
        for (auto *v : {&wv.main_front, &wv.side, &wv.main_rec, &wv.main_post})
            for (auto &s : *v) g->kernels += step_kernels(s);
    *out = g;
    return CJT_OK;
}

// CJT_GROUP_TRACE=1: one line per launch step on stderr (stream, kind, op, length class,
// sequences or work items, CTAs), in issue order, to read beside a profiler's launch list
static void trace_step(const Step &s, int wave, const char *stream) {
    static const bool on = getenv("CJT_GROUP_TRACE") != nullptr;
    if (!on || s.type == ST_RECORD || s.type == ST_WAIT) return;
    static const char *names[] = {"elem", "rec", "reduce", "fft"};
    fprintf(stderr, "[cjt group] wave %d %s %s op=%d prec=%d L=%lld count=%lld grid=%lld total=%lld\n", wave, stream,
            names[s.type], s.op, s.prec, (long long)s.L, (long long)s.count, (long long)s.grid, (long long)s.total);
}

int cjt_group_issue(cjt_group_t g, cudaStream_t origin, bool prof) {
    if (!g) return CJT_OK;
    CJT_CUDA_TRY(cudaEventRecord(g->fork, origin));
    bool used[2] = {false, false};
    for (auto &wv : g->waves) {
        const int a = wv.pair;
        // profiled: every launch on one stream, so that each event pair times its launch alone
        cudaStream_t m = prof ? g->main[0] : g->main[a], s = prof ? g->main[0] : g->side[a];
        const int ua = prof ? 0 : a;
        if (!used[ua]) {
            CJT_CUDA_TRY(cudaStreamWaitEvent(m, g->fork, 0));
            used[ua] = true;
        }
        // the side stream starts with its wave
        CJT_CUDA_TRY(cudaEventRecord(g->ev[a][EV_FORK], m));
        CJT_CUDA_TRY(cudaStreamWaitEvent(s, g->ev[a][EV_FORK], 0));
        int rc;
        const int wi = (int)(&wv - g->waves.data());
        for (auto &st : wv.main_front) {
            trace_step(st, wi, "main");
            if ((rc = run_step_p(g, st, a, m, prof))) return rc;
        }
        for (auto &st : wv.side) {
            trace_step(st, wi, "side");
            if ((rc = run_step_p(g, st, a, s, prof))) return rc;
        }
        for (auto &st : wv.main_rec) {
            trace_step(st, wi, "main");
            if ((rc = run_step_p(g, st, a, m, prof))) return rc;
        }
        for (auto &st : wv.main_post) {
            trace_step(st, wi, "main");
            if ((rc = run_step_p(g, st, a, m, prof))) return rc;
        }
    }
    for (int a = 0; a < 2; ++a) {
        if (!used[a]) continue;
        CJT_CUDA_TRY(cudaEventRecord(g->join[a], g->main[a]));
        CJT_CUDA_TRY(cudaStreamWaitEvent(origin, g->join[a], 0));
    }
    return CJT_OK;
}

int cjt_group_profile(cjt_group_t g, double *ms, int64_t *counts, int n) {
    if (!g) return CJT_OK;
    int rc = CJT_OK;
    for (auto &r : g->prof_pending) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) {
            cjt_internal_set_cuda_error(e, "cudaEventElapsedTime");
            rc = CJT_ECUDA;
        }
        if (r.cat < n) {
            if (ms) ms[r.cat] += t;
            if (counts) counts[r.cat] += 1;
        }
        g->prof_pool.push_back(r.a);
        g->prof_pool.push_back(r.b);
    }
    g->prof_pending.clear();
    return rc;
}

int64_t cjt_group_kernels(cjt_group_t g) { return g ? g->kernels : 0; }
int64_t cjt_group_arena_bytes(cjt_group_t g) { return g ? g->arena_bytes[0] + g->arena_bytes[1] : 0; }
int cjt_group_waves(cjt_group_t g) { return g ? (int)g->waves.size() : 0; }

void cjt_group_destroy(cjt_group_t g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->d_tables) cudaFree(g->d_tables);
    for (int a = 0; a < 2; ++a) {
        if (g->arena[a]) cudaFree(g->arena[a]);
        if (g->main[a]) cudaStreamDestroy(g->main[a]);
        if (g->side[a]) cudaStreamDestroy(g->side[a]);
        if (g->join[a]) cudaEventDestroy(g->join[a]);
        for (int k = 0; k < EV_N; ++k)
            if (g->ev[a][k]) cudaEventDestroy(g->ev[a][k]);
    }
    if (g->fork) cudaEventDestroy(g->fork);
    for (auto &r : g->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : g->prof_pool) cudaEventDestroy(e);
    delete g;
}
