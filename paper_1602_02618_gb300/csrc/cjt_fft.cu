// Shared-memory radix-4 FFT for sm_103a (FP64, FP32 and double-float), used for the
// diagonally scaled DCT-I/DST-I of the asymptotic blocks (Eq. "PNASY"), the
// final inverse DCT-I (Sec. 2) and the inverse transform's front end and
// transposed blocks (Eq. "CJTT").
//
// X[k] = sum_n x[n] exp(-2 pi i n k / L), L a power of two, in place, batched.
//   L <= 4096: one pass, each CTA transforms `tile` sequences held in shared memory.
//   L  > 4096: four-step  L = L1 * L2  (two passes through global memory / L2):
//     pass A: L2 columns of length L1 (stride L2), twiddle omega_L^{n2 k1}, store T[k1][n2]
//     pass B: L1 rows of length L2 (contiguous), store X[k1 + L1 k2]
// Sub-transforms are decimation-in-frequency radix-4 stages (one radix-2 stage
// last when log2 is odd) on a padded [column][element] shared-memory tile,
// with twiddles read from plan-owned tables computed by sincospi (exact argument
// reduction): omega_{Ltab}^j, and per-stage copies laid out so that a warp's loads
// are contiguous (Twiddles::stw).  FP64 transforms with the TwFma tables run the
// same stages in decimation-in-time order instead (digit-reversed load, one radix-2
// stage first when log2 is odd), with the twiddles applied before each butterfly in
// fused multiply-add form: 22 FP64 operations per radix-4 butterfly instead of 28, on
// a device whose FP64 pipe is the limit.
//
// Lengths that are not powers of two (N not a power of two) go through
// Bluestein's chirp-z form on top of the power-of-two transform.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>

#include "cjt_df.cuh"
#include "cjt_internal.cuh"

int cjt_fft_prime();

namespace {

// Launch configuration of the transforms of one (precision, log2 L) class, set by the
// autotuner through cjt_fft_set_config and read when a transform is enqueued:
//   ctas     CTAs per SM the tile size aims at when there is enough work (tiles are powers
//            of two, at most 64 columns and ~64 KB of shared memory);
//   split    four-step factorisation L = L1 L2: 0 -> L1 = 2^ceil(log2 L / 2), 1 -> 2^floor,
//            2 -> 2^(floor - 1) (narrower first-pass columns: each CTA then reads more
//            adjacent columns, whole 64-byte segments of the strided first pass);
//   single   largest log2 L transformed in one pass in shared memory (12 or 13).
// ctas changes only the work split between CTAs; split and single change the order of
// the arithmetic (results differ in rounding), so one configuration holds for a process.
struct FftCfg {
    std::atomic<int> ctas{4}, split{0}, single{12};
};
FftCfg g_fft_cfg[3][32];

// log2 L1 of the four-step split of a length 2^logL; a split whose second pass would exceed
// 2^max2 points falls back to split 0
inline int four_step_log1(int logL, int split, int max2) {
    const int l1 = split == 2 ? logL / 2 - 1 : split == 1 ? logL / 2 : (logL + 1) / 2;
    return (l1 >= 1 && logL - l1 <= max2) ? l1 : (logL + 1) / 2;
}

struct dfloat {};   // tag of the double-float transform (complex type dfc)
template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<dfloat> { using t = dfc; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = fma(a.x, b.x, -a.y * b.y);
    r.y = fma(a.x, b.y, a.y * b.x);
    return r;
}
// multiply by -i
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
template <typename V> __device__ __forceinline__ V czero() { V r; r.x = 0; r.y = 0; return r; }
template <typename V> __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
// times a power of two (exact)
template <typename V> __device__ __forceinline__ V cscale(V a, double s) {
    a.x = a.x * (decltype(a.x))s;
    a.y = a.y * (decltype(a.y))s;
    return a;
}
// sums inside a butterfly that feed another sum at once (double-float: not renormalised)
template <typename V> __device__ __forceinline__ V cadd_t(V a, V b) { return cadd(a, b); }
template <typename V> __device__ __forceinline__ V csub_t(V a, V b) { return csub(a, b); }
template <> __device__ __forceinline__ dfc cadd(dfc a, dfc b) { return dfc_add(a, b); }
template <> __device__ __forceinline__ dfc cadd_t(dfc a, dfc b) { return dfc_add_nr(a, b); }
template <> __device__ __forceinline__ dfc csub_t(dfc a, dfc b) { return dfc_sub_nr(a, b); }
template <> __device__ __forceinline__ dfc csub(dfc a, dfc b) { return dfc_sub(a, b); }
template <> __device__ __forceinline__ dfc cmul(dfc a, dfc b) { return dfc_mul(a, b); }
template <> __device__ __forceinline__ dfc cmul_mi(dfc a) { return dfc_mul_mi(a); }
template <> __device__ __forceinline__ dfc czero<dfc>() { return dfc_zero(); }
template <> __device__ __forceinline__ dfc cconj(dfc a) { return dfc_conj(a); }
template <> __device__ __forceinline__ dfc cscale(dfc a, double s) { return dfc_scale_pow2(a, (float)s); }

constexpr int FFT_THREADS = 256;
constexpr int SMEM_PAD = 1;

// Shared-memory position of element e of a column: the low three bits are XORed with a
// fold of the higher bits.  A bijection on [0, Ls) that spreads the accesses that would
// otherwise share banks (16-byte elements, eight per 128-byte row): the digit-reversed
// read-out and the last radix-4 / radix-2 stages.
__device__ __forceinline__ int swz(int e) { return e ^ (((e >> 3) ^ (e >> 6) ^ (e >> 9)) & 7); }

// frequency k -> its position after the DIF stages: the base-4 digits of k's low
// 2*floor(logLs/2) bits in reverse order (bit reversal, then the two bits of each digit
// swapped back), and for odd logLs the top (radix-2) bit of k at weight 1
__device__ __forceinline__ int dif_revinv(int k, int logLs) {
    const int d2 = logLs & ~1;
    if (d2 == 0) return k;
    unsigned r = __brev((unsigned)k & ((1u << d2) - 1u)) >> (32 - d2);
    r = ((r & 0x55555555u) << 1) | ((r >> 1) & 0x55555555u);
    return (logLs & 1) ? (int)((r << 1) | ((unsigned)k >> d2)) : (int)r;
}

constexpr int FFT_U = 4;   // global loads (and twiddle loads) in flight per thread in the load/store phases

// One radix-4 decimation-in-time butterfly on z_j = w_j x_j (w_0 = 1) with the TwFma
// form of w_1..w_3: X_p = sum_j z_j (-i)^{jp}.
__device__ __forceinline__ void dit4_fma(double2 x0, double2 x1, double2 x2, double2 x3, const TwFma &w,
                                         double2 &X0, double2 &X1, double2 &X2, double2 &X3) {
    auto rot = [](double2 x, bool sw, double t, double &e0, double &e1) {
        const double u0 = sw ? x.y : x.x, u1 = sw ? x.x : x.y;
        e0 = fma(-t, u1, u0);
        e1 = fma(t, u0, u1);
    };
    double e01, e11, e02, e12, e03, e13;
    rot(x1, w.flags & 1, w.t1, e01, e11);
    rot(x2, w.flags & 2, w.t2, e02, e12);
    rot(x3, w.flags & 4, w.t3, e03, e13);
    // a, b = x0 +- w2 x2;  (e, f) sigma_1 = w1 x1 +- w3 x3, componentwise
    const double ax = fma(w.s2x, e02, x0.x), ay = fma(w.s2y, e12, x0.y);
    const double bx = fma(-w.s2x, e02, x0.x), by = fma(-w.s2y, e12, x0.y);
    const double ex = fma(w.rx, e03, e01), ey = fma(w.ry, e13, e11);
    const double fx = fma(-w.rx, e03, e01), fy = fma(-w.ry, e13, e11);
    X0 = make_double2(fma(w.s1x, ex, ax), fma(w.s1y, ey, ay));      // a + c
    X2 = make_double2(fma(-w.s1x, ex, ax), fma(-w.s1y, ey, ay));    // a - c
    X1 = make_double2(fma(w.s1y, fy, bx), fma(-w.s1x, fx, by));     // b - i d
    X3 = make_double2(fma(-w.s1y, fy, bx), fma(w.s1x, fx, by));     // b + i d
}

template <typename R, bool DIT>
__global__ void __launch_bounds__(FFT_THREADS, 4)
k_fft_sub(const typename cplx<R>::t *__restrict__ in, typename cplx<R>::t *__restrict__ out, int logLs,
          int64_t ncols, int tile, int64_t in_es, int64_t in_cs, int64_t in_ts, int64_t out_ks, int64_t out_cs,
          int64_t out_ts, const typename cplx<R>::t *__restrict__ tw, int logLtab, int post_log,
          const typename cplx<R>::t *__restrict__ stw, const TwFma *__restrict__ fmat) {
    using V = typename cplx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s = reinterpret_cast<V *>(smem_raw);
    const int Ls = 1 << logLs;
    const int ld = Ls + SMEM_PAD;
    const int64_t c0 = (int64_t)blockIdx.x * tile;
    const int64_t t = blockIdx.y;
    const int ncl = (int)min((int64_t)tile, ncols - c0);
    const V *src = in + t * in_ts + c0 * in_cs;
    V *dst = out + t * out_ts + c0 * out_cs;

    // load (natural order); lanes run along the contiguous dimension; FFT_U loads in flight
    const int total = ncl * Ls;
    const bool pow2c = (ncl & (ncl - 1)) == 0;
    const int lgc = __ffs(ncl) - 1;
    for (int i0 = threadIdx.x; i0 < total; i0 += FFT_U * blockDim.x) {
        V v[FFT_U];
        int at[FFT_U];
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            const int idx = i0 + u * blockDim.x;
            at[u] = -1;
            if (idx < total) {
                int c, e;
                int64_t g;
                if (in_es == 1) {
                    e = idx & (Ls - 1);
                    c = idx >> logLs;
                    g = c * in_cs + e;
                } else {
                    c = pow2c ? (idx & (ncl - 1)) : idx % ncl;
                    e = pow2c ? (idx >> lgc) : idx / ncl;
                    g = c * in_cs + (int64_t)e * in_es;
                }
                at[u] = c * ld + swz(DIT ? dif_revinv(e, logLs) : e);
                v[u] = src[g];
            }
        }
#pragma unroll
        for (int u = 0; u < FFT_U; ++u)
            if (at[u] >= 0) s[at[u]] = v[u];
    }
    __syncthreads();

    if constexpr (DIT) {
        // decimation in time: the input sits at digit-reversed positions; a radix-2 stage
        // first when logLs is odd, then radix-4 stages of growing block length Lb, whose
        // quarter q + j Lb/4 holds the j-th sub-transform at q (twiddle omega_Lb^{jq})
        int lb = 0;
        if (logLs & 1) {
            const int nb2 = Ls >> 1;
            for (int idx = threadIdx.x; idx < ncl * nb2; idx += blockDim.x) {
                const int c = idx >> (logLs - 1), j = idx & (nb2 - 1);
                V *col = s + c * ld;
                const int i0 = swz(2 * j), i1 = swz(2 * j + 1);
                V x0 = col[i0], x1 = col[i1];
                col[i0] = cadd(x0, x1);
                col[i1] = csub(x0, x1);
            }
            __syncthreads();
            lb = 1;
        }
        const int nb4 = Ls >> 2;
        for (lb += 2; lb <= logLs; lb += 2) {
            const int Lb = 1 << lb, h = Lb >> 2;
            const TwFma *tb = fmat + twfma_base(lb);
            for (int idx = threadIdx.x; idx < ncl * nb4; idx += blockDim.x) {
                const int c = idx >> (logLs - 2), j = idx & (nb4 - 1);
                const int blk = j >> (lb - 2), q = j & (h - 1);
                V *col = s + c * ld;
                const int e0 = blk * Lb + q;
                const int i0 = swz(e0), i1 = swz(e0 + h), i2 = swz(e0 + 2 * h), i3 = swz(e0 + 3 * h);
                const V x0 = col[i0], x1 = col[i1], x2 = col[i2], x3 = col[i3];
                V X0, X1, X2, X3;
                if (h == 1) {   // Lb = 4: all twiddles are 1
                    const V a = cadd(x0, x2), b = csub(x0, x2), cc = cadd(x1, x3), d = csub(x1, x3);
                    X0 = cadd(a, cc);
                    X2 = csub(a, cc);
                    X1 = cadd(b, cmul_mi(d));
                    X3 = csub(b, cmul_mi(d));
                } else {
                    dit4_fma(x0, x1, x2, x3, tb[q], X0, X1, X2, X3);
                }
                col[i0] = X0; col[i1] = X1; col[i2] = X2; col[i3] = X3;
            }
            __syncthreads();
        }
    } else {
        // radix-4 DIF stages
        const int nb4 = Ls >> 2;
        int lb = logLs;
        while (lb >= 2) {
            const int Lb = 1 << lb, h = Lb >> 2;
            const int twstep_log = logLtab - lb;  // omega_{Lb}^j = tw[j << (logLtab - lb)]
            for (int idx = threadIdx.x; idx < ncl * nb4; idx += blockDim.x) {
                const int c = idx >> (logLs - 2), j = idx & (nb4 - 1);   // nb4 = Ls/4
                int blk = j >> (lb - 2), n0 = j & (h - 1);
                V *col = s + c * ld;
                const int e0 = blk * Lb + n0;
                const int i0 = swz(e0), i1 = swz(e0 + h), i2 = swz(e0 + 2 * h), i3 = swz(e0 + 3 * h);
                V x0 = col[i0], x1 = col[i1], x2 = col[i2], x3 = col[i3];
                V t0 = cadd_t(x0, x2), t1 = csub_t(x0, x2), t2 = cadd_t(x1, x3), t3 = cmul_mi(csub_t(x1, x3));
                V y0 = cadd(t0, t2), y2 = csub(t0, t2), y1 = cadd(t1, t3), y3 = csub(t1, t3);
                if (n0 != 0) {
                    if (stw) {
                        const V *w = stw + stw_base(lb) + n0;
                        y1 = cmul(y1, w[0]);
                        y2 = cmul(y2, w[h]);
                        y3 = cmul(y3, w[2 * h]);
                    } else {
                        y1 = cmul(y1, tw[(int64_t)n0 << twstep_log]);
                        y2 = cmul(y2, tw[(int64_t)(2 * n0) << twstep_log]);
                        y3 = cmul(y3, tw[(int64_t)(3 * n0) << twstep_log]);
                    }
                }
                col[i0] = y0; col[i1] = y1; col[i2] = y2; col[i3] = y3;
            }
            __syncthreads();
            lb -= 2;
        }
        if (lb == 1) {
            const int nb2 = Ls >> 1;
            for (int idx = threadIdx.x; idx < ncl * nb2; idx += blockDim.x) {
                const int c = idx >> (logLs - 1), j = idx & (nb2 - 1);   // nb2 = Ls/2
                V *col = s + c * ld;
                const int i0 = swz(2 * j), i1 = swz(2 * j + 1);
                V x0 = col[i0], x1 = col[i1];
                col[i0] = cadd(x0, x1);
                col[i1] = csub(x0, x1);
            }
            __syncthreads();
        }
    }

    // store in natural frequency order, optional four-step twiddle omega_{2^post_log}^{c k};
    // FFT_U twiddle loads in flight
    for (int i0 = threadIdx.x; i0 < total; i0 += FFT_U * blockDim.x) {
        V v[FFT_U], w[FFT_U];
        int64_t at[FFT_U];
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            const int idx = i0 + u * blockDim.x;
            at[u] = -1;
            if (idx < total) {
                int c, k;
                if (out_ks == 1) {
                    k = idx & (Ls - 1);
                    c = idx >> logLs;
                    at[u] = c * out_cs + k;
                } else {
                    c = pow2c ? (idx & (ncl - 1)) : idx % ncl;
                    k = pow2c ? (idx >> lgc) : idx / ncl;
                    at[u] = c * out_cs + (int64_t)k * out_ks;
                }
                v[u] = s[c * ld + swz(DIT ? k : dif_revinv(k, logLs))];
                if (post_log >= 0) {
                    const int64_t ex = ((c0 + c) * (int64_t)k) & ((1LL << post_log) - 1);
                    w[u] = tw[ex << (logLtab - post_log)];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < FFT_U; ++u) {
            if (at[u] < 0) continue;
            dst[at[u]] = post_log >= 0 ? cmul(v[u], w[u]) : v[u];
        }
    }
}

int ilog2(int64_t v) {
    int r = 0;
    while ((1LL << r) < v) ++r;
    return r;
}

template <typename R>
int launch_sub(const void *in, void *out, int logLs, int64_t ncols, int64_t batch, int64_t in_es, int64_t in_cs,
               int64_t in_ts, int64_t out_ks, int64_t out_cs, int64_t out_ts, const void *tw, int logLtab,
               int post_log, const void *stw, const void *fmat, cudaStream_t st, int ctas) {
    using V = typename cplx<R>::t;
    const int Ls = 1 << logLs;
    // Columns per CTA: at most ~64 KB of shared memory (32 KB double-float), and few
    // enough that the launch spreads over every SM of the current device.
    int prc = cjt_fft_prime();
    if (prc) return prc;
    static std::atomic<int> sms_of[64];
    int dev = 0;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CJT_EUNSUPPORTED;
    int sms = sms_of[dev].load(std::memory_order_relaxed);
    if (!sms) {
        int v = 0;
        CJT_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        sms = v > 0 ? v : 152;
        sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    // double-float: half the tile, so that more CTAs (and warps) share an SM
    const int64_t budget_elems = (int64_t)((std::is_same<R, dfloat>::value ? 32768 : 65536) / sizeof(V));
    int64_t tile64 = std::min<int64_t>(std::min<int64_t>(ncols, 64), std::max<int64_t>(1, budget_elems / Ls));
    // at least `ctas` CTAs per SM when there is enough work (fewer, larger CTAs leave a
    // partly empty last wave), and a power of two (shift/mask indexing)
    tile64 = std::min<int64_t>(tile64, std::max<int64_t>(1, ncols * batch / ((int64_t)ctas * sms)));
    int tile = 1;
    while ((int64_t)tile * 2 <= tile64) tile *= 2;
    size_t smem = (size_t)tile * (Ls + SMEM_PAD) * sizeof(V);
    const int threads = (int)std::min<int64_t>(FFT_THREADS, std::max<int64_t>(32, ((int64_t)tile * Ls / 4 + 31) / 32 * 32));
    dim3 grid((unsigned)((ncols + tile - 1) / tile), (unsigned)batch);
    bool launched = false;
    if constexpr (std::is_same<R, double>::value) {
        if (fmat) {
            k_fft_sub<R, true><<<grid, threads, smem, st>>>((const V *)in, (V *)out, logLs, ncols, tile, in_es,
                                                            in_cs, in_ts, out_ks, out_cs, out_ts, (const V *)tw,
                                                            logLtab, post_log, (const V *)stw, (const TwFma *)fmat);
            launched = true;
        }
    }
    if (!launched)
        k_fft_sub<R, false><<<grid, threads, smem, st>>>((const V *)in, (V *)out, logLs, ncols, tile, in_es, in_cs,
                                                         in_ts, out_ks, out_cs, out_ts, (const V *)tw, logLtab,
                                                         post_log, (const V *)stw, nullptr);
    CJT_CUDA_TRY(cudaGetLastError());
    return CJT_OK;
}

template <typename R>
int fft_pow2(void *data, void *scratch, int64_t L, int64_t batch, const Twiddles &T, cudaStream_t st) {
    const void *tw = T.tw, *stw = T.stw, *fmat = T.fma;
    const int64_t Ltab = T.Ltab;
    if (L <= 1 || batch <= 0) return CJT_OK;
    const int logL = ilog2(L), logLtab = ilog2(Ltab);
    if ((1LL << logL) != L || L > Ltab) return CJT_EINVAL;
    const int pr = std::is_same<R, float>::value ? 1 : std::is_same<R, dfloat>::value ? 2 : 0;
    const FftCfg &cfg = g_fft_cfg[pr][logL];
    const int ctas = cfg.ctas.load(std::memory_order_relaxed);
    // one pass up to 2^12 points, or 2^13 when so configured and the stage tables (if any)
    // reach that level
    const bool tables13 = (stw == nullptr && fmat == nullptr) || T.lmax >= 13;
    if (logL <= 12 || (logL == 13 && cfg.single.load(std::memory_order_relaxed) >= 13 && tables13)) {
        // direct: each "column" is one whole transform
        return launch_sub<R>(data, data, logL, batch, 1, 1, L, 0, 1, L, 0, tw, logLtab, -1, stw, fmat, st, ctas);
    }
    if (logL > 24 || scratch == nullptr) return CJT_EUNSUPPORTED;
    const int log1 = four_step_log1(logL, cfg.split.load(std::memory_order_relaxed), tables13 ? 13 : 12),
              log2 = logL - log1;
    const int64_t L1 = 1LL << log1, L2 = 1LL << log2;
    // pass A: columns n2 (L2 of them), elements n1 at stride L2
    int rc = launch_sub<R>(data, scratch, log1, L2, batch, L2, 1, L, L2, 1, L, tw, logLtab, logL, stw, fmat, st, ctas);
    if (rc) return rc;
    // pass B: rows k1 (L1 of them), elements n2 contiguous, output X[k1 + L1 k2]
    return launch_sub<R>(scratch, data, log2, L1, batch, 1, L2, L, L1, 1, L, tw, logLtab, -1, stw, fmat, st, ctas);
}

// ---------------------------------------------------------------------------
// Lengths L = q L2, L2 = 2^b, q = 3 or 5: X[k1 + q k2] = sum_{n2} omega_{L2}^{n2 k2}
// (omega_L^{n2 k1} sum_{n1 < q} x[n1 L2 + n2] omega_q^{n1 k1}): one radix-q step with its
// twiddles, then the power-of-two FFTs of the q rows, whose stores put X in natural order.
// ---------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V cconst(double re, double im) { V r; r.x = re; r.y = im; return r; }
template <> __device__ __forceinline__ dfc cconst<dfc>(double re, double im) { return dfc_make(df_from(re), df_from(im)); }

// the q-point DFT of x[0..q-1] (omega_q = exp(-2 pi i / q)) into y[0..q-1]
template <typename V, int Q> struct SmallDft;
template <typename V> struct SmallDft<V, 3> {
    // omega_3 = -1/2 - i sqrt(3)/2
    static __device__ __forceinline__ void run(const V *x, V *y) {
        const V sum = cadd(x[1], x[2]), dif = csub(x[1], x[2]);
        y[0] = cadd(x[0], sum);
        const V mid = csub(x[0], cscale(sum, 0.5));                                      // x0 - (x1 + x2)/2
        const V rot = cmul(dif, cconst<V>(0.0, -0.86602540378443864676372317075294));   // -i sqrt(3)/2 (x1 - x2)
        y[1] = cadd(mid, rot);
        y[2] = csub(mid, rot);
    }
};
// a times a real constant c (any c: the double-float form's cscale takes powers of two only)
template <typename V> __device__ __forceinline__ V cmul_real(V a, double c) { return cscale(a, c); }
template <> __device__ __forceinline__ dfc cmul_real<dfc>(dfc a, double c) { return cmul(a, cconst<dfc>(c, 0.0)); }
template <typename V> struct SmallDft<V, 5> {
    // with s = x1 + x4, t = x2 + x3, d = x1 - x4, e = x2 - x3, c_k = cos(2 pi k/5),
    // s_k = sin(2 pi k/5): X1, X4 = x0 + c1 s + c2 t -+ i (s1 d + s2 e) and
    // X2, X3 = x0 + c2 s + c1 t -+ i (s2 d - s1 e)
    static __device__ __forceinline__ void run(const V *x, V *y) {
        const double c1 = 0.30901699437494742410229341718282, c2 = -0.80901699437494742410229341718282;
        const double s1 = 0.95105651629515357211643933337938, s2 = 0.58778525229247312916870595463907;
        const V sp = cadd(x[1], x[4]), tp = cadd(x[2], x[3]), dm = csub(x[1], x[4]), em = csub(x[2], x[3]);
        y[0] = cadd(x[0], cadd(sp, tp));
        const V a1 = cadd(x[0], cadd(cmul_real(sp, c1), cmul_real(tp, c2)));
        const V a2 = cadd(x[0], cadd(cmul_real(sp, c2), cmul_real(tp, c1)));
        const V b1 = cadd(cmul_real(dm, s1), cmul_real(em, s2));   // X1 = a1 - i b1
        const V b2 = csub(cmul_real(dm, s2), cmul_real(em, s1));   // X2 = a2 - i b2
        const V mib1 = cmul_mi(b1), mib2 = cmul_mi(b2);
        y[1] = cadd(a1, mib1);
        y[4] = csub(a1, mib1);
        y[2] = cadd(a2, mib2);
        y[3] = csub(a2, mib2);
    }
};

// for each sequence and n2 < L2: the q-point DFT of x[n2 + n1 L2], n1 < q, its output k1
// times omega_L^{k1 n2}, stored at n2 + k1 L2 of `out` (which may be `in`: each thread reads
// and writes its own q slots)
template <typename R, int Q>
__global__ void k_fft_rq(const typename cplx<R>::t *__restrict__ in, typename cplx<R>::t *__restrict__ out, int logL2,
                         int64_t total, const typename cplx<R>::t *__restrict__ twq, int64_t tstride) {
    using V = typename cplx<R>::t;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int64_t L2 = 1LL << logL2;
    const int64_t t = i >> logL2, n2 = i & (L2 - 1);
    const int64_t base = t * Q * L2 + n2;
    V x[Q], y[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) x[k] = in[base + k * L2];
    SmallDft<V, Q>::run(x, y);
    out[base] = y[0];
#pragma unroll
    for (int k = 1; k < Q; ++k) out[base + k * L2] = cmul(y[k], twq[k * n2 * tstride]);
}

template <typename R, int Q>
int fft_rq(void *data, void *scratch, int64_t L, int64_t batch, const Twiddles &T, cudaStream_t st) {
    using V = typename cplx<R>::t;
    const int64_t L2 = L / Q;
    const int logL2 = ilog2(L2), logLtab = ilog2(T.Ltab);
    if (!T.twq || T.Ltabq <= 0 || T.Ltabq % L != 0 || L2 > T.Ltab || !scratch) return CJT_EINVAL;
    const int64_t total = batch * L2, ts = T.Ltabq / L;
    const int pr = std::is_same<R, float>::value ? 1 : std::is_same<R, dfloat>::value ? 2 : 0;
    const FftCfg &cfg = g_fft_cfg[pr][logL2];
    const int ctas = cfg.ctas.load(std::memory_order_relaxed);
    const unsigned nb = (unsigned)((total + 255) / 256);
    if (L2 <= 4096) {
        // radix-q step into the scratch buffer, then the rows (q columns of length L2 per
        // sequence) in one pass, stored at X[k1 + q k2]
        k_fft_rq<R, Q><<<nb, 256, 0, st>>>((const V *)data, (V *)scratch, logL2, total, (const V *)T.twq, ts);
        CJT_CUDA_TRY(cudaGetLastError());
        if (L2 == 1) {
            CJT_CUDA_TRY(cudaMemcpyAsync(data, scratch, sizeof(V) * Q * batch, cudaMemcpyDeviceToDevice, st));
            return CJT_OK;
        }
        return launch_sub<R>(scratch, data, logL2, Q, batch, 1, L2, L, Q, 1, L, T.tw, logLtab, -1, T.stw, T.fma, st,
                             ctas);
    }
    // radix-q step in place; the four-step transform of the q batch rows (contiguous, stride
    // L2): pass A over all rows into the scratch buffer, pass B per row k1 into X[k1 + q k]
    k_fft_rq<R, Q><<<nb, 256, 0, st>>>((const V *)data, (V *)data, logL2, total, (const V *)T.twq, ts);
    CJT_CUDA_TRY(cudaGetLastError());
    if (logL2 > 24) return CJT_EUNSUPPORTED;
    const bool tables13 = (T.stw == nullptr && T.fma == nullptr) || T.lmax >= 13;
    const int log1 = four_step_log1(logL2, cfg.split.load(std::memory_order_relaxed), tables13 ? 13 : 12),
              log2 = logL2 - log1;
    const int64_t A1 = 1LL << log1, A2 = 1LL << log2;
    int rc = launch_sub<R>(data, scratch, log1, A2, Q * batch, A2, 1, L2, A2, 1, L2, T.tw, logLtab, logL2, T.stw, T.fma,
                           st, ctas);
    if (rc) return rc;
    for (int k1 = 0; k1 < Q; ++k1) {
        rc = launch_sub<R>((const V *)scratch + k1 * L2, (V *)data + k1, log2, A1, batch, 1, A2, L, Q * A1, Q, L, T.tw,
                           logLtab, -1, T.stw, T.fma, st, ctas);
        if (rc) return rc;
    }
    return CJT_OK;
}

template <typename R>
int fft_any(void *data, void *scratch, int64_t L, int64_t batch, const Twiddles &T, cudaStream_t st) {
    if (L <= 1 || batch <= 0) return CJT_OK;
    if ((L & (L - 1)) == 0) return fft_pow2<R>(data, scratch, L, batch, T, st);
    if (cjt_is_3pow2(L)) return fft_rq<R, 3>(data, scratch, L, batch, T, st);
    if (cjt_is_5pow2(L)) return fft_rq<R, 5>(data, scratch, L, batch, T, st);
    return CJT_EINVAL;
}

// ---------------------------------------------------------------------------
// Bluestein
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_blue_pre(int64_t L, int64_t S, int64_t P, const V *__restrict__ data, const V *__restrict__ chirp,
                           V *__restrict__ work) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (i >= P) return;
    V v = czero<V>();
    if (i < S) v = cmul(data[b * L + i], chirp[i]);
    work[b * P + i] = v;
}

template <typename V>
__global__ void k_blue_mid(int64_t P, const V *__restrict__ bhat, V *__restrict__ work) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (i >= P) return;
    work[b * P + i] = cconj(cmul(work[b * P + i], bhat[i]));
}

template <typename V>
__global__ void k_blue_post(int64_t L, int64_t K, int64_t P, const V *__restrict__ work, const V *__restrict__ chirp,
                            V *__restrict__ data, double invP) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (k >= K) return;
    const V v = cscale(cconj(work[b * P + k]), invP);   // 1/P is a power of two
    data[b * L + k] = cmul(v, chirp[k]);
}

// w_m = exp(-i pi m^2 / L), the square reduced exactly modulo 2L
__global__ void k_blue_chirp(int64_t L, int64_t n, double2 *w64, float2 *w32) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int64_t r = (m * m) % (2 * L);
    double sv, cv;
    sincospi(-(double)r / (double)L, &sv, &cv);
    if (w64) w64[m] = make_double2(cv, sv);
    if (w32) w32[m] = make_float2((float)cv, (float)sv);
}

// cyclic arrangement of conj(w_m) for m in (-(S-1), K-1]
__global__ void k_blue_b(int64_t S, int64_t K, int64_t P, const double2 *__restrict__ w, double2 *__restrict__ b) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= P) return;
    double2 v = make_double2(0.0, 0.0);
    if (j < K) v = make_double2(w[j].x, -w[j].y);
    else if (P - j < S) v = make_double2(w[P - j].x, -w[P - j].y);
    b[j] = v;
}

__global__ void k_to_f32(int64_t n, const double2 *__restrict__ a, float2 *__restrict__ b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void k_to_dfc(int64_t n, const double2 *__restrict__ a, dfc *__restrict__ b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = dfc_make(df_from(a[i].x), df_from(a[i].y));
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R>
int dft_exec(const Dft &d, void *data, void *work, void *scratch, int64_t batch, const Twiddles &tw, cudaStream_t st) {
    using V = typename cplx<R>::t;
    if (batch <= 0 || d.L <= 1) return CJT_OK;
    if (!d.P) return fft_any<R>(data, scratch, d.L, batch, tw, st);
    dim3 g(nblk(d.P, 256), (unsigned)batch);
    k_blue_pre<V><<<g, 256, 0, st>>>(d.L, d.S, d.P, (const V *)data, (const V *)d.chirp, (V *)work);
    CJT_CUDA_TRY(cudaGetLastError());
    int rc = fft_pow2<R>(work, scratch, d.P, batch, tw, st);
    if (rc) return rc;
    k_blue_mid<V><<<g, 256, 0, st>>>(d.P, (const V *)d.bhat, (V *)work);
    CJT_CUDA_TRY(cudaGetLastError());
    rc = fft_pow2<R>(work, scratch, d.P, batch, tw, st);
    if (rc) return rc;
    dim3 g2(nblk(d.K, 256), (unsigned)batch);
    k_blue_post<V><<<g2, 256, 0, st>>>(d.L, d.K, d.P, (const V *)work, (const V *)d.chirp, (V *)data,
                                       1.0 / (double)d.P);
    CJT_CUDA_TRY(cudaGetLastError());
    return CJT_OK;
}

}  // namespace

int64_t cjt_dft_padded(int64_t L, int64_t S, int64_t K) {
    if (L <= 1 || cjt_odd_radix(L) > 0) return 0;
    int64_t P = 1;
    while (P < S + K - 1) P <<= 1;
    return P;
}

int64_t cjt_dft_work_bytes(const Dft &d, int64_t batch) {
    return d.P ? d.P * batch * prec_cbytes(d.prec) : 0;
}

int64_t cjt_dft_scratch_bytes(const Dft &d, int64_t batch) {
    return cjt_fft_scratch_elems(d.fft_len(), batch) * prec_cbytes(d.prec);
}

int cjt_dft_setup(Dft &d, const void *tw64, int64_t Ltab, cudaStream_t st) {
    if (!d.P) return CJT_OK;
    const int64_t nw = std::max(d.S, d.K);
    double2 *w64 = nullptr, *b64 = nullptr, *scr = nullptr;
    CJT_CUDA_TRY(cjt_tmp_alloc((void **)&w64, sizeof(double2) * nw, st));
    CJT_CUDA_TRY(cjt_tmp_alloc((void **)&b64, sizeof(double2) * d.P, st));
    if (d.P > 4096) CJT_CUDA_TRY(cjt_tmp_alloc((void **)&scr, sizeof(double2) * d.P, st));
    k_blue_chirp<<<nblk(nw, 256), 256, 0, st>>>(d.L, nw, w64, nullptr);
    k_blue_b<<<nblk(d.P, 256), 256, 0, st>>>(d.S, d.K, d.P, w64, b64);
    CJT_CUDA_TRY(cudaGetLastError());
    Twiddles t64;
    t64.tw = tw64;
    t64.Ltab = Ltab;
    int rc = fft_pow2<double>(b64, scr, d.P, 1, t64, st);
    if (rc) return rc;
    if (d.prec == PREC_F32) {
        k_to_f32<<<nblk(nw, 256), 256, 0, st>>>(nw, w64, (float2 *)d.chirp);
        k_to_f32<<<nblk(d.P, 256), 256, 0, st>>>(d.P, b64, (float2 *)d.bhat);
    } else if (d.prec == PREC_DF) {
        k_to_dfc<<<nblk(nw, 256), 256, 0, st>>>(nw, w64, (dfc *)d.chirp);
        k_to_dfc<<<nblk(d.P, 256), 256, 0, st>>>(d.P, b64, (dfc *)d.bhat);
    } else {
        CJT_CUDA_TRY(cudaMemcpyAsync(d.chirp, w64, sizeof(double2) * nw, cudaMemcpyDeviceToDevice, st));
        CJT_CUDA_TRY(cudaMemcpyAsync(d.bhat, b64, sizeof(double2) * d.P, cudaMemcpyDeviceToDevice, st));
    }
    CJT_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(w64, st);
    cudaFreeAsync(b64, st);
    if (scr) cudaFreeAsync(scr, st);
    return CJT_OK;
}

int cjt_dft_exec(const Dft &d, void *data, void *work, void *scratch, int64_t batch, const Twiddles &tw,
                 cudaStream_t st) {
    if (d.prec == PREC_F32) return dft_exec<float>(d, data, work, scratch, batch, tw, st);
    if (d.prec == PREC_DF) return dft_exec<dfloat>(d, data, work, scratch, batch, tw, st);
    return dft_exec<double>(d, data, work, scratch, batch, tw, st);
}

int cjt_fft_pow2(void *data, void *scratch, int64_t L, int64_t batch, const Twiddles &tw, int prec, cudaStream_t st) {
    if (prec == PREC_F32) return fft_pow2<float>(data, scratch, L, batch, tw, st);
    if (prec == PREC_DF) return fft_pow2<dfloat>(data, scratch, L, batch, tw, st);
    return fft_pow2<double>(data, scratch, L, batch, tw, st);
}

int64_t cjt_fft_scratch_elems(int64_t L, int64_t batch) {
    return (L > 4096 || cjt_odd_radix(L) > 1) ? L * batch : 0;
}

int cjt_fft_any(void *data, void *scratch, int64_t L, int64_t batch, const Twiddles &tw, int prec, cudaStream_t st) {
    if (prec == PREC_F32) return fft_any<float>(data, scratch, L, batch, tw, st);
    if (prec == PREC_DF) return fft_any<dfloat>(data, scratch, L, batch, tw, st);
    return fft_any<double>(data, scratch, L, batch, tw, st);
}

namespace {
int prec_index(int precision) {
    return precision == CJT_FP64 ? 0 : precision == CJT_MIXED ? 1 : precision == CJT_DFLOAT ? 2 : -1;
}
}  // namespace

extern "C" int cjt_fft_set_config(int precision, int log2L, int ctas_per_sm, int split, int single_max_log2) {
    const int pr = prec_index(precision);
    if (pr < 0 || log2L < 1 || log2L > 24 || ctas_per_sm < 1 || ctas_per_sm > 32 || split < 0 || split > 2 ||
        (single_max_log2 != 12 && single_max_log2 != 13))
        return CJT_EINVAL;
    g_fft_cfg[pr][log2L].ctas.store(ctas_per_sm);
    g_fft_cfg[pr][log2L].split.store(split);
    g_fft_cfg[pr][log2L].single.store(single_max_log2);
    return CJT_OK;
}

extern "C" int cjt_fft_get_config(int precision, int log2L, int *ctas_per_sm, int *split, int *single_max_log2) {
    const int pr = prec_index(precision);
    if (pr < 0 || log2L < 1 || log2L > 24 || !ctas_per_sm || !split || !single_max_log2) return CJT_EINVAL;
    *ctas_per_sm = g_fft_cfg[pr][log2L].ctas.load();
    *split = g_fft_cfg[pr][log2L].split.load();
    *single_max_log2 = g_fft_cfg[pr][log2L].single.load();
    return CJT_OK;
}

// Function attributes, set once per device (they belong to the device's context), so
// that later launches (possibly under stream capture) make no configuration calls.
int cjt_fft_prime() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CJT_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return CJT_OK;
    CJT_CUDA_TRY(cudaFuncSetAttribute(k_fft_sub<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    CJT_CUDA_TRY(cudaFuncSetAttribute(k_fft_sub<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    CJT_CUDA_TRY(cudaFuncSetAttribute(k_fft_sub<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    CJT_CUDA_TRY(cudaFuncSetAttribute(k_fft_sub<dfloat, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    done[dev] = true;
    return CJT_OK;
}
