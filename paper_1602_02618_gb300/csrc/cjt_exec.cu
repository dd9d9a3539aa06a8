// Execution (Sec. 4, steps 2a-2c) of the forward and inverse transforms.
//
// forward (Eq. "CJT"):
//   REC  k_rec_fwd      y_i^REC = sum_{n < J(i)} c_n P_n(x_i): Clenshaw--Smith for
//                       pi/4 < theta_i < 3pi/4, Reinsch-modified (x0 = +-1) otherwise
//                       (Sec. 4.2), one warp per (32 rows x degree segment);
//                       k_rec_fwd_stored(_df): the same sums from the plan's stored values
//   ASY  k_asy_pack_fwd_s / _df   a_{k,m}[n] = C_{n,m} c_n on degrees n >= j_k (pre-scaled
//                       tables), two (k,m) per complex vector
//        FFT            DCT-I and DST-I sums at theta_i (Eq. "PNASY")
//   sum  k_combine_fwd(_df)  y_i = REC partials + sum_m u_m Re F - v_m Im F on the deepest
//                       box of row i
//   DCT  FFT + k_dct_finish   c_cheb = T_N^{-1} y (inverse scaled DCT-I)
// inverse (Eq. "CJTT"):
//   front  FFT of [c_cheb; 0] -> p_N on the 2N grid, g = w o p_N (Clenshaw--Curtis weights)
//   ASY^T  k_asy_pack_inv_s / _df + FFT: Re sum_i (u_m + i v_m) g_i e^{-i n theta_i} per (k,m) box
//   REC^T  k_rec_inv / k_rec_inv_stored(_df): g_i P_n(x_i) summed over each item's rows,
//          then k_inv_reduce over the items of each degree
//   sum    k_combine_inv y_n = REC^T + sum_m C_{n,m} ASY^T, c_jac_n = y_n / A_n
// The double-float form (CJT_DFLOAT) scales its input by an exact power of two first
// (k_absmax_exp, k_to_dfs_scaled) and undoes the scaling in the combines.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "cjt_df.cuh"
#include "cjt_internal.cuh"
#include "cjt_kern.cuh"

namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// single-transform launches of the bodies in cjt_kern.cuh
// ---------------------------------------------------------------------------
using cjt_kern::SW;
constexpr int RED_WARPS = 32;   // one large transform: few blocks carry the heavy segments
using cjt_kern::re_d;
using cjt_kern::im_d;

__global__ void __launch_bounds__(128) k_rec_fwd(const RecItem *__restrict__ items, int64_t nitems, int64_t Ng,
                                                RecTables t, const double *__restrict__ c,
                                                const double *__restrict__ states, double *__restrict__ partials) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= nitems) return;
    const RecItem it = items[w];
    cjt_kern::rec_fwd_warp(it, threadIdx.x & 31, Ng, t, c, states, partials);
}

constexpr int RI_WARPS = 4;
__global__ void __launch_bounds__(32 * RI_WARPS) k_rec_inv(const RecItem *__restrict__ items, int64_t nitems,
                                                          int64_t Ng, RecTables t, const double *__restrict__ g,
                                                          const double *__restrict__ states,
                                                          double *__restrict__ partials) {
    __shared__ double tile[RI_WARPS][32][33];
    const int wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * RI_WARPS + wib;
    if (w >= nitems) return;
    const RecItem it = items[w];
    cjt_kern::rec_inv_warp(it, threadIdx.x & 31, tile[wib], Ng, t, g, states, partials);
}

__global__ void __launch_bounds__(32 * SW) k_rec_fwd_stored(const RecItem *__restrict__ items, int64_t nitems,
                                                            const double *__restrict__ c, const double *__restrict__ E,
                                                            double *__restrict__ partials) {
    if ((int64_t)blockIdx.x >= nitems) return;
    const RecItem it = items[blockIdx.x];
    cjt_kern::rec_fwd_stored_cta(it, c, E, partials);
}

__global__ void __launch_bounds__(32 * SW) k_rec_inv_stored(const RecItem *__restrict__ items, int64_t nitems,
                                                            int64_t Ng, const double *__restrict__ g,
                                                            const double *__restrict__ E, double *__restrict__ partials) {
    if ((int64_t)blockIdx.x >= nitems) return;
    const RecItem it = items[blockIdx.x];
    cjt_kern::rec_inv_stored_cta(it, Ng, g, E, partials);
}

template <typename V, typename R>
__global__ void k_asy_pack_fwd_s(int64_t N, int64_t L, int M, int nq, const int *__restrict__ box3,
                                 const double *__restrict__ Cnm, const double *__restrict__ scale,
                                 const double *__restrict__ c, V *__restrict__ buf) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= L) return;
    const cjt_kern::PairScale ps = cjt_kern::pair_scale(blockIdx.y, M, nq, scale);
    cjt_kern::asy_pack_fwd_elem<V, R>(n, blockIdx.y, ps, N, L, box3, Cnm, c, buf);
}

template <typename V, typename R>
__global__ void k_asy_pack_inv_s(int64_t Ng, int64_t L, int M, int nq, const int *__restrict__ box3,
                                 const double *__restrict__ u, const double *__restrict__ v,
                                 const double *__restrict__ scale, const double *__restrict__ g, V *__restrict__ buf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // row, 0 <= i < Ng = L / 2
    if (i >= Ng) return;
    const cjt_kern::PairScale ps = cjt_kern::pair_scale(blockIdx.y, M, nq, scale);
    cjt_kern::asy_pack_inv_elem<V, R>(i, blockIdx.y, ps, Ng, L, box3, u, v, g, buf);
}

// ---------------------------------------------------------------------------
// CJT_DFLOAT input: x as double-floats scaled by 2^-e, e the binary exponent of max |x|,
// so that any input within the FP64 range keeps the double-float relative precision.
// k_absmax_exp writes one exponent per block (CJT_EXP_BLOCKS blocks); k_to_dfs_scaled
// takes their maximum (order-independent, so deterministic), converts, and leaves e in
// exps[CJT_EXP_BLOCKS] for the kernels that undo the scaling.
// ---------------------------------------------------------------------------
constexpr int EXP_NONE = -100000;   // all-zero input

__global__ void __launch_bounds__(256) k_absmax_exp(int64_t n, const double *__restrict__ x, int *__restrict__ exps) {
    __shared__ double red[8];
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        int e = EXP_NONE;
        if (m > 0.0 && isfinite(m)) frexp(m, &e);
        else if (!isfinite(m)) e = 0;   // inf / nan: no scaling, they propagate
        exps[blockIdx.x] = e;
    }
}

__global__ void k_to_dfs_scaled(int64_t n, const double *__restrict__ x, int *__restrict__ exps,
                                dfs *__restrict__ xdf) {
    __shared__ int se;
    if (threadIdx.x < 32) {
        int e = EXP_NONE;
        for (int j = threadIdx.x; j < CJT_EXP_BLOCKS; j += 32) e = max(e, exps[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (threadIdx.x == 0) se = e == EXP_NONE ? 0 : e;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) exps[CJT_EXP_BLOCKS] = se;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) xdf[i] = df_from(ldexp(x[i], -se));
}

__global__ void k_asy_pack_fwd_df(int64_t N, int64_t L, int nq, const dfs *__restrict__ Cs,
                                  const dfs *__restrict__ cdf, dfc *__restrict__ buf) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (n >= L) return;
    dfs re = df_make(0.f, 0.f), im = df_make(0.f, 0.f);
    if (n <= N) {
        const dfs cn = cdf[n];
        const int q = 2 * p;
        re = df_mul(Cs[(int64_t)q * (N + 1) + n], cn);
        if (q + 1 < nq) im = df_mul(Cs[(int64_t)(q + 1) * (N + 1) + n], cn);
    }
    buf[(int64_t)p * L + n] = dfc_make(re, im);
}

__global__ void k_asy_pack_inv_df(int64_t Ng, int64_t L, int nq, const dfs *__restrict__ Us,
                                  const dfs *__restrict__ Vs, const dfs *__restrict__ gdf, dfc *__restrict__ buf) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (idx >= L) return;
    // H(idx) = (z(idx) + conj z(L - idx)) / 2: the box rows lie in [1, Ng - 1]
    const bool lo = idx <= Ng;
    const int64_t i = lo ? idx : L - idx;
    const dfs gi = gdf[i];
    const int q = 2 * p;
    const dfs h0r = df_mul(Us[(int64_t)q * (Ng + 1) + i], gi);
    dfs h0i = df_mul(Vs[(int64_t)q * (Ng + 1) + i], gi);
    dfs h1r = df_make(0.f, 0.f), h1i = df_make(0.f, 0.f);
    if (q + 1 < nq) {
        h1r = df_mul(Us[(int64_t)(q + 1) * (Ng + 1) + i], gi);
        h1i = df_mul(Vs[(int64_t)(q + 1) * (Ng + 1) + i], gi);
    }
    if (!lo) {
        h0i = df_neg(h0i);
        h1i = df_neg(h1i);
    }
    buf[(int64_t)p * L + idx] = dfc_make(df_sub(h0r, h1i), df_add(h0i, h1r));
}

// REC with stored double-float values: one double-float multiply-add per entry,
// renormalised at every step (an unnormalised low part would let its own rounding
// errors grow with the segment length)
// as k_rec_fwd_stored, in double-float arithmetic
__global__ void __launch_bounds__(32 * SW) k_rec_fwd_stored_df(const RecItem *__restrict__ items, int64_t nitems,
                                                               const dfs *__restrict__ cdf, const dfs *__restrict__ E,
                                                               double *__restrict__ partials) {
    __shared__ dfs red_e[SW][32], red_o[SW][32];
    if ((int64_t)blockIdx.x >= nitems) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RecItem it = items[blockIdx.x];
    const int len = it.b - it.a;
    const int per = ((len + SW - 1) / SW + 7) & ~7;
    const int k0 = min(len, w * per), k1 = min(len, k0 + per);
    const float2 *e = reinterpret_cast<const float2 *>(E + it.eoff) + lane;
    const dfs *cc = cdf + it.a;
    // eight streaming loads per lane, the next eight issued before the current ones are
    // used (software pipelining: the arithmetic is long enough to hide a load otherwise),
    // four independent accumulators
    dfs acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = df_make(0.f, 0.f);
    int k = k0;
    if (k + 8 <= k1) {
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldcs(e + (int64_t)(k + j) * 32);
        for (; k + 8 <= k1; k += 8) {
            float2 vn[8];
            const bool more = k + 16 <= k1;
#pragma unroll
            for (int j = 0; j < 8; ++j) vn[j] = more ? __ldcs(e + (int64_t)(k + 8 + j) * 32) : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j & 3] = df_mac(acc[j & 3], df_make(v[j].x, v[j].y), cc[k + j]);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = vn[j];
        }
    }
    for (; k < k1; ++k) {
        const float2 v = __ldcs(e + (int64_t)k * 32);
        acc[k & 1] = df_mac(acc[k & 1], df_make(v.x, v.y), cc[k]);
    }
    // accumulators 0, 2 hold the even degrees, 1, 3 the odd ones (as in k_rec_fwd_stored)
    red_e[w][lane] = df_add(acc[0], acc[2]);
    red_o[w][lane] = df_add(acc[1], acc[3]);
    __syncthreads();
    if (w == 0) {
        const dfs Se = df_add(df_add(red_e[0][lane], red_e[1][lane]), df_add(red_e[2][lane], red_e[3][lane]));
        const dfs So = df_add(df_add(red_o[0][lane], red_o[1][lane]), df_add(red_o[2][lane], red_o[3][lane]));
        const bool act = lane < it.nrows;
        reinterpret_cast<dfs *>(partials)[it.out + lane] = act ? df_add(Se, So) : df_make(0.f, 0.f);
        if (it.mirror) reinterpret_cast<dfs *>(partials)[it.out2 + lane] = act ? df_sub(Se, So) : df_make(0.f, 0.f);
    }
}

// as k_rec_inv_stored, in double-float arithmetic (rows in groups of eight loads in flight,
// four independent accumulators per column)
__global__ void __launch_bounds__(32 * SW) k_rec_inv_stored_df(const RecItem *__restrict__ items, int64_t nitems,
                                                               int64_t Ng, const dfs *__restrict__ gdf,
                                                               const dfs *__restrict__ E,
                                                               double *__restrict__ partials) {
    __shared__ dfs gsb[2][32];   // parity fold as in k_rec_inv_stored: [0] even, [1] odd degrees
    if ((int64_t)blockIdx.x >= nitems) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RecItem it = items[blockIdx.x];
    if (w == 0) {
        const bool act = lane < it.nrows;
        const dfs gr = act ? gdf[it.row0 + lane] : df_make(0.f, 0.f);
        const dfs gm = act && it.mirror ? gdf[Ng - it.row0 - lane] : df_make(0.f, 0.f);
        gsb[0][lane] = it.mirror ? df_add(gr, gm) : gr;
        gsb[1][lane] = it.mirror ? df_sub(gr, gm) : gr;
    }
    __syncthreads();
    const dfs *gs = gsb[lane & 1];
    const int len = it.b - it.a, nr = it.nrows;
    const float2 *e = reinterpret_cast<const float2 *>(E + it.eoff);
    double *out = partials + it.out;
    for (int k0 = w * 32; k0 < len; k0 += 32 * SW) {
        const int k = k0 + lane;
        if (k < len) {
            dfs acc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = df_make(0.f, 0.f);
            int r = 0;
            if (r + 8 <= nr) {   // as in the forward kernel: the next eight rows load during this eight's arithmetic
                float2 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = __ldcs(e + (int64_t)(r + j) * len + k);
                for (; r + 8 <= nr; r += 8) {
                    float2 vn[8];
                    const bool more = r + 16 <= nr;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        vn[j] = more ? __ldcs(e + (int64_t)(r + 8 + j) * len + k) : make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[j & 3] = df_mac(acc[j & 3], gs[r + j], df_make(v[j].x, v[j].y));
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = vn[j];
                }
            }
            for (; r < nr; ++r) {
                const float2 v = __ldcs(e + (int64_t)r * len + k);
                acc[0] = df_mac(acc[0], gs[r], df_make(v.x, v.y));
            }
            out[k] = df_to(df_add(df_add(acc[0], acc[1]), df_add(acc[2], acc[3])));
        }
    }
}

// ---------------------------------------------------------------------------
// combine, forward, CJT_DFLOAT: the same sums in double-float arithmetic on the scaled
// input (partials P: double-floats from the stored recurrence, or doubles from the
// recurrence at execution, which ran on the unscaled input); one conversion to double
// and the exact unscaling 2^e at the end
// ---------------------------------------------------------------------------
__device__ __forceinline__ dfs scaled_partial(dfs v, int) { return v; }
__device__ __forceinline__ dfs scaled_partial(double v, int e) { return df_from(ldexp(v, -e)); }

template <typename P>
__global__ void k_combine_fwd_df(int64_t N, int64_t L, int M, const int *__restrict__ rowk,
                                 const double *__restrict__ scale, const dfs *__restrict__ u,
                                 const dfs *__restrict__ v, const dfc *__restrict__ buf,
                                 const int64_t *__restrict__ row_base, const int *__restrict__ row_nseg,
                                 const P *__restrict__ partials, const int *__restrict__ exps,
                                 double2 *__restrict__ ext) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > N) return;
    const int e = exps[CJT_EXP_BLOCKS];
    const int nseg = row_nseg[i];
    const int64_t base = row_base[i];
    // rows near x = +-1 have up to N / seg_len segments: eight loads in flight, four sums
    dfs ya[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) ya[j] = df_make(0.f, 0.f);
    int s = 0;
    for (; s + 8 <= nseg; s += 8) {
        P pv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) pv[j] = partials[base + (int64_t)(s + j) * 32];
#pragma unroll
        for (int j = 0; j < 8; ++j) ya[j & 3] = df_add(ya[j & 3], scaled_partial(pv[j], e));
    }
    for (; s < nseg; ++s) ya[0] = df_add(ya[0], scaled_partial(partials[base + (int64_t)s * 32], e));
    dfs y = df_add(df_add(ya[0], ya[1]), df_add(ya[2], ya[3]));
    const int k = rowk[i];
    if (k >= 0) {
        const int64_t im = i == 0 ? 0 : L - i;
        for (int m = 0; m < M; ++m) {
            const int q = k * M + m, p = q >> 1;
            const dfc Z = buf[(int64_t)p * L + i], W = buf[(int64_t)p * L + im];
            dfs re, imv;
            if ((q & 1) == 0) {
                re = df_add(dfc_re(Z), dfc_re(W));
                imv = df_sub(dfc_im(Z), dfc_im(W));
            } else {
                re = df_add(dfc_im(Z), dfc_im(W));
                imv = df_sub(dfc_re(W), dfc_re(Z));
            }
            // u, v carry 1/2 and the item's unscaling (plan time)
            y = df_add(y, df_mms(u[m * (N + 1) + i], re, v[m * (N + 1) + i], imv));
        }
    }
    // the even extension for the FP64 DCT-I (its errors would reach the inverse of a round
    // trip through 1/A_n), unscaled
    const double yv = ldexp(df_to(y), e);
    ext[i] = make_double2(yv, 0.0);
    if (i >= 1 && i < N) ext[2 * N - i] = make_double2(yv, 0.0);
}


template <typename V>
__global__ void k_combine_fwd(int64_t N, int64_t L, int M, const int *__restrict__ rowk,
                              const double *__restrict__ scale, const double *__restrict__ u,
                              const double *__restrict__ v, const V *__restrict__ buf,
                              const int64_t *__restrict__ row_base, const int *__restrict__ row_nseg,
                              const double *__restrict__ partials, double2 *__restrict__ ext) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > N) return;
    cjt_kern::combine_fwd_elem<V>(i, N, L, M, rowk, scale, u, v, buf, row_base, row_nseg, partials, ext);
}

// c_k for k <= N from the transform of the grid G >= N
__global__ void k_dct_finish(int64_t N, int64_t G, const double2 *__restrict__ Z, double *__restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k > N) return;
    cjt_kern::dct_finish_elem(k, G, Z, out);
}

__global__ void k_inv_front_pack(int64_t N, int64_t L, const double *__restrict__ c, double2 *__restrict__ buf) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= L) return;
    cjt_kern::inv_front_pack_elem(k, N, c, buf);
}

__global__ void k_inv_g(int64_t Ng, const double2 *__restrict__ F, const double *__restrict__ w, double *__restrict__ g) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > Ng) return;
    cjt_kern::inv_g_elem(i, F, w, g);
}

// one block per 32 consecutive degrees
__global__ void __launch_bounds__(32 * RED_WARPS) k_inv_reduce(int64_t N, int seg_len,
                                                               const int64_t *__restrict__ seg_ptr,
                                                               const int64_t *__restrict__ seg_out,
                                                               const int *__restrict__ seg_b,
                                                               const double *__restrict__ partials,
                                                               double *__restrict__ y) {
    cjt_kern::inv_reduce_block<RED_WARPS>(blockIdx.x, N, seg_len, seg_ptr, seg_out, seg_b, partials, y);
}

template <typename V>
__global__ void k_combine_inv(int64_t N, int64_t L, int M, int nblk, const int *__restrict__ box3,
                              const double *__restrict__ scale, const double *__restrict__ Cnm,
                              const V *__restrict__ buf, const double *__restrict__ yrec,
                              const double *__restrict__ s_n, const int *__restrict__ exps, int rec_scaled,
                              double *__restrict__ out) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n > N) return;
    cjt_kern::combine_inv_elem<V>(n, N, L, M, nblk, box3, scale, Cnm, buf, yrec, s_n, exps, rec_scaled, out);
}

__global__ void k_copy(int64_t n, const double *__restrict__ in, double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

// gives an execution's overlap context back to the pool on every return path
struct OvGuard {
    OvCtx *c;
    ~OvGuard() { cjt_internal_ovctx_release(c); }
};

}  // namespace

// ---------------------------------------------------------------------------
// forward / inverse drivers
// ---------------------------------------------------------------------------
int cjt_exec_forward(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st) {
    const int64_t N = p->N;
    if (N == 0) {
        k_copy<<<1, 32, 0, st>>>(1, in, out);
        CJT_CUDA_TRY(cudaGetLastError());
        return CJT_OK;
    }
    GridWork &gw = p->fw;
    const bool fp32 = p->prec_asy == PREC_F32, dfm = p->prec_asy == PREC_DF;
    const int M = p->M;
    int rc;
    const int nq = gw.nblk * M;
    const int64_t L = p->Lf;
    // double-float execution: the input scaled to max |c| < 1 and converted once
    const bool dfx = dfm;
    dfs *cdf = (dfs *)ws.xdf;
    if (dfx) {
        k_absmax_exp<<<CJT_EXP_BLOCKS, 256, 0, st>>>(N + 1, in, ws.exps);
        k_to_dfs_scaled<<<blocks_for(N + 1, 256), 256, 0, st>>>(N + 1, in, ws.exps, cdf);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    // the asymptotic transforms run on a side stream, concurrently with the recurrence
    // (on the caller's stream, or on a second side stream with CJT_OVERLAP_REC_FIRST)
    const bool ovl = nq > 0 && !p->prof;   // profiled: the two chains one after the other
    OvCtx *oc = nullptr;
    if (ovl) {
        rc = cjt_internal_ovctx_acquire(p->opts.overlap, st, &oc);
        if (rc) return rc;
    }
    OvGuard og{oc};
    cudaStream_t sa = ovl ? oc->side : st;
    cudaStream_t sr = (ovl && oc->side_rec) ? oc->side_rec : st;
    if (ovl) {
        CJT_CUDA_TRY(cudaEventRecord(oc->fork, st));
        CJT_CUDA_TRY(cudaStreamWaitEvent(sa, oc->fork, 0));
        if (sr != st) CJT_CUDA_TRY(cudaStreamWaitEvent(sr, oc->fork, 0));
    }
    if (nq > 0) {
        dim3 gp(blocks_for(L, 256), p->npair_f);
        StageTimer tm(p, sa, CJT_STAGE_FWD_PACK);
        if (dfm)
            k_asy_pack_fwd_df<<<gp, 256, 0, sa>>>(N, L, nq, (const dfs *)gw.d_Cs, cdf, (dfc *)ws.fft_f);
        else if (fp32)
            k_asy_pack_fwd_s<float2, float><<<gp, 256, 0, sa>>>(N, L, M, nq, gw.d_box, p->d_Cnm, gw.d_scale, in,
                                                               (float2 *)ws.fft_f);
        else
            k_asy_pack_fwd_s<double2, double><<<gp, 256, 0, sa>>>(N, L, M, nq, gw.d_box, p->d_Cnm, gw.d_scale, in,
                                                                 (double2 *)ws.fft_f);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    if (nq > 0) {
        StageTimer tm(p, sa, CJT_STAGE_FWD_FFT);
        rc = cjt_dft_exec(p->dft_f, ws.fft_f, ws.work, ws.scratch, p->npair_f, p->twiddles(p->prec_asy), sa);
        if (rc) return rc;
    }
    // REC
    if (gw.nitems > 0) {
        StageTimer tm(p, sr, CJT_STAGE_FWD_REC);
        if (gw.d_E && gw.E_df)
            k_rec_fwd_stored_df<<<(unsigned)gw.nitems, 32 * SW, 0, sr>>>(gw.d_items, gw.nitems, cdf,
                                                                                (const dfs *)gw.d_E, ws.part_f);
        else if (gw.d_E)
            k_rec_fwd_stored<<<(unsigned)gw.nitems, 32 * SW, 0, sr>>>(gw.d_items, gw.nitems, in, gw.d_E,
                                                                             ws.part_f);
        else
            k_rec_fwd<<<blocks_for(gw.nitems * 32, 128), 128, 0, sr>>>(gw.d_items, gw.nitems, gw.Ng, p->rt, in,
                                                                      gw.d_states, ws.part_f);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    if (ovl) {
        CJT_CUDA_TRY(cudaEventRecord(oc->join, sa));
        CJT_CUDA_TRY(cudaStreamWaitEvent(st, oc->join, 0));
        if (sr != st) {
            CJT_CUDA_TRY(cudaEventRecord(oc->join_rec, sr));
            CJT_CUDA_TRY(cudaStreamWaitEvent(st, oc->join_rec, 0));
        }
    }
    double2 *ext = (double2 *)ws.dct;
    const int64_t G = p->Gf;   // grid rows 0..G (the combines' "N" is the grid)
    {
    StageTimer tm(p, st, CJT_STAGE_FWD_COMBINE);
    if (dfx && gw.E_df)
        k_combine_fwd_df<dfs><<<blocks_for(G + 1, 256), 256, 0, st>>>(
            G, L, M, gw.d_rowk, gw.d_scale, (const dfs *)gw.d_u, (const dfs *)gw.d_v, (const dfc *)ws.fft_f,
            gw.d_row_base, gw.d_row_nseg, (const dfs *)ws.part_f, ws.exps, ext);
    else if (dfx)
        k_combine_fwd_df<double><<<blocks_for(G + 1, 256), 256, 0, st>>>(
            G, L, M, gw.d_rowk, gw.d_scale, (const dfs *)gw.d_u, (const dfs *)gw.d_v, (const dfc *)ws.fft_f,
            gw.d_row_base, gw.d_row_nseg, ws.part_f, ws.exps, ext);
    else if (fp32)
        k_combine_fwd<float2><<<blocks_for(G + 1, 256), 256, 0, st>>>(
            G, L, M, gw.d_rowk, gw.d_scale, gw.d_u, gw.d_v, (const float2 *)ws.fft_f, gw.d_row_base, gw.d_row_nseg,
            ws.part_f, ext);
    else
        k_combine_fwd<double2><<<blocks_for(G + 1, 256), 256, 0, st>>>(
            G, L, M, gw.d_rowk, gw.d_scale, gw.d_u, gw.d_v, (const double2 *)ws.fft_f, gw.d_row_base, gw.d_row_nseg,
            ws.part_f, ext);
    CJT_CUDA_TRY(cudaGetLastError());
    }
    StageTimer tm(p, st, CJT_STAGE_FWD_DCT);
    rc = cjt_dft_exec(p->dft_dct, ws.dct, ws.work, ws.scratch, 1, p->twiddles(PREC_F64), st);
    if (rc) return rc;
    k_dct_finish<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, G, (const double2 *)ws.dct, out);
    CJT_CUDA_TRY(cudaGetLastError());
    return CJT_OK;
}

int cjt_exec_inverse(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st) {
    const int64_t N = p->N;
    if (N == 0) {
        k_copy<<<1, 32, 0, st>>>(1, in, out);
        CJT_CUDA_TRY(cudaGetLastError());
        return CJT_OK;
    }
    GridWork &gw = p->iv;
    const bool fp32 = p->prec_asy == PREC_F32, dfm = p->prec_asy == PREC_DF;
    dfs *gdf = (dfs *)ws.xdf;
    const int M = p->M;
    const int64_t Ng = 2 * p->Gi, L = p->Li;
    // front end: p_N on the 2N grid, times the Clenshaw--Curtis weights
    int rc;
    {
    StageTimer tm(p, st, CJT_STAGE_INV_FRONT);
    k_inv_front_pack<<<blocks_for(L, 256), 256, 0, st>>>(N, L, in, (double2 *)ws.dct);
    CJT_CUDA_TRY(cudaGetLastError());
    rc = cjt_dft_exec(p->dft_front, ws.dct, ws.work, ws.scratch, 1, p->twiddles(PREC_F64), st);
    if (rc) return rc;
    k_inv_g<<<blocks_for(Ng + 1, 256), 256, 0, st>>>(Ng, (const double2 *)ws.dct, p->d_w, ws.g);
    CJT_CUDA_TRY(cudaGetLastError());
    }
    const int nq = gw.nblk * M;
    // double-float execution: g scaled to max |g| < 1 and converted once.  The front end
    // stays in FP64: its errors reach c_jac_n through 1/A_n, which grows with n.
    const bool dfx = dfm;
    if (dfx) {
        k_absmax_exp<<<CJT_EXP_BLOCKS, 256, 0, st>>>(Ng + 1, ws.g, ws.exps);
        k_to_dfs_scaled<<<blocks_for(Ng + 1, 256), 256, 0, st>>>(Ng + 1, ws.g, ws.exps, gdf);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    // transposed asymptotic blocks, on a side stream concurrently with the recurrence
    // (on the caller's stream, or on a second side stream with CJT_OVERLAP_REC_FIRST)
    const bool ovl = nq > 0 && !p->prof;   // profiled: the two chains one after the other
    OvCtx *oc = nullptr;
    if (ovl) {
        rc = cjt_internal_ovctx_acquire(p->opts.overlap, st, &oc);
        if (rc) return rc;
    }
    OvGuard og{oc};
    cudaStream_t sa = ovl ? oc->side : st;
    cudaStream_t sr = (ovl && oc->side_rec) ? oc->side_rec : st;
    if (ovl) {
        CJT_CUDA_TRY(cudaEventRecord(oc->fork, st));
        CJT_CUDA_TRY(cudaStreamWaitEvent(sa, oc->fork, 0));
        if (sr != st) CJT_CUDA_TRY(cudaStreamWaitEvent(sr, oc->fork, 0));
    }
    if (nq > 0) {
        // the double-float pack takes one element per thread, the others one row (two elements)
        dim3 gp(blocks_for(dfm ? L : Ng, 256), p->npair_i);
        StageTimer tm(p, sa, CJT_STAGE_INV_PACK);
        if (dfm)
            k_asy_pack_inv_df<<<gp, 256, 0, sa>>>(Ng, L, nq, (const dfs *)gw.d_Us, (const dfs *)gw.d_Vs, gdf,
                                                  (dfc *)ws.fft_i);
        else if (fp32)
            k_asy_pack_inv_s<float2, float><<<gp, 256, 0, sa>>>(Ng, L, M, nq, gw.d_box, gw.d_u, gw.d_v, gw.d_scale,
                                                                ws.g, (float2 *)ws.fft_i);
        else
            k_asy_pack_inv_s<double2, double><<<gp, 256, 0, sa>>>(Ng, L, M, nq, gw.d_box, gw.d_u, gw.d_v,
                                                                  gw.d_scale, ws.g, (double2 *)ws.fft_i);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    if (nq > 0) {
        StageTimer tm(p, sa, CJT_STAGE_INV_FFT);
        rc = cjt_dft_exec(p->dft_i, ws.fft_i, ws.work, ws.scratch, p->npair_i, p->twiddles(p->prec_asy), sa);
        if (rc) return rc;
    }
    // transposed recurrence and the fixed-order sums over the items of each degree
    {
        StageTimer tm(p, sr, CJT_STAGE_INV_REC);
        if (gw.nitems > 0) {
            if (gw.d_E && gw.E_df)
                k_rec_inv_stored_df<<<(unsigned)gw.nitems, 32 * SW, 0, sr>>>(gw.d_items, gw.nitems, Ng, gdf,
                                                                               (const dfs *)gw.d_E, ws.part_i);
            else if (gw.d_E)
                k_rec_inv_stored<<<(unsigned)gw.nitems, 32 * SW, 0, sr>>>(gw.d_items, gw.nitems, Ng, ws.g, gw.d_E,
                                                                            ws.part_i);
            else
                k_rec_inv<<<blocks_for(gw.nitems, RI_WARPS), 32 * RI_WARPS, 0, sr>>>(gw.d_items, gw.nitems, Ng, p->rt,
                                                                                     ws.g, gw.d_states, ws.part_i);
            CJT_CUDA_TRY(cudaGetLastError());
        }
        k_inv_reduce<<<blocks_for(N + 1, 32), 32 * RED_WARPS, 0, sr>>>(N, p->seg_len, gw.d_seg_ptr, gw.d_seg_out,
                                                                         gw.d_seg_b, ws.part_i, ws.y);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    if (ovl) {
        CJT_CUDA_TRY(cudaEventRecord(oc->join, sa));
        CJT_CUDA_TRY(cudaStreamWaitEvent(st, oc->join, 0));
        if (sr != st) {
            CJT_CUDA_TRY(cudaEventRecord(oc->join_rec, sr));
            CJT_CUDA_TRY(cudaStreamWaitEvent(st, oc->join_rec, 0));
        }
    }
    StageTimer tm(p, st, CJT_STAGE_INV_COMBINE);
    if (dfx)
        k_combine_inv<dfc><<<blocks_for(N + 1, 256), 256, 0, st>>>(N, L, M, gw.nblk, gw.d_box, gw.d_scale, p->d_Cnm,
                                                                  (const dfc *)ws.fft_i, ws.y, p->d_s, ws.exps,
                                                                  gw.E_df ? 1 : 0, out);
    else if (fp32)
        k_combine_inv<float2><<<blocks_for(N + 1, 256), 256, 0, st>>>(N, L, M, gw.nblk, gw.d_box, gw.d_scale,
                                                                     p->d_Cnm, (const float2 *)ws.fft_i, ws.y, p->d_s,
                                                                     nullptr, 0, out);
    else
        k_combine_inv<double2><<<blocks_for(N + 1, 256), 256, 0, st>>>(N, L, M, gw.nblk, gw.d_box, gw.d_scale,
                                                                      p->d_Cnm, (const double2 *)ws.fft_i, ws.y,
                                                                      p->d_s, nullptr, 0, out);
    CJT_CUDA_TRY(cudaGetLastError());
    return CJT_OK;
}
