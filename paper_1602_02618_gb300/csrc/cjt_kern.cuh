// Per-element, per-warp and per-CTA bodies of the execution kernels (Sec. 4, steps 2a-2c).
//
// Each body computes the work of one element, warp or CTA of ONE transform from that
// transform's tables and buffers.  Two kinds of kernels call them:
//   * cjt_exec.cu: one launch per stage of one transform (the single-transform path);
//   * cjt_group.cu: one launch per stage over many transforms of a batch, each CTA (or
//     warp) finding its transform and its position in it from a table built with the batch.
// Both run the same arithmetic in the same order, so a transform's result does not depend
// on which kind of launch computed it (bit for bit).
#pragma once

#include <type_traits>

#include "cjt_df.cuh"
#include "cjt_internal.cuh"

namespace cjt_kern {

// ---------------------------------------------------------------------------
// REC, forward (Sec. 4.2): one warp per item, lane = row.  Clenshaw--Smith for
// pi/4 < theta < 3pi/4; Reinsch-modified with x0 = +1 or -1 near the ends, in the
// e_n = d_n / r^b_n form (3 DFMA + 1 DMUL per step).  Writes the segment sum of each
// lane's row to partials[it.out + lane].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rec_fwd_warp(const RecItem &it, int lane, int64_t Ng, const RecTables &t,
                                             const double *__restrict__ c, const double *__restrict__ states,
                                             double *__restrict__ partials) {
    const int row = it.row0 + min(lane, it.nrows - 1);
    double P1 = 1.0, P2 = 0.0;
    if (it.state >= 0) {
        const double2 sv = reinterpret_cast<const double2 *>(states)[(int64_t)it.state * 32 + lane];
        P1 = sv.x;
        P2 = sv.y;
    }
    double S;
    if (it.mode == REC_PLAIN) {
        const double x = cospi((double)row / (double)Ng);
        double u1 = 0.0, u2 = 0.0;
        for (int n = it.b - 1; n >= it.a; --n) {
            const double w0 = fma(-__ldg(t.C + n + 1), u2, __ldg(c + n));
            const double u0 = fma(fma(__ldg(t.A + n), x, __ldg(t.B + n)), u1, w0);
            u2 = u1;
            u1 = u0;
        }
        // segment sum = pi_a u_a - C_a pi_{a-1} u_{a+1}
        S = fma(P1, u1, -__ldg(t.C + it.a) * P2 * u2);
    } else {
        const bool plus = it.mode == REC_REINSCH_P1;
        double delta;
        if (plus) {
            const double s = sinpi((double)row / (2.0 * (double)Ng));
            delta = -2.0 * s * s;
        } else {
            const double s = sinpi((double)(Ng - row) / (2.0 * (double)Ng));
            delta = 2.0 * s * s;
        }
        const double *Cr = plus ? t.Cr_p : t.Cr_m;
        const double *rbinv = plus ? t.rbinv_p : t.rbinv_m;
        const double *Ce = plus ? t.Ce_p : t.Ce_m;
        double u = 0.0, e = 0.0, uprev = 0.0;
        for (int n = it.b - 1; n >= it.a; --n) {
            const double wn = fma(__ldg(Cr + n + 1), e, __ldg(c + n));
            const double en = fma(__ldg(t.A + n) * delta, u, wn);
            const double un = fma(u, __ldg(rbinv + n), en);
            uprev = u;
            u = un;
            e = en;
        }
        // segment sum = pi_a e_a + C_a/r^f_{a-1} u_{a+1} e^f_a
        S = fma(P1, e, __ldg(Ce + it.a) * uprev * P2);
    }
    partials[it.out + lane] = lane < it.nrows ? S : 0.0;
}

// ---------------------------------------------------------------------------
// REC, inverse (transposed): one warp per item; lane = row; the degree sums over the
// warp's rows go through a padded 32 x 33 shared-memory tile `tl` owned by the warp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rec_inv_warp(const RecItem &it, int lane, double (*tl)[33], int64_t Ng,
                                             const RecTables &t, const double *__restrict__ g,
                                             const double *__restrict__ states, double *__restrict__ partials) {
    const bool active = lane < it.nrows;
    const int row = it.row0 + min(lane, it.nrows - 1);
    const double gi = active ? g[row] : 0.0;
    double P1 = gi, P2 = 0.0;
    if (active && it.state >= 0) {
        const double2 sv = reinterpret_cast<const double2 *>(states)[(int64_t)it.state * 32 + lane];
        P1 = sv.x * gi;
        P2 = sv.y * gi;
    }
    double *out = partials + it.out - it.a;
    if (it.mode == REC_PLAIN) {
        const double x = cospi((double)row / (double)Ng);
        double p = P1, pm = P2;
        for (int n0 = it.a; n0 < it.b; n0 += 32) {
            const int cnt = min(32, it.b - n0);
            for (int r = 0; r < cnt; ++r) {
                const int n = n0 + r;
                tl[r][lane] = p;
                const double pn = fma(fma(__ldg(t.A + n), x, __ldg(t.B + n)), p, -__ldg(t.C + n) * pm);
                pm = p;
                p = pn;
            }
            __syncwarp();
            if (lane < cnt) {
                double s = 0.0;
#pragma unroll 8
                for (int r = 0; r < 32; ++r) s += tl[lane][r];
                out[n0 + lane] = s;
            }
            __syncwarp();
        }
    } else {
        const bool plus = it.mode == REC_REINSCH_P1;
        double delta;
        if (plus) {
            const double s = sinpi((double)row / (2.0 * (double)Ng));
            delta = -2.0 * s * s;
        } else {
            const double s = sinpi((double)(Ng - row) / (2.0 * (double)Ng));
            delta = 2.0 * s * s;
        }
        const double *Ce = plus ? t.Ce_p : t.Ce_m;
        const double *rf = plus ? t.rf_p : t.rf_m;
        double p = P1, e = P2;
        for (int n0 = it.a; n0 < it.b; n0 += 32) {
            const int cnt = min(32, it.b - n0);
            for (int r = 0; r < cnt; ++r) {
                const int n = n0 + r;
                tl[r][lane] = p;
                const double en = fma(__ldg(t.A + n) * delta, p, __ldg(Ce + n) * e);
                p = fma(p, __ldg(rf + n), en);
                e = en;
            }
            __syncwarp();
            if (lane < cnt) {
                double s = 0.0;
#pragma unroll 8
                for (int r = 0; r < 32; ++r) s += tl[lane][r];
                out[n0 + lane] = s;
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// REC with stored values (rec_store): one fused multiply-add per entry.
// One CTA of SW warps per item: warp w takes a quarter of the item's degrees (eight
// streaming loads in flight per lane), and the four partial sums are added in warp order.
// Splitting the long items (rows near x = +-1) over four warps keeps the SMs busy to the
// end of the launch.  The sums over even and odd degrees are kept apart (accumulator j
// takes the degrees a + k + j, a and k even, so its parity is that of j): their sum is the
// row's partial, and under the parity fold their difference is the mirrored row's, since
// P_n(-x) = (-1)^n P_n(x) when alpha = beta.
// ---------------------------------------------------------------------------
constexpr int SW = 4;
__device__ __forceinline__ void rec_fwd_stored_cta(const RecItem &it, const double *__restrict__ c,
                                                   const double *__restrict__ E, double *__restrict__ partials) {
    __shared__ double red_e[SW][32], red_o[SW][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int len = it.b - it.a;
    const int per = ((len + SW - 1) / SW + 7) & ~7;
    const int k0 = min(len, w * per), k1 = min(len, k0 + per);
    const double *e = E + it.eoff + lane;
    const double *cc = c + it.a;
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int k = k0;
    for (; k + 8 <= k1; k += 8) {
        double v[8], cv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] = __ldcs(e + (int64_t)(k + j) * 32);
            cv[j] = __ldg(cc + k + j);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = fma(v[j], cv[j], acc[j]);
    }
    for (; k < k1; ++k) acc[k & 1] = fma(__ldcs(e + (int64_t)k * 32), __ldg(cc + k), acc[k & 1]);
    red_e[w][lane] = (acc[0] + acc[2]) + (acc[4] + acc[6]);
    red_o[w][lane] = (acc[1] + acc[3]) + (acc[5] + acc[7]);
    __syncthreads();
    if (w == 0) {
        const double Se = (red_e[0][lane] + red_e[1][lane]) + (red_e[2][lane] + red_e[3][lane]);
        const double So = (red_o[0][lane] + red_o[1][lane]) + (red_o[2][lane] + red_o[3][lane]);
        const bool act = lane < it.nrows;
        partials[it.out + lane] = act ? Se + So : 0.0;
        if (it.mirror) partials[it.out2 + lane] = act ? Se - So : 0.0;
    }
}

// One CTA of SW warps per item: warp w takes the item's degree columns w*32 + lane,
// (w + SW)*32 + lane, ...; each column sums its 32 rows in order.  Under the parity fold
// row r also stands for row Ng - row0 - r: degree n gets P_n(x_r) (g_r + (-1)^n g_mirror),
// and column k = k0 + lane (k0 and a multiples of 32) has the parity of its lane.
__device__ __forceinline__ void rec_inv_stored_cta(const RecItem &it, int64_t Ng, const double *__restrict__ g,
                                                   const double *__restrict__ E, double *__restrict__ partials) {
    __shared__ double gs[2][32];   // [0]: even degrees, [1]: odd degrees
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w == 0) {
        const bool act = lane < it.nrows;
        const double gr = act ? g[it.row0 + lane] : 0.0;
        const double gm = act && it.mirror ? g[Ng - it.row0 - lane] : 0.0;
        gs[0][lane] = gr + gm;
        gs[1][lane] = gr - gm;
    }
    __syncthreads();
    const int len = it.b - it.a;
    const double *e = E + it.eoff;
    const double *gl = gs[lane & 1];
    double *out = partials + it.out;
    for (int k0 = w * 32; k0 < len; k0 += 32 * SW) {
        const int k = k0 + lane;
        if (k < len) {
            double acc = 0.0;
            for (int r = 0; r < it.nrows; ++r) acc = fma(gl[r], __ldg(e + (int64_t)r * len + k), acc);
            out[k] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// ASY packs: pair p holds items q = 2p, 2p+1 (q = k*M + m) as the real and imaginary
// parts of one complex transform input; arithmetic in the transform precision R.  Each
// item is scaled by its exact power of two s_q = scale[2q] (so that the two items of a
// transform have comparable magnitudes); the scaled factors are formed here from the
// plan's C_{n,m} (forward) or u_m, v_m (inverse) tables, rounded to R, as
//   forward  Cs_q[n] = s_q C_{n,m}          for n >= j_k (0 below)
//   inverse  Us_q[i] = s_q u_m(theta_i)/2,  Vs_q[i] = s_q v_m(theta_i)/2  on box k's rows
// ---------------------------------------------------------------------------
// The two items of pair p: their (block, term) indices and scales, formed once per pair.
struct PairScale {
    int m0, m1;          // terms of items 2p and 2p+1 (m1 < 0: no second item)
    int k0, k1;          // their blocks
    double s0, s1;       // scale[2q] of each
    int e0, e1;          // s0 = 2^e0, s1 = 2^e1 (exact powers of two)
};
__device__ __forceinline__ int pow2_exponent(double s) {
    return (int)((__double_as_longlong(s) >> 52) & 0x7ff) - 1023;
}
__device__ __forceinline__ PairScale pair_scale(int p, int M, int nq, const double *__restrict__ scale) {
    PairScale ps;
    const int q = 2 * p;
    ps.k0 = q / M;
    ps.m0 = q - ps.k0 * M;
    ps.s0 = scale[2 * q];
    ps.e0 = pow2_exponent(ps.s0);
    if (q + 1 < nq) {
        ps.k1 = (q + 1) / M;
        ps.m1 = q + 1 - ps.k1 * M;
        ps.s1 = scale[2 * (q + 1)];
        ps.e1 = pow2_exponent(ps.s1);
    } else {
        ps.k1 = 0;
        ps.m1 = -1;
        ps.s1 = 0.0;
        ps.e1 = 0;
    }
    return ps;
}

// x 2^k, exact, for s = 2^k: the exponent field is moved by integer arithmetic (the FP64
// pipe, a few lanes per clock on this GPU, is the scarce resource of these kernels); zeros,
// subnormals, infinities, NaNs and results outside the normal range take the multiply,
// which gives the same value
__device__ __forceinline__ double mul_pow2(double x, int k, double s) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff), ek = e + k;
    if (e == 0 || e == 0x7ff || ek <= 0 || ek >= 0x7ff) return x * s;
    return __longlong_as_double(b + ((long long)k << 52));
}
__device__ __forceinline__ double neg_if(double x, bool neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}

// FP64 transforms: s_q C_{n,m} c_n formed as (C_{n,m} c_n) s_q, the same value (the scale
// is a power of two); other precisions: the scaled factor is rounded to R first
template <typename V, typename R>
__device__ __forceinline__ void asy_pack_fwd_elem(int64_t n, int p, const PairScale &ps, int64_t N, int64_t L,
                                                  const int *__restrict__ box3, const double *__restrict__ Cnm,
                                                  const double *__restrict__ c, V *__restrict__ buf) {
    V o;
    o.x = 0;
    o.y = 0;
    if (n <= N) {
        if constexpr (std::is_same<R, double>::value) {
            const double cn = c[n];
            if (n >= box3[3 * ps.k0]) o.x = mul_pow2(Cnm[ps.m0 * (N + 1) + n] * cn, ps.e0, ps.s0);
            if (ps.m1 >= 0 && n >= box3[3 * ps.k1]) o.y = mul_pow2(Cnm[ps.m1 * (N + 1) + n] * cn, ps.e1, ps.s1);
        } else {
            const R cn = (R)c[n];
            o.x = (R)(n >= box3[3 * ps.k0] ? Cnm[ps.m0 * (N + 1) + n] * ps.s0 : 0.0) * cn;
            if (ps.m1 >= 0) o.y = (R)(n >= box3[3 * ps.k1] ? Cnm[ps.m1 * (N + 1) + n] * ps.s1 : 0.0) * cn;
        }
    }
    buf[(int64_t)p * L + n] = o;
}

// Inverse: item q contributes s_q u_m(theta_i) g_i / 2 (real) and +-s_q v_m(theta_i) g_i / 2
// (imaginary) on its box's rows; FP64 transforms form (u_m g_i) s_q / 2, the same value.
// The transform input H(idx) = (z(idx) + conj z(L - idx)) / 2, L = 2 Ng, takes row i at
// idx = i and at idx = L - i with the imaginary parts negated, so one call computes row i's
// products once and writes both: rows 1 .. Ng - 1 at i and L - i; the call for i = 0 also
// writes rows 0 and Ng (the ends of the grid, in no box).
template <typename V, typename R>
__device__ __forceinline__ void inv_pack_row(int64_t i, const PairScale &ps, int64_t Ng, const int *__restrict__ box3,
                                             const double *__restrict__ u, const double *__restrict__ v,
                                             const double *__restrict__ g, V &lo, V &hi) {
    const bool in0 = i >= box3[3 * ps.k0 + 1] && i <= box3[3 * ps.k0 + 2];
    const bool in1 = ps.m1 >= 0 && i >= box3[3 * ps.k1 + 1] && i <= box3[3 * ps.k1 + 2];
    if constexpr (std::is_same<R, double>::value) {
        // every load is issued whether or not the row is in the box (0 <= i <= Ng, so it is
        // within the tables), so that the loads of consecutive rows overlap; the box selects
        // afterwards
        const int m1 = ps.m1 >= 0 ? ps.m1 : ps.m0;
        const double gi = __ldg(g + i);
        const double a0 = __ldg(u + ps.m0 * (Ng + 1) + i), b0 = __ldg(v + ps.m0 * (Ng + 1) + i);
        const double a1 = __ldg(u + m1 * (Ng + 1) + i), b1 = __ldg(v + m1 * (Ng + 1) + i);
        double h0r = 0.0, h0i = 0.0, h1r = 0.0, h1i = 0.0;
        if (in0) {
            h0r = mul_pow2(a0 * gi, ps.e0 - 1, 0.5 * ps.s0);
            h0i = mul_pow2(b0 * gi, ps.e0 - 1, 0.5 * ps.s0);
        }
        if (in1) {
            h1r = mul_pow2(a1 * gi, ps.e1 - 1, 0.5 * ps.s1);
            h1i = mul_pow2(b1 * gi, ps.e1 - 1, 0.5 * ps.s1);
        }
        lo.x = h0r - h1i;
        lo.y = h0i + h1r;
        hi.x = h0r + h1i;
        hi.y = h1r - h0i;
    } else {
        const R gi = (R)g[i];
        const double sc0 = 0.5 * ps.s0;
        const R u0 = (R)(in0 ? sc0 * u[ps.m0 * (Ng + 1) + i] : 0.0), v0 = (R)(in0 ? sc0 * v[ps.m0 * (Ng + 1) + i] : 0.0);
        const R h0r = u0 * gi, h0i = v0 * gi;
        R h1r = 0, h1i = 0;
        if (ps.m1 >= 0) {
            const double sc1 = 0.5 * ps.s1;
            const R u1 = (R)(in1 ? sc1 * u[ps.m1 * (Ng + 1) + i] : 0.0);
            const R v1 = (R)(in1 ? sc1 * v[ps.m1 * (Ng + 1) + i] : 0.0);
            h1r = u1 * gi;
            h1i = v1 * gi;
        }
        lo.x = h0r - h1i;
        lo.y = h0i + h1r;
        hi.x = h0r + h1i;
        hi.y = h1r - h0i;
    }
}
// pair p's transform input at rows i (0 <= i < Ng) and L - i, and at 0 and Ng for i = 0
template <typename V, typename R>
__device__ __forceinline__ void asy_pack_inv_elem(int64_t i, int p, const PairScale &ps, int64_t Ng, int64_t L,
                                                  const int *__restrict__ box3, const double *__restrict__ u,
                                                  const double *__restrict__ v, const double *__restrict__ g,
                                                  V *__restrict__ buf) {
    V *row = buf + (int64_t)p * L;
    V lo, hi;
    inv_pack_row<V, R>(i, ps, Ng, box3, u, v, g, lo, hi);
    row[i] = lo;
    if (i > 0) {
        row[L - i] = hi;
    } else {
        inv_pack_row<V, R>(Ng, ps, Ng, box3, u, v, g, lo, hi);
        row[Ng] = lo;
    }
}

// transform output components as doubles
__device__ __forceinline__ double re_d(double2 v) { return v.x; }
__device__ __forceinline__ double im_d(double2 v) { return v.y; }
__device__ __forceinline__ double re_d(float2 v) { return (double)v.x; }
__device__ __forceinline__ double im_d(float2 v) { return (double)v.y; }
__device__ __forceinline__ double re_d(dfc v) { return df_to(dfc_re(v)); }
__device__ __forceinline__ double im_d(dfc v) { return df_to(dfc_im(v)); }

// ---------------------------------------------------------------------------
// combine, forward: row i's REC segment partials plus the asymptotic terms of its deepest
// box; writes the even extension of y (length 2N, N the grid) for the final DCT-I
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ void combine_fwd_elem(int64_t i, int64_t N, int64_t L, int M, const int *__restrict__ rowk,
                                                 const double *__restrict__ scale, const double *__restrict__ u,
                                                 const double *__restrict__ v, const V *__restrict__ buf,
                                                 const int64_t *__restrict__ row_base,
                                                 const int *__restrict__ row_nseg,
                                                 const double *__restrict__ partials, double2 *__restrict__ ext) {
    const int nseg = row_nseg[i];
    const int64_t base = row_base[i];
    // rows near x = +-1 have up to N / seg_len segments: eight loads in flight, four sums
    double ya[4] = {0.0, 0.0, 0.0, 0.0};
    int s = 0;
    for (; s + 8 <= nseg; s += 8) {
        double pv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) pv[j] = partials[base + (int64_t)(s + j) * 32];
#pragma unroll
        for (int j = 0; j < 8; ++j) ya[j & 3] += pv[j];
    }
    for (; s < nseg; ++s) ya[0] += partials[base + (int64_t)s * 32];
    double y = (ya[0] + ya[1]) + (ya[2] + ya[3]);
    const int k = rowk[i];
    if (k >= 0) {
        const int64_t im = i == 0 ? 0 : L - i;
        for (int m = 0; m < M; ++m) {
            const int q = k * M + m, p = q >> 1;
            const V Z = buf[(int64_t)p * L + i], W = buf[(int64_t)p * L + im];
            double re, imv;
            if ((q & 1) == 0) {
                re = 0.5 * (re_d(Z) + re_d(W));
                imv = 0.5 * (im_d(Z) - im_d(W));
            } else {
                re = 0.5 * (im_d(Z) + im_d(W));
                imv = 0.5 * (re_d(W) - re_d(Z));
            }
            const double us = scale[2 * q + 1];
            y = fma(u[m * (N + 1) + i] * us, re, y);
            y = fma(-v[m * (N + 1) + i] * us, imv, y);
        }
    }
    ext[i] = make_double2(y, 0.0);
    if (i >= 1 && i < N) ext[2 * N - i] = make_double2(y, 0.0);
}

// c_k = Re Z(k) / G, halved at k = 0 and k = G (inverse scaled DCT-I on the grid G >= N)
__device__ __forceinline__ void dct_finish_elem(int64_t k, int64_t G, const double2 *__restrict__ Z,
                                                double *__restrict__ out) {
    double v = Z[k].x / (double)G;
    if (k == 0 || k == G) v *= 0.5;
    out[k] = v;
}

// inverse front end: [c; 0] of length L as complex values
__device__ __forceinline__ void inv_front_pack_elem(int64_t k, int64_t N, const double *__restrict__ c,
                                                    double2 *__restrict__ buf) {
    buf[k] = make_double2(k <= N ? c[k] : 0.0, 0.0);
}

// g_i = w_i p_N(x_i) on the 2N grid (Clenshaw--Curtis weights)
__device__ __forceinline__ void inv_g_elem(int64_t i, const double2 *__restrict__ F, const double *__restrict__ w,
                                           double *__restrict__ g) {
    g[i] = w[i] * F[i].x;
}

// Sum of the recurrence partials of every item covering degree n, in a fixed order that
// does not depend on the block's size: logical warp k (0 <= k < 32) takes items k, k + 32,
// k + 64, ... (round robin, so that short segments spread over all of them), 32 at a time:
// lane l loads the descriptor of the l-th, the warp broadcasts them by shuffles, and eight
// partial loads are in flight; four interleaved accumulators; the 32 logical warps' sums are
// added in order.  A block of W warps runs logical warps w, w + W, ... on warp w: W = 32 for
// one large transform (its heavy segments have few blocks), fewer for the grouped batch's
// many small ones; every W gives the same bits.  Block `blk` covers the degrees from 32 blk.
constexpr int RED_LOGICAL = 32;
template <int W>
__device__ __forceinline__ void inv_reduce_block(int64_t blk, int64_t N, int seg_len,
                                                 const int64_t *__restrict__ seg_ptr,
                                                 const int64_t *__restrict__ seg_out, const int *__restrict__ seg_b,
                                                 const double *__restrict__ partials, double *__restrict__ y) {
    static_assert(RED_LOGICAL % W == 0, "the logical warps are shared out evenly");
    __shared__ double red[RED_LOGICAL][33];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n0 = blk * 32, n = n0 + lane;
    const int64_t s = n0 / seg_len, off = n - s * seg_len;
    const int64_t q0 = seg_ptr[s], q1 = seg_ptr[s + 1];
    for (int lw = w; lw < RED_LOGICAL; lw += W) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        const int64_t kmax = q1 - q0 > lw ? (q1 - q0 - lw + RED_LOGICAL - 1) / RED_LOGICAL : 0;   // its items
        for (int64_t kb = 0; kb < kmax; kb += 32) {
            const int64_t qq = q0 + lw + (int64_t)RED_LOGICAL * (kb + lane);
            const bool ok = kb + lane < kmax;
            const int64_t so = ok ? seg_out[qq] : 0;
            const int sb = ok ? seg_b[qq] : 0;
            const int cnt = (int)min((int64_t)32, kmax - kb);
            int j = 0;
            for (; j + 8 <= cnt; j += 8) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int64_t o = __shfl_sync(0xffffffffu, so, j + t);
                    const int b = __shfl_sync(0xffffffffu, sb, j + t);
                    if (n < b) acc[t & 3] += partials[o + off];
                }
            }
            for (; j < cnt; ++j) {
                const int64_t o = __shfl_sync(0xffffffffu, so, j);
                const int b = __shfl_sync(0xffffffffu, sb, j);
                if (n < b) acc[0] += partials[o + off];
            }
        }
        red[lw][lane] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();
    if (w == 0 && n <= N) {
        double t = 0.0;
        for (int k = 0; k < RED_LOGICAL; ++k) t += red[k][lane];
        y[n] = t;
    }
}

// combine, inverse: y_n = REC^T + sum_m C_{n,m} ASY^T on degree n's block, c_jac_n = y_n / A_n.
// exps (double-float form only): the transposed blocks ran on g scaled by 2^-e, and so did
// the recurrence when rec_scaled; both are unscaled here.
template <typename V>
__device__ __forceinline__ void combine_inv_elem(int64_t n, int64_t N, int64_t L, int M, int nblk,
                                                 const int *__restrict__ box3, const double *__restrict__ scale,
                                                 const double *__restrict__ Cnm, const V *__restrict__ buf,
                                                 const double *__restrict__ yrec, const double *__restrict__ s_n,
                                                 const int *__restrict__ exps, int rec_scaled,
                                                 double *__restrict__ out) {
    const double ua = exps ? ldexp(1.0, exps[CJT_EXP_BLOCKS]) : 1.0;
    double y = rec_scaled ? ua * yrec[n] : yrec[n];
    // degree n belongs to block k when j_k <= n < top_k (top_0 = N+1, top_k = j_{k-1})
    int k = -1;
    for (int kk = 0; kk < nblk; ++kk) {
        const int64_t top = kk == 0 ? N + 1 : box3[3 * (kk - 1)];
        if (n >= box3[3 * kk] && n < top) k = kk;
    }
    if (k >= 0) {
        for (int m = 0; m < M; ++m) {
            const int q = k * M + m, p = q >> 1;
            const V Z = buf[(int64_t)p * L + n];
            const double R = (q & 1) ? im_d(Z) : re_d(Z);
            y = fma(Cnm[m * (N + 1) + n] * (scale[2 * q + 1] * ua), R, y);
        }
    }
    out[n] = s_n[n] * y;
}

}  // namespace cjt_kern
