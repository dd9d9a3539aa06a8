// Planification (Sec. 4, steps 1a-1e): everything that depends only on
// (N, alpha, beta, options) is computed here once, on the GPU, and kept in
// device memory for every later execution.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "cjt_df.cuh"
#include "cjt_internal.cuh"

namespace {


// --------------------------------------------------------------------------
// 1c: recurrence coefficients (Sec. 1.2) and Reinsch ratios at x0 = +-1 (Sec. 4.2)
// --------------------------------------------------------------------------
__global__ void k_rec_tables(int64_t nmax, double a, double b, RecTables t) {
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n > nmax) return;
    const RecRow r = cjt_rec_row(n, a, b);
    t.A[n] = r.A;
    t.B[n] = r.B;
    t.C[n] = r.C;
    t.rf_p[n] = r.rf_p;
    t.rf_m[n] = r.rf_m;
    t.Ce_p[n] = r.Ce_p;
    t.Ce_m[n] = r.Ce_m;
    t.Cr_p[n] = r.Cr_p; t.rbinv_p[n] = r.rbinv_p;
    t.Cr_m[n] = r.Cr_m; t.rbinv_m[n] = r.rbinv_m;
}

// --------------------------------------------------------------------------
// Coefficients C_{n,m} of the plan's expansion: Hahn's (Eq. "Cnmab", computed by
// Eq. "Cnmabasy"/"Cnmabrec") or the ultraspherical C^lambda_{n,m} (App. B.1)
// --------------------------------------------------------------------------
__global__ void k_hahn_C(int64_t N, int Mp1, AsyExp e, double *Cnm) {
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (n > N || m >= Mp1) return;
    Cnm[m * (N + 1) + n] = cjt_asy_C(e, n, m);
}

// --------------------------------------------------------------------------
// diagonals u_m(theta_i), v_m(theta_i) (Eq. "Jacasyuv"; App. B.1) on the grid
// theta_i = pi i / Ng
// --------------------------------------------------------------------------
__global__ void k_hahn_uv(int64_t Ng, int M, AsyExp e, double *u, double *v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > Ng) return;
    for (int m = 0; m < M; ++m) {
        double su = 0.0, sv = 0.0;
        if (i != 0 && i != Ng) cjt_asy_uv(e, m, i, Ng, &su, &sv);
        u[m * (Ng + 1) + i] = su;
        v[m * (Ng + 1) + i] = sv;
    }
}

// envelope of the remainder term M (Sec. 2.2; App. B.1); +inf at the end points
__global__ void k_envelope(int64_t Ng, int M, AsyExp e, double *g) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > Ng) return;
    g[i] = (i == 0 || i == Ng) ? INFINITY : cjt_asy_env(e, M, i, Ng);
}

__global__ void k_box_init(int nk, int *box) {
    int k = threadIdx.x;
    if (k < nk) { box[2 * k] = INT_MAX; box[2 * k + 1] = -1; }
}

// rows where 2 C_{j_k,M} g_M(theta_i) < eps: the smallest and largest such i per block
__global__ void k_boxes(int64_t Ng, const double *g, int nk, const double *thr, int *box) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x + 1; i < Ng;
         i += (int64_t)gridDim.x * blockDim.x) {
        double gi = g[i];
        for (int k = 0; k < nk; ++k) {
            if (gi < thr[k]) {
                atomicMin(&box[2 * k], (int)i);
                atomicMax(&box[2 * k + 1], (int)i);
            }
        }
    }
}

// deepest box containing each row (boxes are nested), -1 if none
__global__ void k_rowk(int64_t Ng, int nblk, const int *box3, int *rowk) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > Ng) return;
    int kk = -1;
    for (int k = 0; k < nblk; ++k)
        if (i >= box3[3 * k + 1] && i <= box3[3 * k + 2]) kk = k;
    rowk[i] = kk;
}

// x (plain rows) or delta = x - x0 (Reinsch rows: -2 sin^2(theta/2) at x0 = 1, 2 cos^2(theta/2)
// at x0 = -1, Sec. 4.2) of grid row `row`
__device__ __forceinline__ void rec_row_point(int row, int mode, int64_t Ng, double &x, double &delta) {
    x = 0.0;
    delta = 0.0;
    if (mode == REC_PLAIN) {
        x = cospi((double)row / (double)Ng);
    } else if (mode == REC_REINSCH_P1) {
        const double sv = sinpi((double)row / (2.0 * (double)Ng));
        delta = -2.0 * sv * sv;
    } else {
        const double sv = sinpi((double)(Ng - row) / (2.0 * (double)Ng));
        delta = 2.0 * sv * sv;
    }
}

// --------------------------------------------------------------------------
// Forward-recurrence state (plain or Reinsch-modified, Sec. 4.2) at every degree-segment
// start of the rows with more than one segment, by a chunked scan.  The recurrence is
// linear in its two-term state, so a run of `len` degrees maps the state at its start to the
// state at its end by a 2x2 matrix: k_rec_seg_maps runs the recurrence over run k from the
// two unit states (the matrix's columns), one thread per (row, run); k_rec_seg_carry then
// applies the matrices in order, one thread per row, and stores the state at every segment
// start.  The runs (len divides the segment length, at most 512 degrees) are shorter than a
// segment: a dependent FP64 chain is slow, so many short chains beat few long ones.
//   lsrow = {row, mode, state_base, lane, nseg} per row; loff[q] = first run of row q
// --------------------------------------------------------------------------
__global__ void k_rec_seg_maps(int64_t nlong, int64_t nmaps, const int *__restrict__ lsrow,
                               const int64_t *__restrict__ loff, int64_t Ng, int len, RecTables t,
                               double *__restrict__ maps) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nmaps) return;
    int64_t lo = 0, hi = nlong - 1;   // the row q with loff[q] <= g < loff[q + 1]
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (loff[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const int64_t q = lo, k = g - loff[q];
    const int *r = lsrow + 5 * q;
    const int row = r[0], mode = r[1];
    double x, delta;
    rec_row_point(row, mode, Ng, x, delta);
    const int64_t n0 = k * len;
    // columns: state (1, 0) and (0, 1) at degree n0
    double p0 = 1.0, q0 = 0.0, p1 = 0.0, q1 = 1.0;
    if (mode == REC_PLAIN) {
#pragma unroll 4
        for (int kk = 0; kk < len; ++kk) {
            const int64_t n = n0 + kk;
            const double an = fma(__ldg(t.A + n), x, __ldg(t.B + n)), cn = __ldg(t.C + n);
            const double pn0 = fma(an, p0, -cn * q0), pn1 = fma(an, p1, -cn * q1);
            q0 = p0; p0 = pn0;
            q1 = p1; p1 = pn1;
        }
    } else {
        const double *Ce = mode == REC_REINSCH_P1 ? t.Ce_p : t.Ce_m;
        const double *rf = mode == REC_REINSCH_P1 ? t.rf_p : t.rf_m;
#pragma unroll 4
        for (int kk = 0; kk < len; ++kk) {
            const int64_t n = n0 + kk;
            const double ad = __ldg(t.A + n) * delta, ce = __ldg(Ce + n), f = __ldg(rf + n);
            const double e0 = fma(ad, p0, ce * q0), e1 = fma(ad, p1, ce * q1);
            p0 = fma(p0, f, e0); q0 = e0;
            p1 = fma(p1, f, e1); q1 = e1;
        }
    }
    double *m = maps + g * 4;
    m[0] = p0; m[1] = q0; m[2] = p1; m[3] = q1;
}

__global__ void k_rec_seg_carry(int64_t nlong, const int *__restrict__ lsrow, const int64_t *__restrict__ loff,
                                int per, const double *__restrict__ maps, double *__restrict__ states) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nlong) return;
    const int *r = lsrow + 5 * q;
    const int base = r[2], lane = r[3], nseg = r[4];
    struct Map { double x, y, z, w; };
    const Map *mp = reinterpret_cast<const Map *>(maps) + loff[q];
    const int nrun = (nseg - 1) * per;   // `per` runs per segment
    double a = 1.0, b = 0.0;   // (p, second state) at degree 0
    for (int k0 = 0; k0 < nrun; k0 += 8) {
        Map m[8];   // loaded ahead: the maps do not depend on the carried state
#pragma unroll
        for (int j = 0; j < 8; ++j) m[j] = k0 + j < nrun ? mp[k0 + j] : Map{0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + j;
            if (k >= nrun) break;
            const double na = fma(a, m[j].x, b * m[j].z), nb = fma(a, m[j].y, b * m[j].w);
            a = na;
            b = nb;
            if ((k + 1) % per == 0) {   // the start of segment (k + 1) / per
                double *st = states + ((int64_t)(base + (k + 1) / per - 1) * 32 + lane) * 2;
                st[0] = a;
                st[1] = b;
            }
        }
    }
}

// --------------------------------------------------------------------------
// pre-scaled transform inputs (the scale of each item is an exact power of two)
// --------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ R to_prec(double v) { return (R)v; }
template <> __device__ __forceinline__ dfs to_prec<dfs>(double v) { return df_from(v); }

template <typename R>
__global__ void k_scaled_C(int64_t N, int M, int nq, const int *__restrict__ box3, const double *__restrict__ Cnm,
                           const double *__restrict__ scale, R *__restrict__ out) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (n > N || q >= nq) return;
    const int k = q / M, m = q - k * M;
    out[(int64_t)q * (N + 1) + n] = to_prec<R>(n >= box3[3 * k] ? Cnm[m * (N + 1) + n] * scale[2 * q] : 0.0);
}

template <typename R>
__global__ void k_scaled_uv(int64_t Ng, int M, int nq, const int *__restrict__ box3, const double *__restrict__ u,
                            const double *__restrict__ v, const double *__restrict__ scale, R *__restrict__ U,
                            R *__restrict__ V) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i > Ng || q >= nq) return;
    const int k = q / M, m = q - k * M;
    const bool in = i >= box3[3 * k + 1] && i <= box3[3 * k + 2];
    const double sc = 0.5 * scale[2 * q];
    U[(int64_t)q * (Ng + 1) + i] = to_prec<R>(in ? sc * u[m * (Ng + 1) + i] : 0.0);
    V[(int64_t)q * (Ng + 1) + i] = to_prec<R>(in ? sc * v[m * (Ng + 1) + i] : 0.0);
}

// --------------------------------------------------------------------------
// rec_store: the values P_n(x_i) of each recurrence item, by the same forward
// recurrences (plain, or Reinsch-modified near x = +-1, Sec. 4.2) from the item's
// segment state.  layout 0: [k][lane] (forward matvec), 1: [lane][k] (transposed).
// --------------------------------------------------------------------------
__global__ void k_rec_fill(const RecItem *__restrict__ items, int64_t nitems, int64_t Ng, RecTables t,
                           const double *__restrict__ states, double *__restrict__ E, int layout) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nitems) return;
    const RecItem it = items[w];
    const bool active = lane < it.nrows;
    const int row = it.row0 + min(lane, it.nrows - 1);
    double P1 = 1.0, P2 = 0.0;
    if (active && it.state >= 0) {
        const double2 sv = reinterpret_cast<const double2 *>(states)[(int64_t)it.state * 32 + lane];
        P1 = sv.x;
        P2 = sv.y;
    }
    const int len = it.b - it.a;
    double *e = E + it.eoff;
    auto put = [&](int k, double v) {
        v = active ? v : 0.0;
        if (layout == 0) e[(int64_t)k * 32 + lane] = v;
        else e[(int64_t)lane * len + k] = v;
    };
    if (it.mode == REC_PLAIN) {
        const double x = cospi((double)row / (double)Ng);
        double p = P1, pm = P2;
        for (int k = 0; k < len; ++k) {
            const int n = it.a + k;
            put(k, p);
            const double pn = fma(fma(__ldg(t.A + n), x, __ldg(t.B + n)), p, -__ldg(t.C + n) * pm);
            pm = p;
            p = pn;
        }
    } else {
        const bool plus = it.mode == REC_REINSCH_P1;
        double delta;
        if (plus) {
            const double sv = sinpi((double)row / (2.0 * (double)Ng));
            delta = -2.0 * sv * sv;
        } else {
            const double sv = sinpi((double)(Ng - row) / (2.0 * (double)Ng));
            delta = 2.0 * sv * sv;
        }
        const double *Ce = plus ? t.Ce_p : t.Ce_m;
        const double *rf = plus ? t.rf_p : t.rf_m;
        double p = P1, ee = P2;
        for (int k = 0; k < len; ++k) {
            const int n = it.a + k;
            put(k, p);
            const double en = fma(__ldg(t.A + n) * delta, p, __ldg(Ce + n) * ee);
            p = fma(p, __ldg(rf + n), en);
            ee = en;
        }
    }
}

// --------------------------------------------------------------------------
// inverse: modified Chebyshev moments by the three-term recurrence of Sec. 3.1
// with mu_1 = (beta-alpha)/(alpha+beta+2) mu_0, written as the even extension
// of length 2*Ng used by the DCT-I of Eq. "CCweights".
// --------------------------------------------------------------------------
// The recurrence for k >= 1 is the linear map (mu_{k-1}, mu_k) -> (mu_k, mu_{k+1}) with
//   mu_{k+1} = c1_k mu_k + c0_k mu_{k-1},  c1_k = -2(a-b)/(a+b+k+2),  c0_k = -(a+b-k+2)/(a+b+k+2).
// It is evaluated as a chunked scan: each chunk of kMomChunk steps forms its 2x2 transfer
// matrix in parallel, a block-wide scan of the matrices gives the true state at every chunk
// start, and every chunk then reruns its steps from that state.  The forward recurrence is stable in the square
// (Sec. 3.1), so the basis solutions carried by the transfer matrices do not outgrow mu.
constexpr int kMomChunk = 64;

__device__ __forceinline__ void mom_coeffs(double ab, double amb, int64_t k, double *c0, double *c1) {
    const double inv = 1.0 / (ab + (double)k + 2.0);
    *c1 = -2.0 * amb * inv;
    *c0 = -(ab - (double)k + 2.0) * inv;
}

struct Mat2 {   // 2x2 transfer matrix [[x0, x1], [y0, y1]] of one chunk
    double x0, x1, y0, y1;
};

__global__ void k_mom_transfer(int64_t Ng, double a, double b, int64_t nchunk, Mat2 *T) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nchunk) return;
    const double ab = a + b, amb = a - b;
    double x0 = 1.0, y0 = 0.0, x1 = 0.0, y1 = 1.0;   // columns: state (mu_{k-1}, mu_k)
    const int64_t k0 = 1 + c * kMomChunk, k1 = min(k0 + kMomChunk, Ng);
    for (int64_t k = k0; k < k1; ++k) {
        double c0, c1;
        mom_coeffs(ab, amb, k, &c0, &c1);
        const double nx = fma(c1, y0, c0 * x0), ny = fma(c1, y1, c0 * x1);
        x0 = y0; y0 = nx;
        x1 = y1; y1 = ny;
    }
    T[c] = Mat2{x0, x1, y0, y1};
}

// The state at every chunk start: start[c] = T[c-1] ... T[0] (mu0, mu1).  One block: thread
// j multiplies the maps of its run of consecutive chunks, the block scans those products in
// shared memory (Hillis--Steele, later runs' products on the left), and each thread then
// carries the state through its own run from the product of all earlier runs.
constexpr int kMomScanThreads = 1024;
__device__ __forceinline__ Mat2 mat2_mul(const Mat2 &l, const Mat2 &r) {   // l r
    return Mat2{fma(l.x0, r.x0, l.x1 * r.y0), fma(l.x0, r.x1, l.x1 * r.y1), fma(l.y0, r.x0, l.y1 * r.y0),
                fma(l.y0, r.x1, l.y1 * r.y1)};
}
__global__ void __launch_bounds__(kMomScanThreads) k_mom_carry(int64_t nchunk, double mu0, double mu1,
                                                               const Mat2 *__restrict__ T,
                                                               double2 *__restrict__ start) {
    __shared__ Mat2 sc[kMomScanThreads];
    const int j = threadIdx.x;
    const int64_t per = (nchunk + kMomScanThreads - 1) / kMomScanThreads;
    const int64_t c0 = min((int64_t)j * per, nchunk), c1 = min(c0 + per, nchunk);
    Mat2 prod{1.0, 0.0, 0.0, 1.0};
    for (int64_t c = c0; c < c1; ++c) prod = mat2_mul(T[c], prod);
    sc[j] = prod;
    __syncthreads();
    for (int d = 1; d < kMomScanThreads; d <<= 1) {
        const Mat2 mine = sc[j];
        const Mat2 earlier = j >= d ? sc[j - d] : Mat2{1.0, 0.0, 0.0, 1.0};
        __syncthreads();
        sc[j] = mat2_mul(mine, earlier);
        __syncthreads();
    }
    // state at c0: the product of all earlier runs applied to (mu0, mu1)
    double u = mu0, v = mu1;
    if (j > 0) {
        const Mat2 e = sc[j - 1];
        u = fma(e.x0, mu0, e.x1 * mu1);
        v = fma(e.y0, mu0, e.y1 * mu1);
    }
    for (int64_t c = c0; c < c1; ++c) {
        start[c] = make_double2(u, v);
        const Mat2 m = T[c];
        const double nu = fma(m.x0, u, m.x1 * v), nv = fma(m.y0, u, m.y1 * v);
        u = nu;
        v = nv;
    }
}

// writes the even extension of length 2 Ng used by the DCT-I of Eq. "CCweights"
__global__ void k_mom_fill(int64_t Ng, double a, double b, int64_t nchunk, const double2 *start, double2 *ext) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nchunk) return;
    const double ab = a + b, amb = a - b;
    double u = start[c].x, v = start[c].y;   // (mu_{k0-1}, mu_{k0})
    const int64_t k0 = 1 + c * kMomChunk, k1 = min(k0 + kMomChunk, Ng);
    if (c == 0) {
        ext[0] = make_double2(u, 0.0);
        ext[1] = make_double2(v, 0.0);
        if (Ng > 1) ext[2 * Ng - 1] = make_double2(v, 0.0);
    }
    for (int64_t k = k0; k < k1; ++k) {
        double c0, c1;
        mom_coeffs(ab, amb, k, &c0, &c1);
        const double w = fma(c1, v, c0 * u);
        u = v;
        v = w;
        ext[k + 1] = make_double2(w, 0.0);
        if (k + 1 < Ng) ext[2 * Ng - (k + 1)] = make_double2(w, 0.0);
    }
}

// w_i = (eps_i / Ng) Re DFT_{2Ng}(ext)_i,  eps_0 = eps_Ng = 1/2
__global__ void k_cc_weights(int64_t Ng, const double2 *F, double *w) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > Ng) return;
    double v = F[i].x / (double)Ng;
    if (i == 0 || i == Ng) v *= 0.5;
    w[i] = v;
}

// s_n = 1/A_n (Eq. "Anab"), by Eq. "Anabasy" for n + min(a, b, a+b, 0) >= 8
__global__ void k_inv_norm(int64_t N, double a, double b, double *s) {
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n > N) return;
    const double ab = a + b, nn = (double)n;
    const double mn = fmin(fmin(a, b), fmin(ab, 0.0));
    double A;
    if (nn + mn >= 8.0) {
        const double r = nn + ab + 1.0, q = nn + 1.0;
        const double t = (0.5 * nn + a + 0.25) * log1p(-b / r) + (0.5 * nn + b + 0.25) * log1p(-a / r) +
                         (0.5 * nn + 0.25) * (log1p(a / q) + log1p(b / q));
        A = exp2(ab + 1.0) / (2.0 * nn + ab + 1.0) * exp(t) * cjt_stirling_S(nn + a + 1.0) *
            cjt_stirling_S(nn + b + 1.0) / (cjt_stirling_S(nn + ab + 1.0) * cjt_stirling_S(nn + 1.0));
    } else if (n == 0) {
        A = exp2(ab + 1.0) * tgamma(a + 1.0) * tgamma(b + 1.0) / tgamma(ab + 2.0);
    } else {
        A = exp2(ab + 1.0) * tgamma(nn + a + 1.0) * tgamma(nn + b + 1.0) /
            ((2.0 * nn + ab + 1.0) * tgamma(nn + ab + 1.0) * tgamma(nn + 1.0));
    }
    s[n] = 1.0 / A;
}

// twiddles omega_L^k = exp(-2 pi i k / L)
__global__ void k_twiddles(int64_t L, double2 *tw64, float2 *tw32, dfc *twdf) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= L) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    tw64[k] = make_double2(c, s);
    if (tw32) tw32[k] = make_float2((float)c, (float)s);
    if (twdf) twdf[k] = dfc_make(df_from(c), df_from(s));
}

// CJT_DFLOAT, forward grid: u_m(theta_i) and v_m(theta_i) times 1/2 and the unscaling of
// item (k(i), m), k(i) the deepest box of row i, as double-floats in place (0 outside the
// boxes).  u_m and v_m alone grow beyond the float range near the ends of the wider boxes
// for large m; the products are bounded by the partition tolerance's envelope.
__global__ void k_fwd_uv_to_df(int64_t Ng, int M, const int *__restrict__ rowk, const double *__restrict__ scale,
                               double *__restrict__ u, double *__restrict__ v) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (i > Ng) return;
    const int k = rowk[i];
    const int64_t at = (int64_t)m * (Ng + 1) + i;
    const double sc = k >= 0 ? 0.5 * scale[2 * (k * M + m) + 1] : 0.0;
    const double uv = u[at] * sc, vv = v[at] * sc;
    reinterpret_cast<dfs *>(u)[at] = df_from(uv);
    reinterpret_cast<dfs *>(v)[at] = df_from(vv);
}

// stage twiddle tables (Twiddles::stw) from omega_{Ltab}^k, in each precision in use
__global__ void k_stage_twiddles(int lmax, int logLtab, const double2 *__restrict__ tw64, double2 *stw64,
                                 float2 *stw32, dfc *stwdf) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= stw_base(lmax + 1)) return;
    int lb = 2;
    while (stw_base(lb + 1) <= t) ++lb;
    const int64_t h = 1LL << (lb - 2), rel = t - stw_base(lb);
    const int64_t r = rel / h, n0 = rel - r * h;
    const double2 w = tw64[((r + 1) * n0) << (logLtab - lb)];
    if (stw64) stw64[t] = w;
    if (stw32) stw32[t] = make_float2((float)w.x, (float)w.y);
    if (stwdf) stwdf[t] = dfc_make(df_from(w.x), df_from(w.y));
}

// FMA-form twiddles of the FP64 decimation-in-time stages (TwFma): entry twfma_base(lb) + q
// for q < 2^(lb-2), from omega_{Ltab}^k
__global__ void k_fma_twiddles(int lmax, int logLtab, const double2 *__restrict__ tw64, TwFma *out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= twfma_base(lmax + 1)) return;
    int lb = 2;
    while (twfma_base(lb + 1) <= t) ++lb;
    const int64_t q = t - twfma_base(lb);
    double tt[3], sx[3], sy[3];
    int flags = 0;
    for (int j = 1; j <= 3; ++j) {
        const double2 w = tw64[((int64_t)j * q) << (logLtab - lb)];
        if (fabs(w.x) >= fabs(w.y)) {   // sigma (1 + i t)
            tt[j - 1] = w.y / w.x;
            sx[j - 1] = w.x;
            sy[j - 1] = w.x;
        } else {                        // sigma (t + i), parts swapped in the butterfly
            tt[j - 1] = w.x / w.y;
            sx[j - 1] = -w.y;
            sy[j - 1] = w.y;
            flags |= 1 << (j - 1);
        }
    }
    TwFma r;
    r.t1 = tt[0]; r.t2 = tt[1]; r.t3 = tt[2];
    r.s1x = sx[0]; r.s1y = sy[0];
    r.s2x = sx[1]; r.s2y = sy[1];
    r.rx = sx[2] / sx[0]; r.ry = sy[2] / sy[0];
    r.flags = flags;
    r.pad_ = 0;
    out[t] = r;
}

// doubles -> double-floats in place (same 8 bytes per entry): stored recurrence values
__global__ void k_to_df_inplace(int64_t n, double *E) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = E[i];
    reinterpret_cast<dfs *>(E)[i] = df_from(v);
}


// --------------------------------------------------------------------------
// Error bound of the mixed form (FP32 transforms).  A transform of length L in FP32
// (unit roundoff u = 2^-24) computes each output within eps_F sum_n |z_n| of the exact
// one: every radix-4 stage adds at most 5u times the sum of the moduli of the inputs that
// feed an output (two levels of additions, the rounded twiddle and the fused complex
// multiply), the radix-2 stage u, the four-step twiddle 3u, and the rounding of the
// packed inputs to float 3u; the transform's unit-modulus weights carry earlier errors
// without growth.  Conservatively eps_F = u (3 log2 L + 8).
//   forward: row i of box k adds sum_m (u_m Re F_q - v_m Im F_q) / s_q, where the complex
//   transform holds items q and q' (its pair partner) scaled by s_q, s_q', and
//   sum_n |a_q[n]| <= s_q C_{j_k,m} ||c||_1 (C_{n,m} decreases in n).  The final inverse
//   DCT-I maps max |dy| to at most 2 max |dy| in the coefficients:
//     err_fwd = 2 eps_F max_i sum_m (|u_m| + |v_m|)(theta_i) (C_{j_k,m} + s_q'/s_q C_{j_k',m'}).
//   inverse: degree n of block k adds C_{n,m} R_q(n) / s_q, with the transform's inputs of
//   moduli <= s_q (|u_m| + |v_m|) |g_i| / 2 at rows i and Ng' - i of the box, |g_i| <=
//   w_i ||c||_1 (|T_k| <= 1), and the result is scaled by 1/A_n:
//     err_inv = eps_F max_n (1/A_n) sum_m C_{n,m} (U_q + s_q'/s_q U_q'),
//     U_q = sum_{i in box k} |w_i| (|u_m| + |v_m|)(theta_i).
// --------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_pos(double *at, double v) {
    // non-negative doubles order like their bit patterns as signed 64-bit integers
    atomicMax(reinterpret_cast<long long *>(at), __double_as_longlong(v));
}

__global__ void k_err_fwd(int64_t N, int64_t Ng, int M, int nq, const int *__restrict__ rowk,
                          const int *__restrict__ box3, const double *__restrict__ Cnm,
                          const double *__restrict__ scale, const double *__restrict__ u,
                          const double *__restrict__ v, double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > Ng) return;
    const int k = rowk[i];
    if (k < 0) return;
    const int64_t j = box3[3 * k];
    double s = 0.0;
    for (int m = 0; m < M; ++m) {
        const int q = k * M + m, qp = q ^ 1;
        double c = Cnm[m * (N + 1) + j];
        if (qp < nq) {
            const int kp = qp / M, mp = qp - kp * M;
            c += scale[2 * qp] * scale[2 * q + 1] * Cnm[mp * (N + 1) + box3[3 * kp]];
        }
        s += (fabs(u[m * (Ng + 1) + i]) + fabs(v[m * (Ng + 1) + i])) * c;
    }
    atomic_max_pos(out, s);
}

// U_q for every item q, one block per q, summed in a fixed order
__global__ void k_err_inv_U(int64_t Ng, int M, const int *__restrict__ box3, const double *__restrict__ w,
                            const double *__restrict__ u, const double *__restrict__ v, double *__restrict__ U) {
    __shared__ double red[256];
    const int q = blockIdx.x, k = q / M, m = q - k * M;
    const int64_t i1 = box3[3 * k + 1], i2 = box3[3 * k + 2];
    double s = 0.0;
    for (int64_t i = i1 + threadIdx.x; i <= i2; i += blockDim.x)
        s += fabs(w[i]) * (fabs(u[m * (Ng + 1) + i]) + fabs(v[m * (Ng + 1) + i]));
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) U[q] = red[0];
}

__global__ void k_err_inv(int64_t N, int M, int nblk, int nq, const int *__restrict__ box3,
                          const double *__restrict__ Cnm, const double *__restrict__ scale,
                          const double *__restrict__ U, const double *__restrict__ s_n, double *__restrict__ out) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n > N) return;
    int k = -1;
    for (int kk = 0; kk < nblk; ++kk) {
        const int64_t top = kk == 0 ? N + 1 : box3[3 * (kk - 1)];
        if (n >= box3[3 * kk] && n < top) k = kk;
    }
    if (k < 0) return;
    double s = 0.0;
    for (int m = 0; m < M; ++m) {
        const int q = k * M + m, qp = q ^ 1;
        double uq = U[q];
        if (qp < nq) uq += scale[2 * qp] * scale[2 * q + 1] * U[qp];
        s += Cnm[m * (N + 1) + n] * uq;
    }
    atomic_max_pos(out, s_n[n] * s);
}

inline double mixed_eps_fft(int64_t L) {
    int lg = 0;
    while ((1LL << lg) < L) ++lg;
    return std::ldexp(1.0, -24) * (3.0 * lg + 8.0);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// CJT_PLAN_TRACE=1: print the wall time of each planning step (synchronising after each)
struct PlanTrace {
    bool on;
    cudaStream_t st;
    std::chrono::steady_clock::time_point t;
    explicit PlanTrace(cudaStream_t s) : on(getenv("CJT_PLAN_TRACE") != nullptr), st(s), t(std::chrono::steady_clock::now()) {}
    void mark(const char *what) {
        if (!on) return;
        cudaStreamSynchronize(st);
        auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[cjt plan] %-28s %8.3f ms\n", what, std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

template <typename T> int dalloc(cjt_plan_s *p, T **ptr, int64_t count) {
    *ptr = nullptr;
    if (count <= 0) return CJT_OK;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
        cjt_internal_set_cuda_error(e, "cudaMalloc");
        return CJT_ENOMEM;
    }
    p->allocs.push_back(v);
    p->device_bytes += (int64_t)count * (int64_t)sizeof(T);
    *ptr = (T *)v;
    return CJT_OK;
}

// A temporary device buffer from cjt_tmp_alloc, given back to the pool in stream order when
// it goes out of scope, so that every early error return releases it too.
template <typename T> struct TmpBuf {
    T *ptr = nullptr;
    cudaStream_t st;
    explicit TmpBuf(cudaStream_t s) : st(s) {}
    TmpBuf(const TmpBuf &) = delete;
    TmpBuf &operator=(const TmpBuf &) = delete;
    ~TmpBuf() { release(); }
    cudaError_t alloc(int64_t count) {
        release();
        return cjt_tmp_alloc((void **)&ptr, sizeof(T) * (size_t)count, st);
    }
    void release() {
        if (ptr) cudaFreeAsync(ptr, st);
        ptr = nullptr;
    }
};

#define TRY(x)                 \
    do {                       \
        int _rc = (x);         \
        if (_rc) return _rc;   \
    } while (0)

// ------------------------------------------------------------------------
// partition of one grid (Sec. 2.2) and the recurrence work that remains
// ------------------------------------------------------------------------
int build_grid(cjt_plan_s *p, GridWork &gw, int64_t Ng, bool inverse, const AsyExp &h, cudaStream_t st) {
    PlanTrace tr(st);
    const int M = p->M;
    gw.Ng = Ng;
    gw.Jcap = p->N + 1;
    const int64_t jtop = Ng + 1;
    gw.nblk = 0;
    gw.jk.clear(); gw.i1.clear(); gw.i2.clear();

    bool use_asy = p->opts.use_asy >= 0 && Ng >= 2;
    if (use_asy && p->corner) {
        // Hahn's series terminates at m = 0 and is exact for every n >= 0: one
        // block of all degrees on every interior row.
        gw.jk.push_back(0); gw.i1.push_back(1); gw.i2.push_back(Ng - 1);
    } else if (use_asy && p->n_M >= 1 && (double)Ng > (double)p->n_M) {
        const double lr = std::log((double)Ng / (double)p->n_M);
        double r = p->opts.ratio > 0 ? p->opts.ratio : std::min(1.0 / lr, 0.5);
        p->ratio = r;
        const int K = (int)std::ceil(lr / std::log(1.0 / r));
        std::vector<int64_t> js;
        std::vector<double> thr;
        double pw = 1.0;
        for (int k = 1; k <= K + 1 && k <= 60; ++k) {
            pw *= r;
            int64_t j = (int64_t)std::floor(pw * (double)Ng);
            if (j <= p->n_M || j < 2) break;
            js.push_back(j);
            thr.push_back(p->opts.eps / (2.0 * cjt_asy_C(h, j, M)));
        }
        if (!js.empty()) {
            TmpBuf<double> d_g(st), d_thr(st);
            TmpBuf<int> d_b2(st);
            CJT_CUDA_TRY(d_g.alloc(Ng + 1));
            CJT_CUDA_TRY(d_thr.alloc((int64_t)thr.size()));
            CJT_CUDA_TRY(d_b2.alloc(2 * (int64_t)thr.size()));
            k_envelope<<<blocks_for(Ng + 1, 256), 256, 0, st>>>(Ng, M, h, d_g.ptr);
            CJT_CUDA_TRY(cudaMemcpyAsync(d_thr.ptr, thr.data(), sizeof(double) * thr.size(), cudaMemcpyHostToDevice, st));
            k_box_init<<<1, 64, 0, st>>>((int)thr.size(), d_b2.ptr);
            unsigned nb = std::min<unsigned>(blocks_for(Ng, 256), 152 * 8);
            k_boxes<<<nb, 256, 0, st>>>(Ng, d_g.ptr, (int)thr.size(), d_thr.ptr, d_b2.ptr);
            CJT_CUDA_TRY(cudaGetLastError());
            std::vector<int> hb(2 * thr.size());
            CJT_CUDA_TRY(cudaMemcpyAsync(hb.data(), d_b2.ptr, sizeof(int) * hb.size(), cudaMemcpyDeviceToHost, st));
            CJT_CUDA_TRY(cudaStreamSynchronize(st));
            for (size_t k = 0; k < js.size(); ++k) {
                int lo = hb[2 * k], hi = hb[2 * k + 1];
                if (hi < lo) break;   // empty box: this and all deeper blocks dropped
                gw.jk.push_back(js[k]); gw.i1.push_back(lo); gw.i2.push_back(hi);
            }
        }
    }
    // blocks whose degrees all exceed N contribute nothing (the inverse grid, and a forward
    // grid larger than N, have more rows than degrees)
    {
        std::vector<int64_t> jk, i1, i2;
        for (size_t k = 0; k < gw.jk.size(); ++k)
            if (gw.jk[k] < gw.Jcap) { jk.push_back(gw.jk[k]); i1.push_back(gw.i1[k]); i2.push_back(gw.i2[k]); }
        gw.jk.swap(jk); gw.i1.swap(i1); gw.i2.swap(i2);
    }
    // parity fold (alpha = beta, stored recurrence values): the boxes are made symmetric
    // about the middle row by intersecting each with its mirror image (a subset of the box,
    // so the remainder bound still holds on it); an empty box drops it and the deeper ones
    gw.fold = p->alpha == p->beta && p->opts.rec_store != 0;
    if (gw.fold) {
        size_t k = 0;
        for (; k < gw.jk.size(); ++k) {
            const int64_t lo = std::max(gw.i1[k], Ng - gw.i2[k]), hi = Ng - lo;
            if (hi < lo) break;
            gw.i1[k] = lo;
            gw.i2[k] = hi;
        }
        gw.jk.resize(k); gw.i1.resize(k); gw.i2.resize(k);
    }
    gw.nblk = (int)gw.jk.size();
    tr.mark(inverse ? "inv: partition" : "fwd: partition");

    // deepest-box index per row and the box list on the device
    TRY(dalloc(p, &gw.d_rowk, Ng + 1));
    if (gw.nblk > 0) {
        std::vector<int> box3(3 * gw.nblk);
        for (int k = 0; k < gw.nblk; ++k) {
            box3[3 * k] = (int)gw.jk[k]; box3[3 * k + 1] = (int)gw.i1[k]; box3[3 * k + 2] = (int)gw.i2[k];
        }
        TRY(dalloc(p, &gw.d_box, 3 * gw.nblk));
        CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_box, box3.data(), sizeof(int) * box3.size(), cudaMemcpyHostToDevice, st));
        TRY(dalloc(p, &gw.d_u, (int64_t)M * (Ng + 1)));
        TRY(dalloc(p, &gw.d_v, (int64_t)M * (Ng + 1)));
        k_hahn_uv<<<blocks_for(Ng + 1, 128), 128, 0, st>>>(Ng, M, h, gw.d_u, gw.d_v);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    if (gw.nblk > 0) {
        // Item scales.  Forward: the transform input C_{n,m} c_n on degrees n >= j_k is
        // at most C_{j_k,m} |c| (C_{n,m} decreases in n, Lemma of Sec. 2.2).  Inverse:
        // the input (u_m + i v_m) g on rows [i1, i2] is bounded by the envelope g_m
        // (Sec. 2.2), which is unimodal, so its maximum over the box is at an end row.
        std::vector<double> sc(2 * (size_t)gw.nblk * M);
        for (int k = 0; k < gw.nblk; ++k) {
            for (int m = 0; m < M; ++m) {
                double mag;
                if (!inverse) {
                    mag = cjt_asy_C(h, gw.jk[k], m);
                } else {
                    mag = std::max(cjt_asy_env(h, m, gw.i1[k], Ng), cjt_asy_env(h, m, gw.i2[k], Ng));
                }
                int e = 0;
                if (mag > 0 && std::isfinite(mag)) std::frexp(mag, &e);
                sc[2 * ((size_t)k * M + m)] = std::ldexp(1.0, -e);
                sc[2 * ((size_t)k * M + m) + 1] = std::ldexp(1.0, e);
            }
        }
        TRY(dalloc(p, &gw.d_scale, (int64_t)sc.size()));
        CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_scale, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, st));
        const int nq = gw.nblk * M;
        const bool df = p->opts.precision == CJT_DFLOAT;
        if (!inverse) {
            dim3 g(blocks_for(p->N + 1, 256), nq);
            if (df) {
                TRY(dalloc(p, (double **)&gw.d_Cs, (int64_t)nq * (p->N + 1)));   // dfs: 8 bytes
                k_scaled_C<dfs><<<g, 256, 0, st>>>(p->N, M, nq, gw.d_box, p->d_Cnm, gw.d_scale, (dfs *)gw.d_Cs);
            }   // FP64 and mixed forms: the packs scale C_{n,m} as they read it
        } else {
            dim3 g(blocks_for(Ng + 1, 256), nq);
            if (df) {
                TRY(dalloc(p, (double **)&gw.d_Us, (int64_t)nq * (Ng + 1)));
                TRY(dalloc(p, (double **)&gw.d_Vs, (int64_t)nq * (Ng + 1)));
                k_scaled_uv<dfs><<<g, 256, 0, st>>>(Ng, M, nq, gw.d_box, gw.d_u, gw.d_v, gw.d_scale,
                                                    (dfs *)gw.d_Us, (dfs *)gw.d_Vs);
            }   // FP64 and mixed forms: the packs scale u_m, v_m as they read them
        }
        CJT_CUDA_TRY(cudaGetLastError());
        CJT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    k_rowk<<<blocks_for(Ng + 1, 256), 256, 0, st>>>(Ng, gw.nblk, gw.d_box, gw.d_rowk);
    CJT_CUDA_TRY(cudaGetLastError());
    if (!inverse && gw.nblk > 0 && p->opts.precision == CJT_DFLOAT) {
        // the double-float combine reads u, v already multiplied by the unscaling of the row's item
        dim3 g(blocks_for(Ng + 1, 256), M);
        k_fwd_uv_to_df<<<g, 256, 0, st>>>(Ng, M, gw.d_rowk, gw.d_scale, gw.d_u, gw.d_v);
        CJT_CUDA_TRY(cudaGetLastError());
        gw.uv_df = true;
    }

    tr.mark(inverse ? "inv: u,v tables, scales" : "fwd: u,v tables, scales");
    // ---- recurrence work: J(i) per row, chunks of <= 32 rows, degree segments
    const int S = p->seg_len;
    auto J_of = [&](int64_t i) -> int64_t {
        int64_t J = jtop;
        for (int k = 0; k < gw.nblk; ++k)
            if (i >= gw.i1[k] && i <= gw.i2[k]) J = gw.jk[k];
        return std::min(J, gw.Jcap);
    };
    auto mode_of = [&](int64_t i) -> int {
        if (4 * i <= Ng) return REC_REINSCH_P1;
        if (4 * i >= 3 * Ng) return REC_REINSCH_M1;
        return REC_PLAIN;
    };
    struct Chunk { int64_t row0; int nrows; int64_t J; int mode; int mirror; };
    std::vector<Chunk> chunks;
    // with the parity fold, chunks of the rows 2i < Ng stand also for their mirror rows
    // Ng - i (same J by the symmetric boxes); the middle row (Ng even) is a chunk of its own
    const int64_t ilast = gw.fold ? (Ng - 1) / 2 : Ng;
    {
        // J(i) and the mode are constant between the rows where a box begins or ends and the
        // two mode breakpoints: runs of equal (J, mode) are cut into chunks of 32 rows from
        // their first row (the rows one by one would give the same chunks)
        std::vector<int64_t> cut = {0, ilast + 1, (Ng + 4) / 4, (3 * Ng + 3) / 4};
        for (int k = 0; k < gw.nblk; ++k) {
            cut.push_back(gw.i1[k]);
            cut.push_back(gw.i2[k] + 1);
        }
        std::sort(cut.begin(), cut.end());
        cut.erase(std::unique(cut.begin(), cut.end()), cut.end());
        int64_t run0 = 0;
        for (size_t t = 0; t + 1 < cut.size() && cut[t] <= ilast; ++t) {
            const int64_t b0 = cut[t], b1 = std::min(cut[t + 1], ilast + 1);
            if (b1 <= ilast && J_of(b1) == J_of(b0) && mode_of(b1) == mode_of(b0)) continue;   // the run goes on
            const int64_t J = J_of(run0);
            const int md = mode_of(run0);
            for (int64_t i = run0; i < b1; i += 32)
                chunks.push_back(Chunk{i, (int)std::min<int64_t>(32, b1 - i), J, md, gw.fold ? 1 : 0});
            run0 = b1;
        }
    }
    if (gw.fold && Ng % 2 == 0) chunks.push_back(Chunk{Ng / 2, 1, J_of(Ng / 2), mode_of(Ng / 2), 0});
    gw.nchunks = (int64_t)chunks.size();
    std::vector<RecItem> items;
    // the forward combine's per-row segment counts and partial offsets (not used inverse)
    std::vector<int> row_nseg(inverse ? 0 : Ng + 1);
    std::vector<int64_t> row_base(inverse ? 0 : Ng + 1);
    std::vector<int> srow;
    int64_t out_f = 0, out_i = 0, nstate = 0, steps = 0, eoff = 0;
    for (size_t c = 0; c < chunks.size(); ++c) {
        const Chunk &ch = chunks[c];
        // rows whose recurrence is short enough run as one item (no segment states)
        const int64_t Sc = (p->opts.seg_whole > 0 && ch.J <= p->opts.seg_whole) ? std::max<int64_t>(ch.J, 1) : S;
        int nseg = (int)((ch.J + Sc - 1) / Sc);
        for (int r = 0; r < ch.nrows && !inverse; ++r) {
            row_nseg[ch.row0 + r] = nseg;
            row_base[ch.row0 + r] = out_f + r;
            if (ch.mirror) {   // the mirrored rows' partials follow the chunk's own
                row_nseg[Ng - ch.row0 - r] = nseg;
                row_base[Ng - ch.row0 - r] = out_f + (int64_t)nseg * 32 + r;
            }
        }
        steps += ch.J * ch.nrows;
        int state_base = (int)nstate;
        for (int s = 0; s < nseg; ++s) {
            RecItem it;
            it.row0 = (int)ch.row0;
            it.nrows = ch.nrows;
            it.a = (int)(s * Sc);
            it.b = (int)std::min<int64_t>((int64_t)(s + 1) * Sc, ch.J);
            it.mode = ch.mode;
            it.state = s == 0 ? -1 : state_base + s - 1;
            it.mirror = ch.mirror;
            it.pad_ = 0;
            it.out2 = -1;
            it.eoff = eoff;
            eoff += 32 * (int64_t)(it.b - it.a);
            if (!inverse) {
                it.out = out_f + (int64_t)s * 32;
                if (ch.mirror) it.out2 = it.out + (int64_t)nseg * 32;
            } else {
                it.out = out_i;
                out_i += it.b - it.a;
            }
            items.push_back(it);
        }
        if (nseg > 1) {
            for (int r = 0; r < ch.nrows; ++r) {
                int row = (int)(ch.row0 + r);
                int v[6] = {row, (int)ch.J, ch.mode, state_base, r, nseg};
                srow.insert(srow.end(), v, v + 6);
            }
            nstate += nseg - 1;
        }
        out_f += (int64_t)nseg * 32 * (ch.mirror ? 2 : 1);
    }
    gw.rec_steps = steps;
    gw.nstate = nstate;
    gw.nsrow = (int64_t)srow.size() / 6;
    gw.npartials = inverse ? out_i : out_f;

    // inverse: contributions to each degree segment, in a fixed order
    if (inverse) {
        gw.nsegs = (gw.Jcap + S - 1) / S;
        // items grouped by degree segment of S, in item order within a segment (a counting
        // sort); an item of a whole row is listed in every segment it spans, with its
        // partials' base shifted to the segment's first degree
        std::vector<int64_t> ptr(gw.nsegs + 1, 0);
        for (const RecItem &it : items)
            for (int64_t s = it.a / S; s <= (int64_t)(it.b - 1) / S; ++s) ++ptr[s + 1];
        for (int64_t s = 0; s < gw.nsegs; ++s) ptr[s + 1] += ptr[s];
        std::vector<int64_t> sout(ptr[gw.nsegs]);
        std::vector<int> sb(ptr[gw.nsegs]);
        std::vector<int64_t> at(ptr.begin(), ptr.end() - 1);
        for (const RecItem &it : items) {
            for (int64_t s = it.a / S; s <= (int64_t)(it.b - 1) / S; ++s) {
                const int64_t q = at[s]++;
                sout[q] = it.out + (s * S - it.a);
                sb[q] = it.b;
            }
        }
        TRY(dalloc(p, &gw.d_seg_ptr, gw.nsegs + 1));
        TRY(dalloc(p, &gw.d_seg_out, (int64_t)sout.size()));
        TRY(dalloc(p, &gw.d_seg_b, (int64_t)sb.size()));
        CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_seg_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice, st));
        if (!sout.empty()) {
            CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_seg_out, sout.data(), sizeof(int64_t) * sout.size(), cudaMemcpyHostToDevice, st));
            CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_seg_b, sb.data(), sizeof(int) * sb.size(), cudaMemcpyHostToDevice, st));
        }
        CJT_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        TRY(dalloc(p, &gw.d_row_base, Ng + 1));
        TRY(dalloc(p, &gw.d_row_nseg, Ng + 1));
        CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_row_base, row_base.data(), sizeof(int64_t) * row_base.size(),
                                     cudaMemcpyHostToDevice, st));
        CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_row_nseg, row_nseg.data(), sizeof(int) * row_nseg.size(),
                                     cudaMemcpyHostToDevice, st));
        CJT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    tr.mark(inverse ? "inv: host work lists" : "fwd: host work lists");
    // longest items first: the block scheduler then balances the SMs (a stable counting sort
    // by length, 1 .. the longest)
    {
        int64_t lmax = S;
        for (const RecItem &it : items) lmax = std::max<int64_t>(lmax, it.b - it.a);
        std::vector<int64_t> cnt(lmax + 2, 0);
        for (const RecItem &it : items) ++cnt[lmax - (it.b - it.a) + 1];
        for (int64_t l = 0; l <= lmax; ++l) cnt[l + 1] += cnt[l];
        std::vector<RecItem> sorted(items.size());
        for (const RecItem &it : items) sorted[cnt[lmax - (it.b - it.a)]++] = it;
        items.swap(sorted);
    }
    gw.nitems = (int64_t)items.size();
    TRY(dalloc(p, &gw.d_items, gw.nitems));
    if (gw.nitems)
        CJT_CUDA_TRY(cudaMemcpyAsync(gw.d_items, items.data(), sizeof(RecItem) * items.size(), cudaMemcpyHostToDevice, st));
    TRY(dalloc(p, &gw.d_states, std::max<int64_t>(nstate * 64, 1)));
    CJT_CUDA_TRY(cudaMemsetAsync(gw.d_states, 0, sizeof(double) * std::max<int64_t>(nstate * 64, 1), st));
    tr.mark(inverse ? "inv: items sorted, uploaded" : "fwd: items sorted, uploaded");
    if (gw.nsrow > 0) {
        // every row with more than one segment: runs of len degrees, `per` to a segment
        int per = (S + 511) / 512;
        while (S % per) ++per;
        const int len = S / per;
        std::vector<int> longrow;
        std::vector<int64_t> loff;
        int64_t nmaps = 0;
        for (int64_t q = 0; q < gw.nsrow; ++q) {
            const int *v = srow.data() + 6 * q;
            const int w[5] = {v[0], v[2], v[3], v[4], v[5]};
            longrow.insert(longrow.end(), w, w + 5);
            loff.push_back(nmaps);
            nmaps += (int64_t)(v[5] - 1) * per;
        }
        const int64_t nlong = (int64_t)longrow.size() / 5;
        TmpBuf<int> d_l(st);
        TmpBuf<int64_t> d_off(st);
        TmpBuf<double> d_maps(st);
        CJT_CUDA_TRY(d_l.alloc((int64_t)longrow.size()));
        CJT_CUDA_TRY(d_off.alloc((int64_t)loff.size()));
        CJT_CUDA_TRY(d_maps.alloc(4 * nmaps));
        CJT_CUDA_TRY(cudaMemcpyAsync(d_l.ptr, longrow.data(), sizeof(int) * longrow.size(), cudaMemcpyHostToDevice, st));
        CJT_CUDA_TRY(cudaMemcpyAsync(d_off.ptr, loff.data(), sizeof(int64_t) * loff.size(), cudaMemcpyHostToDevice, st));
        k_rec_seg_maps<<<blocks_for(nmaps, 128), 128, 0, st>>>(nlong, nmaps, d_l.ptr, d_off.ptr, Ng, len, p->rt,
                                                               d_maps.ptr);
        k_rec_seg_carry<<<blocks_for(nlong, 64), 64, 0, st>>>(nlong, d_l.ptr, d_off.ptr, per, d_maps.ptr, gw.d_states);
        CJT_CUDA_TRY(cudaGetLastError());
        CJT_CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors above go out of scope
    }
    gw.nE = eoff;
    if (p->opts.rec_store && gw.nitems > 0) {
        TRY(dalloc(p, &gw.d_E, std::max<int64_t>(gw.nE, 1)));
        k_rec_fill<<<blocks_for(gw.nitems * 32, 128), 128, 0, st>>>(gw.d_items, gw.nitems, Ng, p->rt, gw.d_states,
                                                                   gw.d_E, inverse ? 1 : 0);
        CJT_CUDA_TRY(cudaGetLastError());
        if (p->opts.precision == CJT_DFLOAT) {
            k_to_df_inplace<<<blocks_for(gw.nE, 256), 256, 0, st>>>(gw.nE, gw.d_E);
            CJT_CUDA_TRY(cudaGetLastError());
            gw.E_df = true;
        }
    }
    CJT_CUDA_TRY(cudaStreamSynchronize(st));  // host vectors go out of scope
    tr.mark(inverse ? "inv: segment states" : "fwd: segment states");
    return CJT_OK;
}

}  // namespace

// A pool per device (created on first use) whose freed memory, up to 1 GiB, stays reserved
// for the next plan build instead of going back to the CUDA driver.
cudaError_t cjt_tmp_alloc(void **ptr, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(ptr, bytes, st);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&pools[dev], &props);
            if (e != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = 1ull << 30;   // freed memory kept for reuse (the pool is ours alone)
            cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

// ------------------------------------------------------------------------
// Twiddle tables shared by plans.  They depend only on (device, Ltab, Ltabq, transform
// precision), so plans of the same lengths take one copy: a plan built while a copy exists
// waits for its construction on its own stream (an event) and launches nothing.  Unused
// copies stay cached up to CJT_TWIDDLE_CACHE_MB (default 1024) and are freed least
// recently used first beyond that.
// ------------------------------------------------------------------------
namespace {
struct TwShared {
    int dev = 0, pa = 0;
    int64_t Ltab = 0, Ltabq = 0;
    void *tw64 = nullptr, *tw32 = nullptr, *twdf = nullptr;
    void *stw64 = nullptr, *stw32 = nullptr, *stwdf = nullptr, *twfma = nullptr;
    void *twq_64 = nullptr, *twq_32 = nullptr, *twqdf = nullptr;
    int lmax = 0;
    int64_t bytes = 0;
    int refs = 0;
    uint64_t last = 0;
    cudaEvent_t ready = nullptr;
    std::vector<void *> allocs;
};
std::mutex g_tw_mu;
std::vector<TwShared *> g_tw;
uint64_t g_tw_clock = 0;

// frees a copy's tables on the device that holds them (the caller's device is restored)
void tw_free(TwShared *e) {
    int cur = -1;
    const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != e->dev && cudaSetDevice(e->dev) == cudaSuccess;
    if (e->ready) {
        cudaEventSynchronize(e->ready);
        cudaEventDestroy(e->ready);
    }
    for (void *v : e->allocs) cudaFree(v);
    if (other) cudaSetDevice(cur);
    delete e;
}

template <typename T> int tw_alloc(TwShared *e, void **ptr, int64_t count) {
    *ptr = nullptr;
    if (count <= 0) return CJT_OK;
    void *v = nullptr;
    cudaError_t rc = cudaMalloc(&v, (size_t)count * sizeof(T));
    if (rc != cudaSuccess) {
        cjt_internal_set_cuda_error(rc, "cudaMalloc");
        return CJT_ENOMEM;
    }
    e->allocs.push_back(v);
    e->bytes += (int64_t)count * (int64_t)sizeof(T);
    *ptr = v;
    return CJT_OK;
}

int tw_build(TwShared *e, cudaStream_t st) {
    const int pa = e->pa;
    if (e->Ltabq > 0) {
        TRY(tw_alloc<double2>(e, &e->twq_64, e->Ltabq));
        if (pa == PREC_F32) TRY(tw_alloc<float2>(e, &e->twq_32, e->Ltabq));
        if (pa == PREC_DF) TRY(tw_alloc<double2>(e, &e->twqdf, e->Ltabq));   // dfc: 16 bytes
        k_twiddles<<<blocks_for(e->Ltabq, 256), 256, 0, st>>>(e->Ltabq, (double2 *)e->twq_64, (float2 *)e->twq_32,
                                                              (dfc *)e->twqdf);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    TRY(tw_alloc<double2>(e, &e->tw64, e->Ltab));
    if (pa == PREC_F32) TRY(tw_alloc<float2>(e, &e->tw32, e->Ltab));
    if (pa == PREC_DF) TRY(tw_alloc<double2>(e, &e->twdf, e->Ltab));   // dfc: 16 bytes
    k_twiddles<<<blocks_for(e->Ltab, 256), 256, 0, st>>>(e->Ltab, (double2 *)e->tw64, (float2 *)e->tw32,
                                                         (dfc *)e->twdf);
    CJT_CUDA_TRY(cudaGetLastError());
    int logLtab = 0;
    while ((1LL << logLtab) < e->Ltab) ++logLtab;
    // stage tables to block length 2^13: one-pass transforms of up to 8192 points
    // (cjt_fft_set_config)
    const int lmax = std::min(13, logLtab);
    e->lmax = lmax;
    if (lmax >= 2) {
        const int64_t n = stw_base(lmax + 1);
        TRY(tw_alloc<double2>(e, &e->stw64, n));
        if (pa == PREC_F32) TRY(tw_alloc<float2>(e, &e->stw32, n));
        if (pa == PREC_DF) TRY(tw_alloc<double2>(e, &e->stwdf, n));   // dfc: 16 bytes
        k_stage_twiddles<<<blocks_for(n, 256), 256, 0, st>>>(lmax, logLtab, (const double2 *)e->tw64,
                                                             (double2 *)e->stw64, (float2 *)e->stw32,
                                                             (dfc *)e->stwdf);
        CJT_CUDA_TRY(cudaGetLastError());
        // every plan has FP64 transforms (final DCT-I, inverse front end)
        const int64_t nf = twfma_base(lmax + 1);
        TRY(tw_alloc<TwFma>(e, &e->twfma, nf));
        k_fma_twiddles<<<blocks_for(nf, 256), 256, 0, st>>>(lmax, logLtab, (const double2 *)e->tw64,
                                                           (TwFma *)e->twfma);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    CJT_CUDA_TRY(cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming));
    CJT_CUDA_TRY(cudaEventRecord(e->ready, st));
    return CJT_OK;
}

int64_t tw_cache_cap() {
    const char *v = getenv("CJT_TWIDDLE_CACHE_MB");
    const long long mb = v ? atoll(v) : 1024;
    return (int64_t)std::max(0LL, mb) << 20;
}

// with g_tw_mu held: free unused copies, least recently used first, beyond the cap
void tw_trim_locked() {
    const int64_t cap = tw_cache_cap();
    for (;;) {
        int64_t unused = 0;
        TwShared *victim = nullptr;
        for (TwShared *e : g_tw) {
            if (e->refs > 0) continue;
            unused += e->bytes;
            if (!victim || e->last < victim->last) victim = e;
        }
        if (!victim || unused <= cap) return;
        g_tw.erase(std::find(g_tw.begin(), g_tw.end(), victim));
        tw_free(victim);
    }
}
}  // namespace

int cjt_build_twiddles(cjt_plan_s *p, int pa, cudaStream_t st) {
    int dev = 0;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tw_mu);
    TwShared *e = nullptr;
    for (TwShared *c : g_tw)
        if (c->dev == dev && c->pa == pa && c->Ltab == p->Ltab && c->Ltabq == p->Ltabq) e = c;
    if (e) {
        CJT_CUDA_TRY(cudaStreamWaitEvent(st, e->ready, 0));
    } else {
        e = new TwShared;
        e->dev = dev;
        e->pa = pa;
        e->Ltab = p->Ltab;
        e->Ltabq = p->Ltabq;
        const int rc = tw_build(e, st);
        if (rc) {
            cudaStreamSynchronize(st);
            tw_free(e);
            return rc;
        }
        g_tw.push_back(e);
    }
    ++e->refs;
    e->last = ++g_tw_clock;
    p->twc = e;
    p->d_tw64 = e->tw64;
    p->d_tw32 = e->tw32;
    p->d_twdf = e->twdf;
    p->d_stw64 = e->stw64;
    p->d_stw32 = e->stw32;
    p->d_stwdf = e->stwdf;
    p->d_twfma = e->twfma;
    p->d_twq_64 = e->twq_64;
    p->d_twq_32 = e->twq_32;
    p->d_twqdf = e->twqdf;
    p->stw_lmax = e->lmax;
    p->device_bytes += e->bytes;   // counted in every plan that uses them (an upper bound)
    return CJT_OK;
}

void cjt_release_twiddles(cjt_plan_s *p) {
    if (!p->twc) return;
    std::lock_guard<std::mutex> lk(g_tw_mu);
    TwShared *e = (TwShared *)p->twc;
    p->twc = nullptr;
    --e->refs;
    e->last = ++g_tw_clock;
    tw_trim_locked();
}

int cjt_plan_build(cjt_plan_s *p, cudaStream_t st) {
    PlanTrace tr(st);
    TRY(cjt_fft_prime());
    const int64_t N = p->N;
    const double a = p->alpha, b = p->beta;
    p->corner = (std::fabs(std::fabs(a) - 0.5) == 0.0) && (std::fabs(std::fabs(b) - 0.5) == 0.0);
    p->M = p->corner ? 1 : p->opts.M;
    const int M = p->M;

    // the expansion (Hahn's formula, or the ultraspherical one for alpha = beta, App. B.1)
    // and n_M from its remainder bound at pi/2 (Sec. 2.2)
    AsyExp h;
    TRY(cjt_asy_make(a, b, p->corner ? CJT_EXPANSION_HAHN : p->opts.expansion, &h));
    p->expansion_used = h.ultra ? CJT_EXPANSION_ULTRASPHERICAL : CJT_EXPANSION_HAHN;
    p->n_M = cjt_asy_nM(h, M, p->opts.eps);

    // 1c: recurrence tables for degrees 0..N+1
    p->Jcap = N + 1;
    const int64_t nt = N + 2;
    TRY(dalloc(p, &p->d_tabs, 11 * nt));
    double *q = p->d_tabs;
    p->rt.A = q; p->rt.B = q + nt; p->rt.C = q + 2 * nt;
    p->rt.Cr_p = q + 3 * nt; p->rt.rbinv_p = q + 4 * nt; p->rt.Ce_p = q + 5 * nt; p->rt.rf_p = q + 6 * nt;
    p->rt.Cr_m = q + 7 * nt; p->rt.rbinv_m = q + 8 * nt; p->rt.Ce_m = q + 9 * nt; p->rt.rf_m = q + 10 * nt;
    k_rec_tables<<<blocks_for(nt, 256), 256, 0, st>>>(nt - 1, a, b, p->rt);
    CJT_CUDA_TRY(cudaGetLastError());

    // coefficients C_{n,m} for m = 0..M (row M is the partition's remainder term)
    TRY(dalloc(p, &p->d_Cnm, (int64_t)(M + 1) * (N + 1)));
    {
        dim3 g(blocks_for(N + 1, 256), M + 1);
        k_hahn_C<<<g, 256, 0, st>>>(N, M + 1, h, p->d_Cnm);
        CJT_CUDA_TRY(cudaGetLastError());
    }

    tr.mark("tables: recurrence, C_nm");
    const bool fwd = p->opts.directions & CJT_FWD, inv = p->opts.directions & CJT_INV;
    // Lobatto grid: N, or the least power of two G >= N (the same map: degree-N polynomials
    // are interpolated exactly on G+1 points, and the (2G+1)-point Clenshaw--Curtis rule is
    // exact wherever the (2N+1)-point rule is); power-of-two transforms then need no
    // Bluestein form
    {
        const bool pow2 = (N & (N - 1)) == 0;
        int64_t G = N;
        int64_t G2 = 1;
        while (G2 < N) G2 <<= 1;
        if (p->opts.grid == 1) {
            G = G2;
        } else if (p->opts.grid == 0 && !pow2 && !cjt_is_3pow2(N) && !cjt_is_5pow2(N)) {
            // the least G >= N of the forms 2^a, 3 2^a and 5 2^a: transforms of lengths 2G
            // and 4G then take one radix-3 or radix-5 step at most, and the grid is at most
            // 4/3 N
            int64_t G3 = 3, G5 = 5;
            while (G3 < N) G3 <<= 1;
            while (G5 < N) G5 <<= 1;
            G = std::min(G2, std::min(G3, G5));
        }
        p->Gf = p->Gi = G;
    }
    if (fwd) TRY(build_grid(p, p->fw, p->Gf, false, h, st));
    if (inv) TRY(build_grid(p, p->iv, 2 * p->Gi, true, h, st));

    // transforms: forward ASY/DCT length 2N, inverse 4N; Bluestein when N is not a power of two
    p->prec_asy = p->opts.precision == CJT_MIXED ? PREC_F32 : p->opts.precision == CJT_DFLOAT ? PREC_DF : PREC_F64;
    const int pa = p->prec_asy;
    p->Lf = fwd ? 2 * p->Gf : 0;
    p->Li = inv ? 4 * p->Gi : 0;
    p->npair_f = (p->fw.nblk * M + 1) / 2;
    p->npair_i = (p->iv.nblk * M + 1) / 2;
    auto mk = [](Dft &d, int64_t L, int64_t S, int64_t K, int prec) {
        d.L = L; d.S = S; d.K = K; d.prec = prec; d.P = cjt_dft_padded(L, S, K);
    };
    std::vector<std::pair<Dft *, int64_t>> used;   // transform and its batch
    if (fwd) {
        const int64_t G = p->Gf;
        mk(p->dft_f, 2 * G, N + 1, 2 * G, pa);   // both Z(i) and Z(L-i) are read by the pair separation
        mk(p->dft_dct, 2 * G, 2 * G, N + 1, PREC_F64);
        if (p->npair_f) used.push_back({&p->dft_f, p->npair_f});
        used.push_back({&p->dft_dct, 1});
    }
    if (inv) {
        const int64_t G = p->Gi;
        mk(p->dft_front, 4 * G, N + 1, 2 * G + 1, PREC_F64);
        mk(p->dft_i, 4 * G, 4 * G, N + 1, pa);
        mk(p->dft_cc, 4 * G, 4 * G, 2 * G + 1, PREC_F64);
        used.push_back({&p->dft_front, 1});
        if (p->npair_i) used.push_back({&p->dft_i, p->npair_i});
        used.push_back({&p->dft_cc, 1});
    }
    // twiddle tables: powers of two up to the longest power-of-two (sub-)transform, and for
    // lengths q 2^b (q = 3 or 5, one q per plan) the radix-q table of the longest such length
    // (a multiple of the others)
    p->Ltab = 2;
    p->Ltabq = 0;
    for (auto &u : used) {
        const Dft &d = *u.first;
        const int q = d.P ? 1 : cjt_odd_radix(d.L);
        if (d.P) {
            p->Ltab = std::max(p->Ltab, d.P);
        } else if (q > 1) {
            p->Ltab = std::max(p->Ltab, d.L / q);
            p->Ltabq = std::max(p->Ltabq, d.L);
        } else {
            p->Ltab = std::max(p->Ltab, d.L);
        }
    }
    for (auto &u : used)
        if (!u.first->P && cjt_odd_radix(u.first->L) > 1 && p->Ltabq % u.first->L != 0) return CJT_EUNSUPPORTED;
    TRY(cjt_build_twiddles(p, pa, st));
    int64_t work = 0, scratch = 0;
    for (auto &u : used) {
        Dft &d = *u.first;
        if (d.P) {
            const int64_t nw = std::max(d.S, d.K);
            if (d.prec == PREC_F32) {
                TRY(dalloc(p, (float2 **)&d.chirp, nw));
                TRY(dalloc(p, (float2 **)&d.bhat, d.P));
            } else {   // double2 or dfc: 16 bytes
                TRY(dalloc(p, (double2 **)&d.chirp, nw));
                TRY(dalloc(p, (double2 **)&d.bhat, d.P));
            }
            TRY(cjt_dft_setup(d, p->d_tw64, p->Ltab, st));
        }
        work = std::max(work, cjt_dft_work_bytes(d, u.second));
        scratch = std::max(scratch, cjt_dft_scratch_bytes(d, u.second));
    }
    tr.mark("transforms: twiddles, chirps");
    // execution workspace layout
    {
        const int64_t csz = prec_cbytes(pa);
        const int64_t Ld = std::max<int64_t>(std::max(p->Lf, p->Li), 2);
        p->ws_size[WS_FFT_F] = csz * p->npair_f * p->Lf;
        p->ws_size[WS_FFT_I] = csz * p->npair_i * p->Li;
        p->ws_size[WS_SCRATCH] = scratch;
        p->ws_size[WS_WORK] = work;
        p->ws_size[WS_DCT] = (int64_t)sizeof(double2) * Ld;
        const int64_t G = std::max(p->Gf, p->Gi);
        p->ws_size[WS_Y] = (int64_t)sizeof(double) * (2 * G + 2);
        p->ws_size[WS_G] = inv ? (int64_t)sizeof(double) * (2 * p->Gi + 1) : 0;
        p->ws_size[WS_PART_F] = (int64_t)sizeof(double) * (fwd ? std::max<int64_t>(p->fw.npartials, 1) : 0);
        p->ws_size[WS_PART_I] = (int64_t)sizeof(double) * (inv ? std::max<int64_t>(p->iv.npartials, 1) : 0);
        p->ws_size[WS_XDF] = pa == PREC_DF ? (int64_t)sizeof(dfs) * (inv ? 2 * p->Gi + 1 : N + 1) : 0;
        p->ws_size[WS_EXPS] = pa == PREC_DF ? (int64_t)sizeof(int) * (CJT_EXP_BLOCKS + 1) : 0;
        p->ws_size[WS_CONV] = (p->shift_a || p->shift_b)
                                  ? (int64_t)sizeof(double) * (2 * (N + 1) + 3 * cjt_conv_chunks(N)) : 0;
        int64_t off = 0;
        for (int k = 0; k < WS_COUNT; ++k) {
            p->ws_off[k] = off;
            off += (p->ws_size[k] + 255) / 256 * 256;
        }
        p->ws_bytes = off;
    }
    p->shared_ws = p->opts.shared_workspace != 0;
    TmpBuf<unsigned char> tmp_ws(st);
    if (!p->shared_ws) {
        unsigned char *arena = nullptr;
        TRY(dalloc(p, &arena, p->ws_bytes));
        p->ws = cjt_carve(p, arena);
    }
    TRY(dalloc(p, &p->d_in, N + 1));
    TRY(dalloc(p, &p->d_out, N + 1));

    if (inv && N >= 1) {
        const int64_t Ng = 2 * p->Gi;
        Workspace ws = p->ws;
        if (p->shared_ws) {   // temporary buffers for the weights' transform (DCT, work, scratch)
            const int64_t a0 = (p->ws_size[WS_DCT] + 255) / 256 * 256, a1 = (p->ws_size[WS_WORK] + 255) / 256 * 256;
            const int64_t a2 = (p->ws_size[WS_SCRATCH] + 255) / 256 * 256;
            CJT_CUDA_TRY(tmp_ws.alloc(a0 + a1 + a2));
            unsigned char *b = tmp_ws.ptr;
            ws = Workspace{};
            ws.dct = (double *)b;
            ws.work = p->ws_size[WS_WORK] ? b + a0 : nullptr;
            ws.scratch = p->ws_size[WS_SCRATCH] ? b + a0 + a1 : nullptr;
        }
        TRY(dalloc(p, &p->d_w, Ng + 1));
        TRY(dalloc(p, &p->d_s, N + 1));
        const double mu0 = std::exp2(a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) / std::tgamma(a + b + 2.0);
        // modified moments mu_0..mu_Ng (Sec. 3.1, mu_1 with the sign of the weight's mean)
        const double mu1 = (b - a) / (a + b + 2.0) * mu0;
        const int64_t nchunk = std::max<int64_t>(1, (Ng - 1 + kMomChunk - 1) / kMomChunk);
        TmpBuf<Mat2> T(st);
        TmpBuf<double2> start(st);
        CJT_CUDA_TRY(T.alloc(nchunk));
        CJT_CUDA_TRY(start.alloc(nchunk));
        k_mom_transfer<<<blocks_for(nchunk, 128), 128, 0, st>>>(Ng, a, b, nchunk, T.ptr);
        k_mom_carry<<<1, kMomScanThreads, 0, st>>>(nchunk, mu0, mu1, T.ptr, start.ptr);
        k_mom_fill<<<blocks_for(nchunk, 128), 128, 0, st>>>(Ng, a, b, nchunk, start.ptr, (double2 *)ws.dct);
        CJT_CUDA_TRY(cudaGetLastError());
        T.release();
        start.release();
        TRY(cjt_dft_exec(p->dft_cc, ws.dct, ws.work, ws.scratch, 1, p->twiddles(PREC_F64), st));
        k_cc_weights<<<blocks_for(Ng + 1, 256), 256, 0, st>>>(Ng, (const double2 *)ws.dct, p->d_w);
        k_inv_norm<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, a, b, p->d_s);
        CJT_CUDA_TRY(cudaGetLastError());
    }
    tmp_ws.release();
    tr.mark("buffers, inverse weights");
    if (pa == PREC_F32 && (p->fw.nblk > 0 || p->iv.nblk > 0)) {
        // bound on the FP32 transforms' error (see k_err_fwd): two maxima read back once
        TmpBuf<double> acc(st), U(st);
        const int nqi = p->iv.nblk * M;
        CJT_CUDA_TRY(acc.alloc(2));
        CJT_CUDA_TRY(cudaMemsetAsync(acc.ptr, 0, 2 * sizeof(double), st));
        if (fwd && p->fw.nblk > 0)
            k_err_fwd<<<blocks_for(p->Gf + 1, 256), 256, 0, st>>>(N, p->Gf, M, p->fw.nblk * M, p->fw.d_rowk,
                                                                   p->fw.d_box, p->d_Cnm, p->fw.d_scale, p->fw.d_u,
                                                                   p->fw.d_v, acc.ptr);
        if (inv && nqi > 0) {
            CJT_CUDA_TRY(U.alloc(nqi));
            k_err_inv_U<<<nqi, 256, 0, st>>>(2 * p->Gi, M, p->iv.d_box, p->d_w, p->iv.d_u, p->iv.d_v, U.ptr);
            k_err_inv<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, M, p->iv.nblk, nqi, p->iv.d_box, p->d_Cnm,
                                                               p->iv.d_scale, U.ptr, p->d_s, acc.ptr + 1);
        }
        CJT_CUDA_TRY(cudaGetLastError());
        double h[2] = {0.0, 0.0};
        CJT_CUDA_TRY(cudaMemcpyAsync(h, acc.ptr, sizeof(h), cudaMemcpyDeviceToHost, st));
        CJT_CUDA_TRY(cudaStreamSynchronize(st));
        p->err_mixed_fwd = fwd ? 2.0 * mixed_eps_fft(p->Lf) * h[0] : 0.0;
        p->err_mixed_inv = inv ? mixed_eps_fft(p->Li) * h[1] : 0.0;
    }
    CJT_CUDA_TRY(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming));
    CJT_CUDA_TRY(cudaStreamSynchronize(st));
    return CJT_OK;
}

Workspace cjt_carve(const cjt_plan_s *p, void *base) {
    Workspace w;
    if (!base) return w;
    unsigned char *b = (unsigned char *)base;
    auto at = [&](int k) -> void * { return p->ws_size[k] ? (void *)(b + p->ws_off[k]) : nullptr; };
    w.fft_f = at(WS_FFT_F);
    w.fft_i = at(WS_FFT_I);
    w.scratch = at(WS_SCRATCH);
    w.work = at(WS_WORK);
    w.dct = (double *)at(WS_DCT);
    w.y = (double *)at(WS_Y);
    w.g = (double *)at(WS_G);
    w.part_f = (double *)at(WS_PART_F);
    w.part_i = (double *)at(WS_PART_I);
    w.xdf = at(WS_XDF);
    w.exps = (int *)at(WS_EXPS);
    w.conv = (double *)at(WS_CONV);
    return w;
}
