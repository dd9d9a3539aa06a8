// Internal declarations of the Chebyshev--Jacobi transform library (sm_103a).
//
// Layout of a plan in device memory (all FP64 unless noted):
//   recurrence tables, index n = 0..Jcap (Sec. 1.2 and Sec. 4.2):
//     A, B, C                 plain three-term recurrence
//     for x0 = +1 and x0 = -1 (Reinsch-modified recurrences, Sec. 4.2):
//       Cr[n] = C_n r^b_n     rbinv[n] = 1/r^b_n  (backward / Clenshaw--Smith form)
//       Ce[n] = C_n/r^f_{n-1} rf[n] = r^f_n      (forward form, e_n = d_n r^f_{n-1})
//   Hahn coefficients  Cnm[m*(N+1) + n], m = 0..M      (Eq. "Cnmab")
//   diagonals          u[m*(Ng+1) + i], v[...], m < M   (Eq. "Jacasyuv"), per grid
//   partition          boxes (j_k, i_k^1, i_k^2)        (Sec. 2.2), per grid
//   recurrence work    warp items over (32 rows) x (degree segment), with the
//                      forward-recurrence state at every segment start
//   transform buffers  complex FP64, FP32 or double-float (cjt_df.cuh), twiddle
//                      table omega_{Ltab}^k in each precision the plan uses
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include <string>
#include <vector>

#include "../../include/cjt.h"

#define CJT_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            cjt_internal_set_cuda_error(_e, #expr);          \
            return CJT_ECUDA;                                \
        }                                                    \
    } while (0)

void cjt_internal_set_cuda_error(cudaError_t e, const char *what);
struct cjt_plan_s;
int cjt_internal_begin_use(cjt_plan_s *p, cudaStream_t st);
int cjt_internal_end_use(cjt_plan_s *p, cudaStream_t st);
// CJT_OK when the plan's device is the current one, CJT_EINVAL when another device is
// current (its tables would be read from the wrong device), CJT_ECUDA without a device.
int cjt_internal_check_device(const cjt_plan_s *p);
// Side streams and events of one execution's two concurrent chains (the asymptotic blocks
// and the recurrence, option overlap).  Each execution takes a context of its own from a
// per-device pool for the time it enqueues its work and gives it back at once (cudaEvent
// records and waits are resolved when they are enqueued), so executions on different host
// threads never share a fork or join event.  The pool hands out its contexts in turn, so
// consecutive executions on different streams put their asymptotic chains on different side
// streams, and it skips a context whose stream still belongs to another open stream capture.
struct OvCtx {
    int dev = 0, mode = 0;
    cudaStream_t side = nullptr, side_rec = nullptr;   // side_rec: CJT_OVERLAP_REC_FIRST only
    cudaEvent_t fork = nullptr, join = nullptr, join_rec = nullptr;
};
int cjt_internal_ovctx_acquire(int overlap, cudaStream_t origin, OvCtx **out);
void cjt_internal_ovctx_release(OvCtx *c);

// ---------------------------------------------------------------------------
// recurrence work items
// ---------------------------------------------------------------------------
enum { REC_PLAIN = 0, REC_REINSCH_P1 = 1, REC_REINSCH_M1 = 2 };

struct RecItem {
    int row0;    // first grid row of the 32-row chunk
    int nrows;   // rows in the chunk (1..32)
    int a, b;    // degree segment [a, b)
    int mode;    // REC_PLAIN / REC_REINSCH_P1 / REC_REINSCH_M1
    int state;   // state block index (32 lanes x 2 doubles), -1 when a == 0
    int mirror;  // 1: parity fold (alpha = beta): lane r also stands for row Ng - row0 - r
    int pad_;
    int64_t out; // forward: partial index base (32 values); inverse: base of b-a values
    int64_t eoff;// stored recurrence values of this item (rec_store): 32 x (b-a) doubles
    int64_t out2;// forward, mirror: partial index base of the mirrored rows
};

// Recurrence tables for one direction (degrees 0..Jcap).
struct RecTables {
    double *A, *B, *C;
    double *Cr_p, *rbinv_p, *Ce_p, *rf_p;   // x0 = +1
    double *Cr_m, *rbinv_m, *Ce_m, *rf_m;   // x0 = -1
};

// One degree's entries of the recurrence tables: the three-term coefficients (Sec. 1.2)
// and the Reinsch quantities at x0 = +-1 (Sec. 4.2).  Used by the plan kernel that fills
// RecTables and by the host entry point cjt_rec_coefficients.
struct RecRow {
    double A, B, C;
    double rf_p, rf_m;         // forward ratios r^f_n(+-1) = pi_{n+1}(+-1)/pi_n(+-1)
    double rb_p, rb_m;         // backward ratios r^b_n(+-1) (Lemma of Sec. 4.2); n >= 1
    double Ce_p, Ce_m;         // e-form coefficient C_n / r^f_{n-1}(+-1)
    double Cr_p, Cr_m;         // C_n r^b_n(+-1)
    double rbinv_p, rbinv_m;   // 1 / r^b_n(+-1)
};
__host__ __device__ __forceinline__ RecRow cjt_rec_row(int64_t n, double a, double b) {
    RecRow r;
    const double nn = (double)n, ab = a + b;
    double A, B, C;
    if (n == 0) {
        // from P_1 = (a-b)/2 + (a+b+2)/2 x (avoids 0/0 when a+b = 0 or -1)
        A = 0.5 * (ab + 2.0);
        B = 0.5 * (a - b);
        C = 0.0;
    } else {
        const double t0 = 2.0 * nn + ab, t1 = t0 + 1.0, t2 = t0 + 2.0, s1 = nn + ab + 1.0;
        A = t1 * t2 / (2.0 * (nn + 1.0) * s1);
        B = (a - b) * ab * t1 / (2.0 * (nn + 1.0) * s1 * t0);
        C = (nn + a) * (nn + b) * t2 / ((nn + 1.0) * s1 * t0);
    }
    r.A = A;
    r.B = B;
    r.C = C;
    r.rf_p = (nn + a + 1.0) / (nn + 1.0);
    r.rf_m = -(nn + b + 1.0) / (nn + 1.0);
    if (n == 0) {
        r.Ce_p = 0.0;
        r.Ce_m = 0.0;
    } else {
        r.Ce_p = C * nn / (nn + a);
        r.Ce_m = -C * nn / (nn + b);
    }
    // r^b_0 is infinite: its slots hold 0, which the kernels never read at n = 0
    if (n == 0) {
        r.rb_p = 0.0; r.Cr_p = 0.0; r.rbinv_p = 0.0;
        r.rb_m = 0.0; r.Cr_m = 0.0; r.rbinv_m = 0.0;
    } else {
        const double common = (nn + 1.0) / nn * (ab + nn + 1.0) * (ab + 2.0 * nn) / (ab + 2.0 * nn + 2.0);
        const double rbp = common / (nn + b);
        const double rbm = -common / (nn + a);
        r.rb_p = rbp; r.Cr_p = C * rbp; r.rbinv_p = 1.0 / rbp;
        r.rb_m = rbm; r.Cr_m = C * rbm; r.rbinv_m = 1.0 / rbm;
    }
    return r;
}

// Partition and recurrence work of one grid (N points for forward, 2N for inverse).
struct GridWork {
    int64_t Ng = 0;        // grid: points x_i = cos(pi i / Ng), i = 0..Ng
    int64_t Jcap = 0;      // degrees handled: 0..Jcap-1 (= N+1)
    int nblk = 0;          // asymptotic blocks kept
    std::vector<int64_t> jk, i1, i2;  // block k: degrees [jk[k], jtop(k)), rows [i1[k], i2[k]]
    int64_t rec_steps = 0;
    // device
    int *d_rowk = nullptr;        // per row: deepest box index k (0-based) or -1
    int64_t *d_row_base = nullptr;// forward: partial index of segment 0 of each row
    int *d_row_nseg = nullptr;    // forward: degree segments of each row
    RecItem *d_items = nullptr;
    int64_t nitems = 0;
    double *d_states = nullptr;   // [nstate][32][2]
    int64_t nstate = 0;
    int64_t npartials = 0;        // recurrence partial sums (in the workspace)
    // state computation rows
    int64_t nsrow = 0;
    // inverse combine: CSR over degree segments
    int64_t nsegs = 0;
    int64_t *d_seg_ptr = nullptr;
    int64_t *d_seg_out = nullptr; // partial base of each contributing item
    int *d_seg_b = nullptr;       // item end degree b
    int64_t nchunks = 0;
    // stored recurrence values (rec_store): forward [item][k][lane], inverse [item][lane][k];
    // doubles, or double-floats (dfs, same 8 bytes) when E_df
    double *d_E = nullptr;
    bool E_df = false;
    bool uv_df = false;           // forward grid: u, v held as double-floats, premultiplied (CJT_DFLOAT)
    // parity fold (alpha = beta with rec_store): P_n(-x) = (-1)^n P_n(x), so the recurrence
    // items cover the rows i <= Ng/2 and each also yields row Ng - i; the boxes are
    // symmetric about the middle row
    bool fold = false;
    int64_t nE = 0;
    // diagonals u_m, v_m on this grid
    double *d_u = nullptr, *d_v = nullptr;
    int *d_box = nullptr;         // [nblk][3] = j, i1, i2
    // per asymptotic item q = k*M + m: exact power-of-two scale applied before the
    // transform (d_scale[2q]) and removed after it (d_scale[2q+1]), so that the two
    // items sharing one complex transform have comparable magnitudes
    double *d_scale = nullptr;
    // transform inputs pre-scaled per item, in the transform precision:
    //   forward  Cs[q][n] = s_q C_{n,m} for n >= j_k (0 below)            (q x (N+1))
    //   inverse  Us[q][i] = s_q u_m(theta_i)/2, Vs = s_q v_m(theta_i)/2 on box rows (q x (Ng+1))
    void *d_Cs = nullptr, *d_Us = nullptr, *d_Vs = nullptr;
};

// A discrete Fourier transform X_k = sum_{n<S} x_n exp(-2 pi i n k / L), k < K, batched over
// rows of length L.  L a power of two: direct radix-4 FFT (P = 0).  Otherwise Bluestein's
// chirp-z form: X_k = w_k sum_n (x_n w_n) conj(w_{k-n}), w_m = exp(-i pi m^2 / L), as a cyclic
// convolution of power-of-two length P >= S + K - 1.
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_DF = 2 };   // element type of a transform

// Twiddle tables of one precision: tw[k] = omega_{Ltab}^k (k < Ltab) and, when stw is set,
// the stage tables of the shared-memory radix-4 stages: for block length Lb = 2^lb
// (lb = 2..min(12, log2 Ltab)), stw[stw_base(lb) + r*(Lb/4) + n0] = omega_{Lb}^{(r+1) n0},
// r = 0..2, contiguous in n0 so that a warp's twiddle loads are coalesced.
struct Twiddles {
    const void *tw = nullptr;
    int64_t Ltab = 0;
    const void *stw = nullptr;
    const void *fma = nullptr;   // FP64 only: TwFma tables of the decimation-in-time stages
    int lmax = 0;                // the stage tables cover block lengths up to 2^lmax
    const void *twq = nullptr;   // omega_{Ltabq}^k, k < Ltabq, for the odd-radix step of lengths q 2^b
    int64_t Ltabq = 0;           // a multiple of every such length (0: none)
};
// L = q 2^b (b >= 0, q = 3 or 5): transforms of such lengths take one radix-q step and
// power-of-two FFTs
__host__ __device__ inline bool cjt_is_qpow2(int64_t L, int q) {
    if (L < q || L % q != 0) return false;
    const int64_t r = L / q;
    return (r & (r - 1)) == 0;
}
__host__ __device__ inline bool cjt_is_3pow2(int64_t L) { return cjt_is_qpow2(L, 3); }
__host__ __device__ inline bool cjt_is_5pow2(int64_t L) { return cjt_is_qpow2(L, 5); }
// the odd factor q of L = q 2^b (3 or 5), 1 for a power of two, 0 for any other length
__host__ __device__ inline int cjt_odd_radix(int64_t L) {
    if (L >= 1 && (L & (L - 1)) == 0) return 1;
    return cjt_is_3pow2(L) ? 3 : cjt_is_5pow2(L) ? 5 : 0;
}
__host__ __device__ inline int64_t stw_base(int lb) { return 3 * ((1LL << (lb - 2)) - 1); }

// Radix-4 decimation-in-time twiddles in fused multiply-add form (FP64 transforms).  For a
// stage of block length Lb = 2^lb and q < Lb/4, each w_j = omega_Lb^{jq} (j = 1, 2, 3) is
// written as sigma (1 + i t) when |Re w| >= |Im w| (sigma = Re w, t = Im w / Re w), else
// as sigma (t + i) (sigma = Im w, t = Re w / Im w): |t| <= 1 and |sigma| >= 1/sqrt(2).
// Then w x = (sx e0, sy e1) with e0 = u0 - t u1, e1 = u1 + t u0, where (u0, u1) is x or,
// in the second form, x with its parts swapped, and (sx, sy) = (sigma, sigma) or
// (-sigma, sigma).  Factoring sigma_1 out of w1 x1 +- w3 x3 leaves 22 multiply-adds per
// butterfly instead of 28 operations (Goedecker's FMA radix-4 butterfly).
struct __align__(16) TwFma {
    double t1, t2, t3;    // t of w1, w2, w3
    double s1x, s1y;      // (sx, sy) of w1
    double s2x, s2y;      // (sx, sy) of w2
    double rx, ry;        // (sx, sy) of w3 divided by those of w1
    int flags;            // bit j-1: w_j in the sigma (t + i) form
    int pad_;
};
__host__ __device__ inline int64_t twfma_base(int lb) { return (1LL << (lb - 2)) - 1; }
inline int64_t prec_cbytes(int prec) { return prec == PREC_F32 ? 8 : 16; }   // bytes of one complex
struct Dft {
    int64_t L = 0, S = 0, K = 0, P = 0;
    int prec = PREC_F64;
    void *chirp = nullptr;  // w_m, m < max(S, K)
    void *bhat = nullptr;   // FFT_P of the cyclically arranged conj(w)
    int64_t fft_len() const { return P ? P : L; }
};

// Execution workspace of a plan: one arena carved into these buffers.  A plan owns
// one unless it was built with shared_workspace, in which case the caller (or the
// batched executor) supplies the arena.
struct Workspace {
    void *fft_f = nullptr, *fft_i = nullptr, *scratch = nullptr, *work = nullptr;
    double *dct = nullptr, *y = nullptr, *g = nullptr, *part_f = nullptr, *part_i = nullptr;
    void *xdf = nullptr;   // CJT_DFLOAT: the input c (forward) or g (inverse) as double-floats,
                           // scaled by an exact power of two 2^-e so that max |x| < 1
    int *exps = nullptr;   // CJT_DFLOAT: per-block exponents of max |x|, then e at [CJT_EXP_BLOCKS]
    double *conv = nullptr;// parameter shifts: two coefficient buffers of N+1 and the scan's chunk maps
};
constexpr int CJT_CONV_CHUNK = 1024;   // degrees per chunk of the bidiagonal solve's scan
__host__ __device__ inline int64_t cjt_conv_chunks(int64_t N) { return (N + 1 + CJT_CONV_CHUNK - 1) / CJT_CONV_CHUNK; }
enum { WS_FFT_F, WS_FFT_I, WS_SCRATCH, WS_WORK, WS_DCT, WS_Y, WS_G, WS_PART_F, WS_PART_I, WS_XDF, WS_EXPS,
       WS_CONV, WS_COUNT };
constexpr int CJT_EXP_BLOCKS = 128;

struct cjt_plan_s {
    int64_t N = 0;
    int dev = 0;                         // the device current when the plan was built
    double alpha = 0, beta = 0;          // the parameters the method runs on, in [-1/2, 1/2]^2
    double alpha_user = 0, beta_user = 0;// the caller's: alpha + shift_a, beta + shift_b
    int shift_a = 0, shift_b = 0;        // integer shifts (-1, 0, +1), Sec. 1.2
    cjt_plan_opts opts{};
    int M = 7;
    int64_t n_M = 0;
    double ratio = 0.5;
    bool corner = false;          // (alpha, beta) at a corner of the square: Hahn's series terminates
    int expansion_used = CJT_EXPANSION_HAHN;   // the asymptotic formula of the plan
    int seg_len = 2048;

    RecTables rt{};
    double *d_tabs = nullptr;     // one allocation holding the recurrence tables
    int64_t Jcap = 0;
    double *d_Cnm = nullptr;      // (M+1) x (N+1)

    GridWork fw, iv;

    // transforms
    int64_t Gf = 0, Gi = 0;       // Lobatto grids: forward x_j = cos(pi j/Gf), inverse cos(pi j/(2 Gi))
    int64_t Lf = 0, Li = 0;       // forward ASY/DCT length 2 Gf; inverse 4 Gi
    int64_t Ltab = 0;
    void *d_tw64 = nullptr;       // double2[Ltab]
    void *d_tw32 = nullptr;       // float2[Ltab]
    void *d_twdf = nullptr;       // dfc[Ltab]
    void *d_stw64 = nullptr, *d_stw32 = nullptr, *d_stwdf = nullptr;   // stage tables (Twiddles)
    void *d_twfma = nullptr;      // TwFma tables (FP64 decimation-in-time stages)
    int64_t Ltabq = 0;            // odd-radix twiddles omega_{Ltabq}^k (grids q 2^a, q = 3, 5): 4G, or 2G
    void *d_twq_64 = nullptr, *d_twq_32 = nullptr, *d_twqdf = nullptr;
    int stw_lmax = 0;             // the stage tables' top level (block length 2^stw_lmax)
    void *twc = nullptr;          // the shared twiddle tables the fields above point into
    Twiddles twiddles(int prec) const {
        Twiddles t;
        t.Ltab = Ltab;
        t.tw = prec == PREC_F32 ? d_tw32 : prec == PREC_DF ? d_twdf : d_tw64;
        t.stw = prec == PREC_F32 ? d_stw32 : prec == PREC_DF ? d_stwdf : d_stw64;
        t.fma = prec == PREC_F64 ? d_twfma : nullptr;
        t.lmax = stw_lmax;
        t.twq = prec == PREC_F32 ? d_twq_32 : prec == PREC_DF ? d_twqdf : d_twq_64;
        t.Ltabq = Ltabq;
        return t;
    }
    int prec_asy = PREC_F64;      // element type of the asymptotic transforms
    int npair_f = 0, npair_i = 0; // complex transforms of ASY item pairs
    Dft dft_f, dft_dct, dft_front, dft_i, dft_cc;
    // workspace layout (byte offsets and sizes within the arena) and the owned workspace
    int64_t ws_off[WS_COUNT] = {0};
    int64_t ws_size[WS_COUNT] = {0};
    int64_t ws_bytes = 0;
    bool shared_ws = false;
    Workspace ws{};
    double *d_w = nullptr;        // inverse: Clenshaw--Curtis weights (2N+1)
    double *d_s = nullptr;        // inverse: 1/A_n (N+1)
    double *d_in = nullptr, *d_out = nullptr;  // staging for cjt_execute_host

    // concurrency guard
    cudaStream_t last_stream = nullptr;
    cudaEvent_t done = nullptr;
    bool has_pending = false;

    int64_t device_bytes = 0;
    double plan_ms = 0;
    // CJT_MIXED: bound on the error the FP32 transforms add, per unit ||c_in||_1, for each
    // direction (cjt_error_bound); 0 in the other forms
    double err_mixed_fwd = 0, err_mixed_inv = 0;
    std::vector<void *> allocs;

    // stage profiling (CUDA events on the launching stream)
    bool prof = false;
    struct ProfRec { int stage; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
};

// Records an event pair around a stage when the plan is being profiled.
struct StageTimer {
    cjt_plan_s *p;
    cudaStream_t st;
    int stage;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(cjt_plan_s *p_, cudaStream_t st_, int stage_) : p(p_), st(st_), stage(stage_) {
        if (!p->prof) return;
        a = take();
        b = take();
        if (a) cudaEventRecord(a, st);
    }
    ~StageTimer() {
        if (!p->prof || !a || !b) return;
        cudaEventRecord(b, st);
        p->prof_pending.push_back({stage, a, b});
    }
    cudaEvent_t take() {
        if (!p->prof_pool.empty()) {
            cudaEvent_t e = p->prof_pool.back();
            p->prof_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
};

// ---------------------------------------------------------------------------
// Stirling series and Hahn coefficients (host and device)
// ---------------------------------------------------------------------------
#include "stirling_coeffs.h"
static __constant__ double cjt_stirling_a_dev[CJT_STIRLING_NCOEF] = {CJT_STIRLING_LIST};

// Terms of the truncated Stirling series S_eps(z), z >= 9 (Sec. 4.1, Table "Stirling").
__host__ __device__ inline int cjt_stirling_terms(double z) {
    if (z >= 3275) return 4;
    if (z >= 591) return 5;
    if (z >= 196) return 6;
    if (z >= 92) return 7;
    if (z >= 53) return 8;
    if (z >= 35) return 9;
    if (z >= 26) return 10;
    if (z >= 20) return 11;
    if (z >= 17) return 12;
    if (z >= 14) return 13;
    if (z >= 12) return 14;
    if (z >= 11) return 15;
    if (z >= 10) return 16;
    return 17;
}

__host__ __device__ inline double cjt_stirling_S(double z) {
#ifdef __CUDA_ARCH__
    const double *a = cjt_stirling_a_dev;
#else
    const double *a = cjt_stirling_a_host;
#endif
    int nt = cjt_stirling_terms(z);
    double w = 1.0 / z, s = 0.0;
    for (int k = nt - 1; k >= 0; --k) s = fma(s, w, a[k]);
    return s;
}

// C_{n,m} by the Stirling/log1p form Eq. "Cnmabasy"; valid for n + min(a,b) >= 8.
__host__ __device__ inline double cjt_hahn_C_asy(double n, int m, double a, double b) {
    const double c = 2.0 * n + a + b + m + 2.0;
    double t = (n + a + 0.5) * log1p((a - b - m) / c) + (n + b + 0.5) * log1p((b - a - m) / c) -
               (m + 0.5) * log1p((a + b + m + 2.0) / (2.0 * n));
    double pre = exp((double)m) * ldexp(1.0, -2 * m) * 0.56418958354775628695;  // e^m / (4^m sqrt(pi))
    return pre * pow(n, -(m + 0.5)) * exp(t) * cjt_stirling_S(n + a + 1.0) * cjt_stirling_S(n + b + 1.0) /
           cjt_stirling_S(c);
}

// C_{n,m} for any n >= 0: Eq. "Cnmabasy" where valid, otherwise the downward
// recurrence of Eq. "Cnmabrec" from the first valid degree.
__host__ __device__ inline double cjt_hahn_C(int64_t n, int m, double a, double b) {
    double mn = a < b ? a : b;
    int64_t n0 = (int64_t)ceil(8.0 - mn);
    if (n >= n0) return cjt_hahn_C_asy((double)n, m, a, b);
    double C = cjt_hahn_C_asy((double)n0, m, a, b);
    for (int64_t k = n0; k > n; --k) {
        double kk = (double)k;
        C = C * (kk + 0.5 * (a + b + m + 1.0)) * (kk + 0.5 * (a + b + m)) / ((kk + a) * (kk + b));
    }
    return C;
}

// h_l(a) = (1/2+a)_l (1/2-a)_l / l!  (the factors of f_m, Eq. "Jacasy")
__host__ __device__ inline double cjt_hahn_h(int l, double a) {
    double r = 1.0;
    for (int k = 0; k < l; ++k) r *= (0.5 + a + k) * (0.5 - a + k) / (k + 1.0);
    return r;
}

// ---------------------------------------------------------------------------
// The asymptotic expansion a plan uses.  Each term m has the DCT-I / DST-I form
//   C_{n,m} [u_m(theta) cos(n theta) + v_m(theta) sin(n theta)]          (Eq. "Jacasyuv")
// from cos(n theta - phi) = cos(n theta) cos(phi) + sin(n theta) sin(phi).
//  * Hahn's formula for general (alpha, beta) (Eq. "Jacasy"): term m sums the m+1
//    cosines h_l(a) h_{m-l}(b) cos(n theta - phi_{m,l}) / (sin^{l+a+1/2}(theta/2)
//    cos^{m-l+b+1/2}(theta/2)), phi_{m,l} = (a+l+1/2) pi/2 - (a+b+m+1) theta/2.  Since
//    h_l(+-1/2) = 0 for l >= 1, the sum keeps only l = 0 when a = +-1/2 and only l = m
//    when b = +-1/2 (App. B.2-B.3): those terms are skipped, not evaluated.
//  * The ultraspherical formula for alpha = beta = lambda - 1/2 (App. B.1): term m is the
//    single cosine C^lambda_{n,m} cos(n theta - (m+lambda)(pi/2 - theta)) /
//    sin^{m+lambda}(theta); for lambda in (0, 1) the remainder after M terms is below
//    twice the first neglected term.
// ---------------------------------------------------------------------------
struct AsyExp {
    int ultra = 0;            // 1: ultraspherical formula; 0: Hahn's formula
    double a = 0, b = 0;      // Jacobi parameters (a = b when ultra)
    double lam = 0;           // lambda = a + 1/2 (ultra)
    double ha[21] = {0}, hb[21] = {0};   // h_l(a), h_l(b), l = 0..20
};

// C^lambda_{n,0} = 2^lambda Gamma(n+lambda+1/2) / (sqrt(pi) Gamma(n+lambda+1)).  With
// x = n + lambda >= 9, the Stirling series (Sec. 4.1) gives the gamma ratio as
// e^{1/2} (x+1)^{-1/2} exp(x log1p(-1/(2(x+1)))) S(x+1/2) / S(x+1); below, the downward
// recurrence C^lambda_{n-1,0} = C^lambda_{n,0} (n+lambda) / (n+lambda-1/2).  Then
// C^lambda_{n,m} = C^lambda_{n,m-1} (lambda+m-1)(m-lambda) / (2m(n+lambda+m))  (App. B.1).
__host__ __device__ inline double cjt_ultra_C0_asy(double x) {
    return 1.6487212707001281468 / sqrt(x + 1.0) * exp(x * log1p(-0.5 / (x + 1.0))) *
           cjt_stirling_S(x + 0.5) / cjt_stirling_S(x + 1.0);
}
__host__ __device__ inline double cjt_ultra_C(int64_t n, int m, double lam) {
    const int64_t n0 = (int64_t)ceil(9.0 - lam);
    double C;
    if (n >= n0) {
        C = cjt_ultra_C0_asy((double)n + lam);
    } else {
        C = cjt_ultra_C0_asy((double)n0 + lam);
        for (int64_t k = n0; k > n; --k) C = C * ((double)k + lam) / ((double)k + lam - 0.5);
    }
    C *= exp2(lam) * 0.56418958354775628695;   // 2^lambda / sqrt(pi)
    for (int k = 1; k <= m; ++k) C = C * ((lam + k - 1.0) * (k - lam)) / (2.0 * k * ((double)n + lam + k));
    return C;
}

// sin(pi x) and cos(pi x): the device's sinpi/cospi; on the host, sin and cos after an exact
// reduction of x to [0, 1/2] (x mod 2, then 1 - r and 1/2 - r, exact by Sterbenz's lemma),
// so that the values keep their relative accuracy near the zeros.
inline double cjt_host_sinpi(double x) {
    double r = std::fmod(std::fabs(x), 2.0), sg = x < 0 ? -1.0 : 1.0;
    if (r >= 1.0) { r -= 1.0; sg = -sg; }
    if (r > 0.5) r = 1.0 - r;
    return sg * std::sin(3.14159265358979323846 * r);
}
inline double cjt_host_cospi(double x) {
    double r = std::fmod(std::fabs(x), 2.0), sg = 1.0;
    if (r >= 1.0) { r -= 1.0; sg = -1.0; }
    if (r <= 0.25) return sg * std::cos(3.14159265358979323846 * r);
    if (r <= 0.75) return sg * std::sin(3.14159265358979323846 * (0.5 - r));
    return -sg * std::cos(3.14159265358979323846 * (1.0 - r));
}
__host__ __device__ inline void cjt_sincospi_(double x, double *s, double *c) {
#ifdef __CUDA_ARCH__
    sincospi(x, s, c);
#else
    *s = cjt_host_sinpi(x);
    *c = cjt_host_cospi(x);
#endif
}
__host__ __device__ inline double cjt_sinpi_(double x) {
#ifdef __CUDA_ARCH__
    return sinpi(x);
#else
    return cjt_host_sinpi(x);
#endif
}
__host__ __device__ inline double cjt_cospi_(double x) {
#ifdef __CUDA_ARCH__
    return cospi(x);
#else
    return cjt_host_cospi(x);
#endif
}

// C_{n,m} of the plan's expansion
__host__ __device__ inline double cjt_asy_C(const AsyExp &e, int64_t n, int m) {
    return e.ultra ? cjt_ultra_C(n, m, e.lam) : cjt_hahn_C(n, m, e.a, e.b);
}

// Envelope of |term m| / C_{n,m} at theta = pi i / Ng, 0 < i < Ng: Hahn's g_m (Sec. 2.2),
// or 1/sin^{m+lambda}(theta) (App. B.1)
// Hahn's terms at theta = pi i / Ng share powers of S = 1/sin(theta/2) and C = 1/cos(theta/2):
// the l-th term of order m has the magnitude h_l(a) h_{m-l}(b) S^(l+a+1/2) C^(m-l+b+1/2)
// = P_m h_l(a) h_{m-l}(b) t^l with P_m = S^(a+1/2) C^(m+b+1/2) and t = S / C = cot(theta/2),
// so the sums over l are polynomials in t, evaluated by Horner's rule (their coefficients
// are non-negative for |a|, |b| <= 1/2), with one exponential and two logarithms per (row, m).
__host__ __device__ inline double cjt_asy_env(const AsyExp &e, int m, int64_t i, int64_t Ng) {
    if (e.ultra) return exp(-(m + e.lam) * log(cjt_sinpi_((double)i / (double)Ng)));
    const double half = (double)i / (2.0 * (double)Ng);
    const double sh = cjt_sinpi_(half), ch = cjt_cospi_(half);
    const double P = exp(-(e.a + 0.5) * log(sh) - (m + e.b + 0.5) * log(ch));
    const double t = ch / sh;
    double s = 0.0;
    for (int l = m; l >= 0; --l) s = fma(s, t, e.ha[l] * e.hb[m - l]);
    return P * s;
}

// u_m and v_m at theta = pi i / Ng, 0 < i < Ng.  The l-th term's phase is
// phi_{m,l} / pi = (a + l + 1/2)/2 - (a + b + m + 1) theta / (2 pi) = phi_{m,0} / pi + l / 2, so
// u_m + i v_m = P_m e^{i phi_{m,0}} sum_l h_l(a) h_{m-l}(b) (i t)^l = P_m e^{i phi_{m,0}} (A + i B),
// A and B the even and odd parts, polynomials in -t^2.
__host__ __device__ inline void cjt_asy_uv(const AsyExp &e, int m, int64_t i, int64_t Ng, double *u, double *v) {
    if (e.ultra) {
        const double x = (double)i / (double)Ng;
        const double mag = exp(-(m + e.lam) * log(cjt_sinpi_(x)));
        double s, c;
        cjt_sincospi_((m + e.lam) * (0.5 - x), &s, &c);   // phi / pi = (m+lambda)(1/2 - theta/pi)
        *u = mag * c;
        *v = mag * s;
        return;
    }
    const double half = (double)i / (2.0 * (double)Ng);
    const double sh = cjt_sinpi_(half), ch = cjt_cospi_(half);
    const double P = exp(-(e.a + 0.5) * log(sh) - (m + e.b + 0.5) * log(ch));
    const double t = ch / sh, w = -t * t;
    double A = 0.0, B = 0.0;
    for (int l = m - (m & 1); l >= 0; l -= 2) A = fma(A, w, e.ha[l] * e.hb[m - l]);
    for (int l = (m & 1) ? m : m - 1; l >= 1; l -= 2) B = fma(B, w, e.ha[l] * e.hb[m - l]);
    B *= t;
    double s, c;
    cjt_sincospi_(0.5 * (e.a + 0.5) - (e.a + e.b + m + 1.0) * half, &s, &c);
    *u = P * (A * c - B * s);
    *v = P * (A * s + B * c);
}

// The expansion for (a, b) in [-1/2, 1/2]^2 and the plan option (CJT_EXPANSION_*):
// ultraspherical when requested or by default when a = b with lambda in (0, 1).
// Returns CJT_EINVAL for an ultraspherical request with a != b.
inline int cjt_asy_make(double a, double b, int option, AsyExp *e) {
    *e = AsyExp{};
    e->a = a;
    e->b = b;
    for (int l = 0; l <= 20; ++l) { e->ha[l] = cjt_hahn_h(l, a); e->hb[l] = cjt_hahn_h(l, b); }
    if (option == CJT_EXPANSION_ULTRASPHERICAL && a != b) return CJT_EINVAL;
    const bool interior = a > -0.5 && a < 0.5;
    if (option != CJT_EXPANSION_HAHN && a == b && interior) {
        e->ultra = 1;
        e->lam = a + 0.5;
    }
    return CJT_OK;
}

// n_M (Sec. 2.2; App. B.1 for the ultraspherical formula): the degree above which the
// M-term remainder bound at theta = pi/2 is below eps
inline int64_t cjt_asy_nM(const AsyExp &e, int M, double eps) {
    double v;
    if (e.ultra) {
        double poch = 1.0, fact = 1.0;   // (lambda)_M (1-lambda)_M and M!
        for (int k = 0; k < M; ++k) { poch *= (e.lam + k) * (1.0 - e.lam + k); fact *= k + 1.0; }
        if (!(poch > 0)) return 0;
        v = std::pow(eps * 1.77245385090551602730 * std::ldexp(fact, M) / (std::exp2(e.lam + 1.0) * poch),
                     -1.0 / (M + 0.5));
    } else {
        // g_M(pi/2) = sum_l h_l(a) h_{M-l}(b) 2^{(M+a+b+1)/2}
        double gh = 0.0;
        for (int l = 0; l <= M; ++l) gh += e.ha[l] * e.hb[M - l];
        gh *= std::pow(2.0, 0.5 * (M + e.a + e.b + 1.0));
        if (!(gh > 0)) return 0;
        v = std::pow(eps * std::ldexp(1.0, 2 * M - 1) * 1.77245385090551602730 / gh, -1.0 / (M + 0.5));
    }
    return (int64_t)std::floor(v);
}

// ---------------------------------------------------------------------------
// launchers implemented in the .cu files
// ---------------------------------------------------------------------------
int cjt_fft_pow2(void *data, void *scratch, int64_t L, int64_t batch, const Twiddles &tw, int prec, cudaStream_t st);
// L a power of two, 3 2^b or 5 2^b (scratch of cjt_fft_scratch_elems(L, batch) elements)
int cjt_fft_any(void *data, void *scratch, int64_t L, int64_t batch, const Twiddles &tw, int prec, cudaStream_t st);
int64_t cjt_fft_scratch_elems(int64_t L, int64_t batch);
int cjt_fft_prime();
// Bluestein length (0 when L is a power of two)
int64_t cjt_dft_padded(int64_t L, int64_t S, int64_t K);
// chirp and bhat for a Bluestein transform (in d.prec); tw64 must cover P
int cjt_dft_setup(Dft &d, const void *tw64, int64_t Ltab, cudaStream_t st);
int cjt_dft_exec(const Dft &d, void *data, void *work, void *scratch, int64_t batch, const Twiddles &tw,
                 cudaStream_t st);
int64_t cjt_dft_work_bytes(const Dft &d, int64_t batch);
int64_t cjt_dft_scratch_bytes(const Dft &d, int64_t batch);

int cjt_plan_build(cjt_plan_s *p, cudaStream_t st);
// Stream-ordered temporary device memory for plan building, from a library-owned pool per
// device that keeps up to 1 GiB of freed memory for the next plans (free with cudaFreeAsync).
cudaError_t cjt_tmp_alloc(void **ptr, size_t bytes, cudaStream_t st);
// The plan's twiddle tables (from p->Ltab, p->Ltabq and the transform precision pa): taken
// from a per-device cache of tables shared by plans, built on `st` when absent.  A plan
// that took tables gives them back with cjt_release_twiddles.
int cjt_build_twiddles(cjt_plan_s *p, int pa, cudaStream_t st);
void cjt_release_twiddles(cjt_plan_s *p);
Workspace cjt_carve(const cjt_plan_s *p, void *base);
int cjt_exec_forward(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st);
int cjt_exec_inverse(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st);
// the transform entry points with the integer parameter shifts applied (Sec. 1.2)
int cjt_exec_forward_shifted(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st);
int cjt_exec_inverse_shifted(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st);
int cjt_conv_kernels(const cjt_plan_s *p);   // launches the conversions add to one execution
