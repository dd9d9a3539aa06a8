// Integer parameter shifts (Sec. 1.2): the method runs on (alpha, beta) in [-1/2, 1/2]^2;
// a parameter in (1/2, 3/2] is reached from the square by one unit step.  The forward
// transform first solves R x = c (the caller's coefficients c are exact, and the solve is
// well conditioned: double-precision errors stay at 1e-16 ||c||_1); the inverse transform
// ends with the product R y.  (A step up from below -1/2 would need the solve on the
// inverse transform's output, whose errors it sums over all higher degrees.)
//
// The relation between Jacobi polynomials whose parameters differ by one,
//   (2n+a+b+1) P_n^{(a,b)} = (n+a+b+1) P_n^{(a,b+1)} + (n+a) P_{n-1}^{(a,b+1)},
// and its mirror image under the symmetry P_n^{(a,b)}(x) = (-1)^n P_n^{(b,a)}(-x),
//   (2n+a+b+1) P_n^{(a,b)} = (n+a+b+1) P_n^{(a+1,b)} - (n+b) P_{n-1}^{(a+1,b)},
// turn coefficients c in the basis (a, b) into coefficients in the raised basis by the
// upper-bidiagonal map R:  (R c)_n = f_n c_n + g_n c_{n+1},
//   f_n = (n+a+b+1)/(2n+a+b+1)   (f_0 = 1: P_0 = 1 in every basis),
//   g_n = +(n+1+a)/(2n+a+b+3)    raising b,
//   g_n = -(n+1+b)/(2n+a+b+3)    raising a.
// Lowering solves R x = y backwards, x_n = (y_n - g_n x_{n+1}) / f_n: a first-order linear
// recurrence, run as a chunked scan (chunk maps, one carry pass, chunk fill).
#include <cuda_runtime.h>

#include "cjt_internal.cuh"

namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ double conv_f(int64_t n, double a, double b) {
    return n == 0 ? 1.0 : ((double)n + a + b + 1.0) / (2.0 * (double)n + a + b + 1.0);
}
__device__ __forceinline__ double conv_g(int64_t n, double a, double b, int raise_alpha) {
    const double den = 2.0 * (double)n + a + b + 3.0;
    return raise_alpha ? -((double)n + 1.0 + b) / den : ((double)n + 1.0 + a) / den;
}

// out = R in  (in != out)
__global__ void k_conv_raise(int64_t N, double a, double b, int raise_alpha, const double *__restrict__ in,
                             double *__restrict__ out) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n > N) return;
    double v = conv_f(n, a, b) * in[n];
    if (n < N) v = fma(conv_g(n, a, b, raise_alpha), in[n + 1], v);
    out[n] = v;
}

// x_n = p_n + q_n x_{n+1} with p_n = y_n / f_n, q_n = -g_n / f_n (g_N taken as 0).
// Chunk c covers n in [c*CH, min(N, c*CH + CH - 1)]; its map x_start = P + Q x_{end+1}.
__global__ void k_conv_solve_chunk(int64_t N, double a, double b, int raise_alpha, const double *__restrict__ y,
                                   double2 *__restrict__ PQ) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= cjt_conv_chunks(N)) return;
    const int64_t n0 = c * CJT_CONV_CHUNK, n1 = min(N, n0 + CJT_CONV_CHUNK - 1);
    double P = 0.0, Q = 1.0;
    for (int64_t n = n1; n >= n0; --n) {
        const double f = conv_f(n, a, b), g = n < N ? conv_g(n, a, b, raise_alpha) : 0.0;
        const double q = -g / f;
        P = fma(q, P, y[n] / f);
        Q *= q;
    }
    PQ[c] = make_double2(P, Q);
}

// carry[c] = x at the first degree of chunk c+1 (x_{N+1} = 0 for the last chunk)
__global__ void k_conv_solve_carry(int64_t nchunk, const double2 *__restrict__ PQ, double *__restrict__ carry) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double x = 0.0;
    for (int64_t c = nchunk - 1; c >= 0; --c) {
        carry[c] = x;
        x = fma(PQ[c].y, x, PQ[c].x);
    }
}

// x may alias y: each thread reads y_n before writing x_n, within its own chunk
__global__ void k_conv_solve_fill(int64_t N, double a, double b, int raise_alpha, const double *y,
                                  const double *__restrict__ carry, double *x) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= cjt_conv_chunks(N)) return;
    const int64_t n0 = c * CJT_CONV_CHUNK, n1 = min(N, n0 + CJT_CONV_CHUNK - 1);
    double v = carry[c];
    for (int64_t n = n1; n >= n0; --n) {
        const double f = conv_f(n, a, b), g = n < N ? conv_g(n, a, b, raise_alpha) : 0.0;
        v = fma(-g / f, v, y[n] / f);
        x[n] = v;
    }
}

struct ConvStep {
    double a, b;      // the lower basis of the unit step
    int raise_alpha;  // which parameter the step raises
    int solve;        // 0: multiply by R (lower basis -> raised); 1: solve R x = y (raised -> lower)
};

// Steps from the caller's basis (alpha0 + shift_a, beta0 + shift_b) to the square
// (forward) or back (inverse); shifts are 0 or 1.
int conv_steps(const cjt_plan_s *p, bool forward, ConvStep *s) {
    const double a0 = p->alpha, b0 = p->beta, bu = p->beta_user;
    int k = 0;
    if (forward) {
        // alpha first (beta still the caller's), then beta (alpha already in the square)
        if (p->shift_a) s[k++] = {a0, bu, 1, 1};
        if (p->shift_b) s[k++] = {a0, b0, 0, 1};
    } else {
        if (p->shift_b) s[k++] = {a0, b0, 0, 0};
        if (p->shift_a) s[k++] = {a0, bu, 1, 0};
    }
    return k;
}

int apply_step(int64_t N, const ConvStep &s, const double *src, double *dst, double *scan, cudaStream_t st) {
    if (!s.solve) {
        k_conv_raise<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, s.a, s.b, s.raise_alpha, src, dst);
    } else {
        const int64_t nchunk = cjt_conv_chunks(N);
        double2 *PQ = reinterpret_cast<double2 *>(scan);
        double *carry = scan + 2 * nchunk;
        k_conv_solve_chunk<<<blocks_for(nchunk, 128), 128, 0, st>>>(N, s.a, s.b, s.raise_alpha, src, PQ);
        k_conv_solve_carry<<<1, 1, 0, st>>>(nchunk, PQ, carry);
        k_conv_solve_fill<<<blocks_for(nchunk, 128), 128, 0, st>>>(N, s.a, s.b, s.raise_alpha, src, carry, dst);
    }
    CJT_CUDA_TRY(cudaGetLastError());
    return CJT_OK;
}

}  // namespace

int cjt_conv_kernels(const cjt_plan_s *p) {
    if (p->N == 0) return 0;
    ConvStep s[2];
    const int k = conv_steps(p, true, s);
    int n = 0;
    for (int i = 0; i < k; ++i) n += s[i].solve ? 3 : 1;
    return n;   // the inverse uses the opposite steps: the same count
}

int cjt_exec_forward_shifted(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st) {
    ConvStep s[2];
    const int k = p->N > 0 ? conv_steps(p, true, s) : 0;
    if (k == 0) return cjt_exec_forward(p, ws, in, out, st);
    const int64_t N = p->N;
    double *buf[2] = {ws.conv, ws.conv + (N + 1)};
    double *scan = ws.conv + 2 * (N + 1);
    const double *cur = in;
    for (int i = 0; i < k; ++i) {
        double *dst = buf[i & 1];
        int rc = apply_step(N, s[i], cur, dst, scan, st);
        if (rc) return rc;
        cur = dst;
    }
    return cjt_exec_forward(p, ws, cur, out, st);
}

int cjt_exec_inverse_shifted(cjt_plan_s *p, const Workspace &ws, const double *in, double *out, cudaStream_t st) {
    ConvStep s[2];
    const int k = p->N > 0 ? conv_steps(p, false, s) : 0;
    if (k == 0) return cjt_exec_inverse(p, ws, in, out, st);
    const int64_t N = p->N;
    double *buf[2] = {ws.conv, ws.conv + (N + 1)};
    double *scan = ws.conv + 2 * (N + 1);
    int rc = cjt_exec_inverse(p, ws, in, buf[0], st);
    if (rc) return rc;
    const double *cur = buf[0];
    for (int i = 0; i < k; ++i) {
        double *dst = i == k - 1 ? out : buf[1];
        rc = apply_step(N, s[i], cur, dst, scan, st);
        if (rc) return rc;
        cur = dst;
    }
    return CJT_OK;
}
