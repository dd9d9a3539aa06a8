// Allocation-free entry point: Chebyshev coefficients from values at the
// Chebyshev--Lobatto points, c = T_N^{-1} y (the last step of the forward
// transform), with all working memory in a fixed, file-scope device array.
//
// Who needs it: callers that cannot call cudaMalloc -- code that runs inside a
// host framework whose pool allocator owns the device memory and forbids raw
// allocations, latency-critical paths where an allocation may block or
// synchronise the device, and plug-ins whose host has already reserved almost
// all device memory.  Such callers pass only their input and output buffers.
//
// Limits and sharing: N <= CJT_NOALLOC_MAX_N (2^16) and N a power of two.  The
// array (3 x 2^17 complex doubles, 6 MiB) is reserved in every GPU that loads
// the library, for the life of the process.  Every call uses the same array
// and leaves its contents behind; each call rewrites every entry it reads, so
// nothing carries over between calls, but two calls whose work overlaps on the
// GPU (different streams, or different host threads) race on the array.
//
// Setup: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress while that device is current (the name is only a
// host-side stand-in in host code).  Make that first call before capturing a
// stream into a CUDA graph.
#include <cuda_runtime.h>

#include <mutex>

#include "cjt_internal.cuh"

namespace {

constexpr int64_t kMaxL = 2 * (int64_t)CJT_NOALLOC_MAX_N;   // transform length 2N
// [0, kMaxL): transform data; [kMaxL, 2 kMaxL): four-step scratch; [2 kMaxL, 3 kMaxL): twiddles
static __device__ __align__(256) double2 cjt_noalloc_scratch[3 * kMaxL];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2 *g_addr[kMaxDevices] = {nullptr};

int scratch_address(double2 **out) {
    int dev = 0;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CJT_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        CJT_CUDA_TRY(cudaGetSymbolAddress(&p, cjt_noalloc_scratch));
        g_addr[dev] = (double2 *)p;
    }
    *out = g_addr[dev];
    return CJT_OK;
}

__global__ void k_na_twiddles(int64_t L, double2 *tw) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= L) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    tw[k] = make_double2(c, s);
}

// even extension of y (length 2N): every entry of the transform buffer is written
__global__ void k_na_pack(int64_t N, const double *__restrict__ y, double2 *__restrict__ buf) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j > N) return;
    const double v = y[j];
    buf[j] = make_double2(v, 0.0);
    if (j >= 1 && j < N) buf[2 * N - j] = make_double2(v, 0.0);
}

// c_k = Re Z(k) / N, halved at k = 0 and k = N
__global__ void k_na_finish(int64_t N, const double2 *__restrict__ Z, double *__restrict__ c) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k > N) return;
    double v = Z[k].x / (double)N;
    if (k == 0 || k == N) v *= 0.5;
    c[k] = v;
}

__global__ void k_na_copy1(const double *__restrict__ y, double *__restrict__ c) { c[0] = y[0]; }

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" int cjt_cheb_coeffs_noalloc(int64_t N, const double *values_dev, double *c_cheb_dev, void *stream) {
    if (N < 0 || !values_dev || !c_cheb_dev) return CJT_EINVAL;
    if (N > CJT_NOALLOC_MAX_N || (N > 0 && (N & (N - 1)) != 0)) return CJT_EUNSUPPORTED;
    double2 *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0) {
        k_na_copy1<<<1, 1, 0, st>>>(values_dev, c_cheb_dev);
        CJT_CUDA_TRY(cudaGetLastError());
        return CJT_OK;
    }
    const int64_t L = 2 * N;
    double2 *buf = base, *scratch = base + kMaxL, *tw = base + 2 * kMaxL;
    k_na_twiddles<<<blocks_for(L, 256), 256, 0, st>>>(L, tw);
    k_na_pack<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, values_dev, buf);
    CJT_CUDA_TRY(cudaGetLastError());
    Twiddles T;
    T.tw = tw;
    T.Ltab = L;
    rc = cjt_fft_pow2(buf, scratch, L, 1, T, PREC_F64, st);
    if (rc) return rc;
    k_na_finish<<<blocks_for(N + 1, 256), 256, 0, st>>>(N, buf, c_cheb_dev);
    CJT_CUDA_TRY(cudaGetLastError());
    return CJT_OK;
}
