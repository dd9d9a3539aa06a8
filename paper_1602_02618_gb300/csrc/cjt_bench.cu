// Peak arithmetic microbenchmark: independent dependent-FMA chains on every SM.
// Used to state the FP64 / FP32 pipe peak, and the double-float rate, that the
// recurrence and transform kernels are compared against.
#include <cuda_runtime.h>

#include "cjt_df.cuh"
#include "cjt_internal.cuh"

namespace {
constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T *out, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)12345.678) out[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_df_chain(float *out, float ah, float al, float bh, float bl) {
    const dfs a = df_make(ah, al), b = df_make(bh, bl);
    dfs x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = df_make((float)(threadIdx.x + c) * 1e-3f, 0.f);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = df_add(df_mul(x[c], a), b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].h + x[c].l;
    if (s == 12345.678f) out[0] = s;  // keeps the chains live
}

template <typename T>
void launch_chain(int blocks, int threads, T *out, cudaStream_t st) {
    k_fma_chain<T><<<blocks, threads, 0, st>>>(out, (T)0.999999, (T)1e-7);
}
struct DfTag {};
template <>
void launch_chain<DfTag>(int blocks, int threads, DfTag *out, cudaStream_t st) {
    k_df_chain<<<blocks, threads, 0, st>>>((float *)out, 0.999999f, 1e-9f, 1e-7f, 1e-15f);
}

template <typename T>
int run(double *flops, cudaStream_t st) {
    int dev = 0, sms = 0;
    CJT_CUDA_TRY(cudaGetDevice(&dev));
    CJT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    T *out = nullptr;
    CJT_CUDA_TRY(cudaMallocAsync((void **)&out, 8, st));
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    CJT_CUDA_TRY(cudaEventCreate(&e0));
    CJT_CUDA_TRY(cudaEventCreate(&e1));
    launch_chain<T>(blocks, threads, out, st);  // warm-up
    CJT_CUDA_TRY(cudaEventRecord(e0, st));
    const int reps = sizeof(T) == 8 ? 2 : (sizeof(T) == 4 ? 20 : 4);
    for (int r = 0; r < reps; ++r) launch_chain<T>(blocks, threads, out, st);
    CJT_CUDA_TRY(cudaEventRecord(e1, st));
    CJT_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CJT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    *flops = 2.0 * kChains * (double)kIters * blocks * threads * reps / (ms * 1e-3);
    return CJT_OK;
}
}  // namespace

extern "C" int cjt_microbench_fma(int kind, double *flops, void *stream) {
    if (!flops) return CJT_EINVAL;
    if (kind == 0) return run<float>(flops, (cudaStream_t)stream);
    if (kind == 1) return run<double>(flops, (cudaStream_t)stream);
    if (kind == 2) return run<DfTag>(flops, (cudaStream_t)stream);
    return CJT_EINVAL;
}

// Transform microbenchmark for the autotuner: `batch` transforms of length 2^log2L in the
// precision's transform type (complex double, float or double-float), under the current
// cjt_fft_set_config of that class, timed with CUDA events on `stream` (average of `reps`
// after one warm-up).  The tables are taken as a plan takes them; the buffers are freed
// before returning.
extern "C" int cjt_fft_time(int precision, int log2L, int64_t batch, int reps, double *ms, void *stream) {
    if (!ms || log2L < 1 || log2L > 22 || batch < 1 || reps < 1) return CJT_EINVAL;
    if (precision != CJT_FP64 && precision != CJT_MIXED && precision != CJT_DFLOAT) return CJT_EINVAL;
    const int pa = precision == CJT_MIXED ? PREC_F32 : precision == CJT_DFLOAT ? PREC_DF : PREC_F64;
    const int64_t L = 1LL << log2L;
    if ((double)batch * (double)L * 16.0 > 8e9) return CJT_EUNSUPPORTED;   // at most 8 GB of data
    cudaStream_t st = (cudaStream_t)stream;
    cjt_plan_s tmp;
    tmp.Ltab = L;
    int rc = cjt_build_twiddles(&tmp, pa, st);
    void *data = nullptr, *scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t bytes = (size_t)(batch * L * prec_cbytes(pa));
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        if (data) cudaFree(data);
        if (scratch) cudaFree(scratch);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        for (void *v : tmp.allocs) cudaFree(v);
        tmp.allocs.clear();
        cjt_release_twiddles(&tmp);
    };
    if (!rc && cudaMalloc(&data, bytes) != cudaSuccess) rc = CJT_ENOMEM;
    if (!rc && L > 4096 && cudaMalloc(&scratch, bytes) != cudaSuccess) rc = CJT_ENOMEM;
    if (!rc && (cudaMemsetAsync(data, 0, bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                cudaEventCreate(&e1) != cudaSuccess))
        rc = CJT_ECUDA;
    const Twiddles tw = tmp.twiddles(pa);
    if (!rc) rc = cjt_fft_pow2(data, scratch, L, batch, tw, pa, st);
    if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = CJT_ECUDA;
    for (int r = 0; r < reps && !rc; ++r) rc = cjt_fft_pow2(data, scratch, L, batch, tw, pa, st);
    if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = CJT_ECUDA;
    float t = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        rc = CJT_ECUDA;
    if (!rc) *ms = (double)t / reps;
    cleanup();
    return rc;
}
