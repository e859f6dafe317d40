// Measured FMA throughput of the GPU: the denominators of the FP64-pipe and FP32-pipe
// fractions that the benchmark reports beside the HBM roofline.  Not part of the method;
// the paper has no counterpart (its timings are CPU wall times).
//
// Every thread runs kChains independent FMA chains of `iters` steps (x <- x * a + b with
// |a| < 1, so the values stay normal and bounded), the grid holds 8 CTAs of 256 threads
// per SM, and the kernel is timed with CUDA events on the given stream.  The result of the
// chains is written only under a condition that never holds, which keeps the compiler
// from removing them without adding memory traffic.
#include <algorithm>

#include "sci_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) x[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < kChains; i++) x[i] = fma(x[i], a, b);
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += x[i];
    if (s == (T)-1.5e30) out[blockIdx.x] = s;
}

template <typename T>
int run(int device, int iters, cudaStream_t st, double *rate)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SCI_ERR_CUDA;
    const int blocks = sms * 8;
    T *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return SCI_ERR_NOMEM;
    int rc = SCI_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SCI_ERR_CUDA;
    if (rc == SCI_OK) {
        // one warm-up launch, then the timed one
        k_fma_rate<T><<<blocks, kThreads, 0, st>>>(out, std::max(1, iters / 8), (T)0.9999999, (T)1e-7);
        cudaEventRecord(e0, st);
        k_fma_rate<T><<<blocks, kThreads, 0, st>>>(out, iters, (T)0.9999999, (T)1e-7);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            rc = SCI_ERR_CUDA;
    }
    if (rc == SCI_OK) *rate = (double)blocks * kThreads * kChains * (double)iters / (ms * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

}  // namespace

extern "C" int sci_peak_fma(int device, int prec, int iters, void *cuda_stream, double *fma_per_s)
{
    if (!fma_per_s || iters < 8 || (prec != SCI_PREC_F64 && prec != SCI_PREC_F32_STORE_F64_ACC))
        return SCI_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SCI_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SCI_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return prec == SCI_PREC_F64 ? run<double>(device, iters, st, fma_per_s) : run<float>(device, iters, st, fma_per_s);
}
