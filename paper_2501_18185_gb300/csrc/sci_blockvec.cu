// Block-vector kernels for the subspace algebra of block Davidson.
//
// The diagonalisation works through products sigma = H X (Sec. 2.4, the diagonalisation
// paragraph); around them a block Davidson solver keeps the search space V [M x k], its
// image W = H V, and for every new block T [M x a] needs only tall-skinny products:
//     P = A^T B          (A: M x k, B: M x a; projections, Gram matrices, new rows of G)
//     C = A1 S1 + A2 S2  (S: small; Gram-Schmidt updates, Ritz vectors, residuals)
// with M ~ 10^6 and k <= 256, a <= 16.  On GB300 the FP64 pipe (2 FMA/clk/SM) bounds these
// by a factor ~10 over HBM, and cuBLAS reaches ~20% of it at these shapes.  Both kernels
// take an arithmetic policy: FP64 (DFMA) or paired FP32 (sci_ds.cuh; 48-bit significands,
// FP64 folds every tile, ~5x the FP64 rate).
//
// P = A^T B: each CTA owns a contiguous range of rows, stages 32-row tiles of A and B in
// shared memory (split into float pairs there for the paired policy) and keeps the k x a
// outputs in registers, one column j and up to 8 rows i per thread.  Partials go to a
// context-owned buffer [grid][k][a] and a second kernel sums them in a fixed order (one
// warp per output), so the result is deterministic.
//
// C = A1 S1 + A2 S2: grid-stride over 32-row tiles; S1, S2 are staged once per CTA; a
// thread owns one row and columns j = slot, slot + 8.  Row-local: C may alias A1 or A2
// (same base and stride) when beta = 0, which the solver uses to update blocks in place.
// Optional epilogue for the Davidson residual: column sums of squares of the result
// (FP64 atomics, order not fixed) and the preconditioned output result / (shift_j - d_m)
// with the denominator clamped away from zero at 1e-8; the quotient is taken in FP32 (a
// search direction needs no more).
#include <algorithm>

#include "sci_ds.cuh"
#include "sci_internal.cuh"

namespace {

constexpr int kBvThreads = 256;
constexpr int kTnRows = 32;
constexpr int kNnRows = 32;

struct PolF64 {
    using E = double;
    using Acc = double;
    static __device__ __forceinline__ E load(double x) { return x; }
    static __device__ __forceinline__ void zero(Acc &a) { a = 0.0; }
    static __device__ __forceinline__ void fma(Acc &a, E x, E y) { a = ::fma(x, y, a); }
    static __device__ __forceinline__ void renorm(Acc &) {}
    static __device__ __forceinline__ double value(Acc a) { return a; }
    static __device__ __forceinline__ E zero_e() { return 0.0; }
};

struct PolDS {
    using E = float2;
    using Acc = sci::Ds;
    static __device__ __forceinline__ E load(double x) { return sci::ds_split_int(x); }
    static __device__ __forceinline__ void zero(Acc &a) { sci::ds_zero(a); }
    static __device__ __forceinline__ void fma(Acc &a, E x, E y) { sci::ds_fma(a, x, y); }
    static __device__ __forceinline__ void renorm(Acc &a) { sci::ds_renorm(a); }
    static __device__ __forceinline__ double value(Acc a) { return sci::ds_value(a); }
    static __device__ __forceinline__ E zero_e() { return make_float2(0.f, 0.f); }
};

// smallest power of two >= a (a in 1..16)
__host__ __device__ __forceinline__ int pow2_at_least(int a) { return a <= 1 ? 1 : a <= 2 ? 2 : a <= 4 ? 4 : a <= 8 ? 8 : 16; }

// ------------------------------------------------------------------ P = A^T B
template <class P, int NOUT>
__global__ void __launch_bounds__(kBvThreads)
k_bv_tn(int64_t M, int k, int a, const double *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb,
        double *__restrict__ part)
{
    using E = typename P::E;
    extern __shared__ __align__(16) unsigned char smem[];
    E *As = reinterpret_cast<E *>(smem);  // [kTnRows][k]
    E *Bs = As + kTnRows * k;             // [kTnRows][a]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int apad = pow2_at_least(a);
    const int j = t % apad, ig = t / apad, istep = kBvThreads / apad;
    const int64_t chunk = (M + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(M, r0 + chunk);

    typename P::Acc acc[NOUT];
    double tot[NOUT];
#pragma unroll
    for (int s = 0; s < NOUT; s++) P::zero(acc[s]), tot[s] = 0.0;

    for (int64_t base = r0; base < r1; base += kTnRows) {
        const int nr = (int)min((int64_t)kTnRows, r1 - base);
        __syncthreads();
        for (int r = warp; r < nr; r += kBvThreads / 32) {
            const double *arow = A + (base + r) * lda;
            for (int i = lane; i < k; i += 32) As[r * k + i] = P::load(arow[i]);
            if (lane < a) Bs[r * a + lane] = P::load(B[(base + r) * ldb + lane]);
        }
        __syncthreads();
        if (j < a) {
            for (int r = 0; r < nr; r++) {
                const E bv = Bs[r * a + j];
#pragma unroll
                for (int s = 0; s < NOUT; s++) {
                    const int i = ig + s * istep;
                    if (i < k) P::fma(acc[s], As[r * k + i], bv);
                }
            }
#pragma unroll
            for (int s = 0; s < NOUT; s++) tot[s] += P::value(acc[s]), P::zero(acc[s]);
        }
    }
    if (j < a) {
        double *out = part + (int64_t)blockIdx.x * k * a;
#pragma unroll
        for (int s = 0; s < NOUT; s++) {
            const int i = ig + s * istep;
            if (i < k) out[i * a + j] = tot[s];
        }
    }
}

// P[w] = sum_g part[g][w], one warp per output, fixed order
__global__ void k_bv_reduce(const double *__restrict__ part, int G, int n, double *__restrict__ out)
{
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= n) return;
    double s = 0.0;
    for (int g = lane; g < G; g += 32) s += part[(int64_t)g * n + w];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[w] = s;
}

// ------------------------------------------------------------------ C = A1 S1 + A2 S2
template <class P, int NJ>
__global__ void __launch_bounds__(kBvThreads)
k_bv_nn(int64_t M, int a, const double *A1, int64_t lda1, int k1, const double *__restrict__ S1, const double *A2,
        int64_t lda2, int k2, const double *__restrict__ S2, double beta, double *C, int64_t ldc,
        const double *__restrict__ dg, const double *__restrict__ shift, double *__restrict__ colsq)
{
    using E = typename P::E;
    constexpr int JW = 8 * NJ;  // staged width of S
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = k1 + k2, ldA = K + 1;
    E *Ss = reinterpret_cast<E *>(smem);  // [K][JW], zero beyond column a
    E *As = Ss + K * JW;                   // [kNnRows][K + 1]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int idx = t; idx < K * JW; idx += kBvThreads) {
        const int i = idx / JW, j = idx - i * JW;
        Ss[idx] = j >= a ? P::zero_e() : P::load(i < k1 ? S1[i * a + j] : S2[(i - k1) * a + j]);
    }
    const int r = t >> 3, slot = t & 7;
    double cs[NJ];
#pragma unroll
    for (int q = 0; q < NJ; q++) cs[q] = 0.0;

    for (int64_t base = (int64_t)blockIdx.x * kNnRows; base < M; base += (int64_t)gridDim.x * kNnRows) {
        const int nr = (int)min((int64_t)kNnRows, M - base);
        __syncthreads();
        for (int rr = warp; rr < nr; rr += kBvThreads / 32) {
            const double *a1 = k1 ? A1 + (base + rr) * lda1 : nullptr;
            const double *a2 = k2 ? A2 + (base + rr) * lda2 : nullptr;
            for (int i = lane; i < k1; i += 32) As[rr * ldA + i] = P::load(a1[i]);
            for (int i = lane; i < k2; i += 32) As[rr * ldA + k1 + i] = P::load(a2[i]);
        }
        __syncthreads();
        if (r < nr) {
            typename P::Acc acc[NJ];
#pragma unroll
            for (int q = 0; q < NJ; q++) P::zero(acc[q]);
            const E *arow = As + r * ldA;
            for (int i0 = 0; i0 < K; i0 += 16) {
                const int i1 = min(K, i0 + 16);
                for (int i = i0; i < i1; i++) {
                    const E av = arow[i];
#pragma unroll
                    for (int q = 0; q < NJ; q++) P::fma(acc[q], av, Ss[i * JW + slot + 8 * q]);
                }
#pragma unroll
                for (int q = 0; q < NJ; q++) P::renorm(acc[q]);
            }
            const int64_t m = base + r;
#pragma unroll
            for (int q = 0; q < NJ; q++) {
                const int j = slot + 8 * q;
                if (j >= a) continue;
                double v = P::value(acc[q]);
                double *cp = C + m * ldc + j;
                if (beta != 0.0) v = ::fma(beta, *cp, v);
                if (colsq) cs[q] = ::fma(v, v, cs[q]);
                if (dg) {
                    float den = sci::ds_split_int(shift[j] - dg[m]).x;
                    if (fabsf(den) < 1e-8f) den = 1e-8f;
                    v = sci::f2d_int(sci::ds_split_int(v).x / den);
                }
                *cp = v;
            }
        }
    }
    if (colsq) {
#pragma unroll
        for (int q = 0; q < NJ; q++) {
            double s = cs[q];
            s += __shfl_xor_sync(0xffffffffu, s, 8);
            s += __shfl_xor_sync(0xffffffffu, s, 16);
            if (lane < 8 && slot + 8 * q < a) atomicAdd(colsq + slot + 8 * q, s);
        }
    }
}

template <class P, int NOUT>
int launch_tn_n(sci_ctx *ctx, int64_t M, int k, int a, const double *A, int64_t lda, const double *B, int64_t ldb, double *P_out)
{
    using E = typename P::E;
    const size_t smem = (size_t)kTnRows * (k + a) * sizeof(E);
    auto kern = k_bv_tn<P, NOUT>;
    if (smem > 48 * 1024 &&
        sci_cuda_check(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "bv_tn attr"))
        return SCI_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (sci_cuda_check(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBvThreads, smem), "bv_tn occupancy") ||
        sci_cuda_check(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "bv_tn sms"))
        return SCI_ERR_CUDA;
    int64_t G = (int64_t)std::max(1, per_sm) * sms;
    G = std::max<int64_t>(1, std::min<int64_t>(G, (M + kTnRows - 1) / kTnRows));
    const size_t need = (size_t)G * k * a * sizeof(double);
    if (need > ctx->bv_bytes) {
        if (ctx->bv_part) cudaFree(ctx->bv_part);
        ctx->bv_part = nullptr, ctx->bv_bytes = 0;
        if (cudaMalloc(&ctx->bv_part, need) != cudaSuccess) return sci_fail(ctx, SCI_ERR_NOMEM, "bv_tn: partial buffer");
        ctx->bv_bytes = need;
    }
    double *part = static_cast<double *>(ctx->bv_part);
    kern<<<(unsigned)G, kBvThreads, smem, ctx->stream>>>(M, k, a, A, lda, B, ldb, part);
    const int n = k * a;
    k_bv_reduce<<<(unsigned)((n * 32 + 255) / 256), 256, 0, ctx->stream>>>(part, (int)G, n, P_out);
    return sci_cuda_check(ctx, cudaGetLastError(), "bv_tn launch") ? SCI_ERR_CUDA : SCI_OK;
}

template <class P>
int launch_tn(sci_ctx *ctx, int64_t M, int k, int a, const double *A, int64_t lda, const double *B, int64_t ldb, double *P_out)
{
    const int istep = kBvThreads / pow2_at_least(a);
    switch ((k + istep - 1) / istep) {
        case 1: return launch_tn_n<P, 1>(ctx, M, k, a, A, lda, B, ldb, P_out);
        case 2: return launch_tn_n<P, 2>(ctx, M, k, a, A, lda, B, ldb, P_out);
        case 3: return launch_tn_n<P, 3>(ctx, M, k, a, A, lda, B, ldb, P_out);
        case 4: return launch_tn_n<P, 4>(ctx, M, k, a, A, lda, B, ldb, P_out);
        case 5: return launch_tn_n<P, 5>(ctx, M, k, a, A, lda, B, ldb, P_out);
        case 6: return launch_tn_n<P, 6>(ctx, M, k, a, A, lda, B, ldb, P_out);
        case 7: return launch_tn_n<P, 7>(ctx, M, k, a, A, lda, B, ldb, P_out);
        case 8: return launch_tn_n<P, 8>(ctx, M, k, a, A, lda, B, ldb, P_out);
        default: return sci_fail(ctx, SCI_ERR_ARG, "bv_tn: k too large for a");
    }
}

template <class P, int NJ>
int launch_nn_n(sci_ctx *ctx, int64_t M, int a, const double *A1, int64_t lda1, int k1, const double *S1, const double *A2,
                int64_t lda2, int k2, const double *S2, double beta, double *C, int64_t ldc, const double *dg,
                const double *shift, double *colsq)
{
    using E = typename P::E;
    const int K = k1 + k2;
    const size_t smem = ((size_t)K * 8 * NJ + (size_t)kNnRows * (K + 1)) * sizeof(E);
    auto kern = k_bv_nn<P, NJ>;
    if (smem > 48 * 1024 &&
        sci_cuda_check(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "bv_nn attr"))
        return SCI_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (sci_cuda_check(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBvThreads, smem), "bv_nn occupancy") ||
        sci_cuda_check(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "bv_nn sms"))
        return SCI_ERR_CUDA;
    int64_t G = (int64_t)std::max(1, per_sm) * sms;
    G = std::max<int64_t>(1, std::min<int64_t>(G, (M + kNnRows - 1) / kNnRows));
    kern<<<(unsigned)G, kBvThreads, smem, ctx->stream>>>(M, a, A1, lda1, k1, S1, A2, lda2, k2, S2, beta, C, ldc, dg, shift,
                                                          colsq);
    return sci_cuda_check(ctx, cudaGetLastError(), "bv_nn launch") ? SCI_ERR_CUDA : SCI_OK;
}

}  // namespace

extern "C" int sci_bv_gemm_tn(sci_ctx *ctx, int64_t M, int k, int a, const double *A, int64_t lda, const double *B,
                              int64_t ldb, double *P, int prec)
{
    if (!ctx) return SCI_ERR_ARG;
    if (M < 0 || k < 1 || a < 1 || a > 16 || k > 8 * (kBvThreads / pow2_at_least(a)))
        return sci_fail(ctx, SCI_ERR_ARG, "bv_tn: need M >= 0, 1 <= a <= 16, 1 <= k <= 8*256/pow2(a)");
    if (!P || (M > 0 && (!A || !B)) || lda < k || ldb < a)
        return sci_fail(ctx, SCI_ERR_ARG, "bv_tn: null pointer or leading dimension below the width");
    if (prec != SCI_PREC_F64 && prec != SCI_PREC_F64_DS) return sci_fail(ctx, SCI_ERR_ARG, "bv_tn: prec must be F64 or F64_DS");
    if (sci_cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) return SCI_ERR_CUDA;
    if (M == 0) return sci_cuda_check(ctx, cudaMemsetAsync(P, 0, sizeof(double) * k * a, ctx->stream), "bv_tn zero") ? SCI_ERR_CUDA : SCI_OK;
    return prec == SCI_PREC_F64 ? launch_tn<PolF64>(ctx, M, k, a, A, lda, B, ldb, P)
                                : launch_tn<PolDS>(ctx, M, k, a, A, lda, B, ldb, P);
}

extern "C" int sci_bv_gemm_nn(sci_ctx *ctx, int64_t M, int a, const double *A1, int64_t lda1, int k1, const double *S1,
                              const double *A2, int64_t lda2, int k2, const double *S2, double beta, double *C, int64_t ldc,
                              const double *dg, const double *shift, double *colsq, int prec)
{
    if (!ctx) return SCI_ERR_ARG;
    if (M < 0 || a < 1 || a > 16 || k1 < 0 || k2 < 0 || k1 + k2 < 1 || k1 + k2 > 256)
        return sci_fail(ctx, SCI_ERR_ARG, "bv_nn: need M >= 0, 1 <= a <= 16, 1 <= k1 + k2 <= 256");
    if ((k1 > 0 && (!S1 || lda1 < k1 || (M > 0 && !A1))) || (k2 > 0 && (!S2 || lda2 < k2 || (M > 0 && !A2))) ||
        (M > 0 && !C) || ldc < a || (dg && !shift))
        return sci_fail(ctx, SCI_ERR_ARG, "bv_nn: null pointer or leading dimension below the width");
    if (prec != SCI_PREC_F64 && prec != SCI_PREC_F64_DS) return sci_fail(ctx, SCI_ERR_ARG, "bv_nn: prec must be F64 or F64_DS");
    if (sci_cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) return SCI_ERR_CUDA;
    if (M == 0) return SCI_OK;
    if (a <= 8)
        return prec == SCI_PREC_F64
                   ? launch_nn_n<PolF64, 1>(ctx, M, a, A1, lda1, k1, S1, A2, lda2, k2, S2, beta, C, ldc, dg, shift, colsq)
                   : launch_nn_n<PolDS, 1>(ctx, M, a, A1, lda1, k1, S1, A2, lda2, k2, S2, beta, C, ldc, dg, shift, colsq);
    return prec == SCI_PREC_F64
               ? launch_nn_n<PolF64, 2>(ctx, M, a, A1, lda1, k1, S1, A2, lda2, k2, S2, beta, C, ldc, dg, shift, colsq)
               : launch_nn_n<PolDS, 2>(ctx, M, a, A1, lda1, k1, S1, A2, lda2, k2, S2, beta, C, ldc, dg, shift, colsq);
}
