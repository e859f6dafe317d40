// Segmented block-vector products: the subspace algebra of many independent Davidson
// solvers whose vectors are stored end to end (the instances of a batch).
//
// The diagonalisation works through products sigma = H X (Sec. 2.4, the diagonalisation
// paragraph).  When many small Hamiltonians are diagonalised together, their search
// spaces share one column-major array A [k][M_total]: column j of instance s is the
// contiguous range [off_s, off_{s+1}) of row j.  Each solver needs, per instance,
//     out_s[j] = sum_{i in s} A[j][i] t[i]                       (projections, norms)
//     y[i] = beta_s y[i] + alpha1 sum_j A1[j][i] c1_s[j]
//                        + alpha2 sum_j A2[j][i] c2_s[j]          (Gram-Schmidt, Ritz
//                                                                  vectors, residuals)
// optionally followed by the diagonal preconditioner y[i] /= (shift_s - dg[i]).
//
// Work is cut into items of at most kSegRows rows that never straddle an instance, one
// CTA per item.  Columns are contiguous, so a warp reads 32 consecutive rows of a column
// (coalesced, one read of every element), and the passes are HBM-bound.  The projections
// write one partial row per item and a second kernel sums the items of each instance in
// item order: the result does not depend on scheduling.
#include <algorithm>
#include <string>
#include <vector>

#include "sci_internal.cuh"

namespace {

constexpr int kSegThreads = 256;
constexpr int kSegRows = 2048;
constexpr int kSegCols = 8;     // projection columns accumulated per pass over an item
constexpr int kSegKmax = 256;   // widest operand

struct SegItem {
    int seg;
    int64_t r0, r1;
};

__global__ void __launch_bounds__(kSegThreads)
k_seg_tn(const SegItem *__restrict__ items, int k, const double *__restrict__ A, int64_t lda,
         const double *__restrict__ t, double *__restrict__ part)
{
    __shared__ double red[kSegCols][kSegThreads / 32];
    const SegItem it = items[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j0 = 0; j0 < k; j0 += kSegCols) {
        const int nc = min(kSegCols, k - j0);
        double acc[kSegCols];
#pragma unroll
        for (int c = 0; c < kSegCols; c++) acc[c] = 0.0;
        for (int64_t i = it.r0 + threadIdx.x; i < it.r1; i += kSegThreads) {
            const double ti = __ldg(t + i);
#pragma unroll
            for (int c = 0; c < kSegCols; c++)
                if (c < nc) acc[c] = fma(__ldg(A + (int64_t)(j0 + c) * lda + i), ti, acc[c]);
        }
#pragma unroll
        for (int c = 0; c < kSegCols; c++) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
            if (lane == 0) red[c][warp] = acc[c];
        }
        __syncthreads();
        if (threadIdx.x < nc) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kSegThreads / 32; w++) s += red[threadIdx.x][w];
            part[(int64_t)blockIdx.x * k + j0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// out[s][j] = sum of the partial rows of the items of instance s (items [ib_s, ib_{s+1}))
__global__ void k_seg_reduce(const int *__restrict__ ib, int nseg, int k, const double *__restrict__ part,
                             double *__restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)nseg * k) return;
    const int s = (int)(q / k), j = (int)(q % k);
    double acc = 0.0;
    for (int it = ib[s]; it < ib[s + 1]; it++) acc += part[(int64_t)it * k + j];
    out[q] = acc;
}

__global__ void __launch_bounds__(kSegThreads)
k_seg_nn(const SegItem *__restrict__ items, double *y, const double *__restrict__ beta, int k1,
         const double *__restrict__ A1, int64_t lda1, const double *__restrict__ c1, double alpha1, int k2,
         const double *__restrict__ A2, int64_t lda2, const double *__restrict__ c2, double alpha2,
         const double *__restrict__ dg, const double *__restrict__ shift)
{
    __shared__ double sc[2 * kSegKmax];
    const SegItem it = items[blockIdx.x];
    const int s = it.seg;
    for (int j = threadIdx.x; j < k1; j += kSegThreads) sc[j] = alpha1 * c1[(int64_t)s * k1 + j];
    for (int j = threadIdx.x; j < k2; j += kSegThreads) sc[k1 + j] = alpha2 * c2[(int64_t)s * k2 + j];
    __syncthreads();
    const double b = beta ? beta[s] : 0.0;
    const double sh = dg ? shift[s] : 0.0;
    for (int64_t i = it.r0 + threadIdx.x; i < it.r1; i += kSegThreads) {
        double acc = b != 0.0 ? b * y[i] : 0.0;   // beta 0: y is not read
        for (int j = 0; j < k1; j++) acc = fma(__ldg(A1 + (int64_t)j * lda1 + i), sc[j], acc);
        for (int j = 0; j < k2; j++) acc = fma(__ldg(A2 + (int64_t)j * lda2 + i), sc[k1 + j], acc);
        if (dg) {
            double den = sh - __ldg(dg + i);
            if (fabs(den) < 1e-8) den = 1e-8;
            acc = acc / den;
        }
        y[i] = acc;
    }
}

}  // namespace

struct sci_seg {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nseg = 0, kmax = 0, nitems = 0;
    int64_t M = 0;
    SegItem *d_items = nullptr;
    int *d_ib = nullptr;          // [nseg + 1]: first item of each instance
    double *d_part = nullptr;     // [nitems][kmax] projection partials
    std::string err;
};

namespace {

int sfail(sci_seg *s, int code, const std::string &m)
{
    s->err = m;
    return code;
}

#define SCK(x)                                                                 \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess) return sfail(s, SCI_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" int sci_seg_create(sci_seg **out, int device, int nseg, const int64_t *offsets, int kmax, void *cuda_stream)
{
    if (!out) return SCI_ERR_ARG;
    *out = nullptr;
    if (nseg < 1 || !offsets || kmax < 1 || kmax > kSegKmax || offsets[0] != 0) return SCI_ERR_ARG;
    for (int q = 0; q < nseg; q++)
        if (offsets[q + 1] < offsets[q]) return SCI_ERR_ARG;
    std::vector<SegItem> items;
    std::vector<int> ib(nseg + 1, 0);
    for (int q = 0; q < nseg; q++) {
        ib[q] = (int)items.size();
        for (int64_t r = offsets[q]; r < offsets[q + 1]; r += kSegRows)
            items.push_back(SegItem{q, r, std::min(offsets[q + 1], r + kSegRows)});
        if (items.size() > (size_t)INT32_MAX / 2) return SCI_ERR_OVERFLOW;
    }
    ib[nseg] = (int)items.size();
    auto *s = new sci_seg();
    s->device = device;
    s->stream = (cudaStream_t)cuda_stream;
    s->nseg = nseg, s->kmax = kmax, s->nitems = (int)items.size(), s->M = offsets[nseg];
    const size_t ni = std::max<size_t>(1, items.size());
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&s->d_items, sizeof(SegItem) * ni) != cudaSuccess ||
        cudaMalloc(&s->d_ib, sizeof(int) * (nseg + 1)) != cudaSuccess ||
        cudaMalloc(&s->d_part, sizeof(double) * ni * kmax) != cudaSuccess ||
        (!items.empty() && cudaMemcpy(s->d_items, items.data(), sizeof(SegItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(s->d_ib, ib.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        sci_seg_destroy(s);
        return SCI_ERR_NOMEM;
    }
    *out = s;
    return SCI_OK;
}

extern "C" int sci_seg_destroy(sci_seg *s)
{
    if (!s) return SCI_OK;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    if (s->d_items) cudaFree(s->d_items);
    if (s->d_ib) cudaFree(s->d_ib);
    if (s->d_part) cudaFree(s->d_part);
    delete s;
    return SCI_OK;
}

extern "C" int sci_seg_tn(sci_seg *s, int k, const double *A, int64_t lda, const double *t, double *out)
{
    if (!s) return SCI_ERR_ARG;
    if (k < 1 || k > s->kmax) return sfail(s, SCI_ERR_ARG, "seg_tn: need 1 <= k <= kmax");
    if (!out || (s->M > 0 && (!A || !t)) || (k > 1 && lda < s->M)) return sfail(s, SCI_ERR_ARG, "seg_tn: null pointer or lda below M");
    SCK(cudaSetDevice(s->device));
    if (s->nitems > 0) {
        k_seg_tn<<<s->nitems, kSegThreads, 0, s->stream>>>(s->d_items, k, A, lda, t, s->d_part);
        SCK(cudaGetLastError());
    }
    const int64_t nq = (int64_t)s->nseg * k;
    k_seg_reduce<<<(unsigned)((nq + 255) / 256), 256, 0, s->stream>>>(s->d_ib, s->nseg, k, s->d_part, out);
    SCK(cudaGetLastError());
    return SCI_OK;
}

extern "C" int sci_seg_nn(sci_seg *s, double *y, const double *beta, int k1, const double *A1, int64_t lda1,
                          const double *c1, double alpha1, int k2, const double *A2, int64_t lda2, const double *c2,
                          double alpha2, const double *dg, const double *shift)
{
    if (!s) return SCI_ERR_ARG;
    if (k1 < 0 || k2 < 0 || k1 > s->kmax || k2 > s->kmax) return sfail(s, SCI_ERR_ARG, "seg_nn: need 0 <= k1, k2 <= kmax");
    if ((s->M > 0 && !y) || (k1 > 0 && (!c1 || (s->M > 0 && !A1) || (k1 > 1 && lda1 < s->M))) ||
        (k2 > 0 && (!c2 || (s->M > 0 && !A2) || (k2 > 1 && lda2 < s->M))) || (dg && !shift))
        return sfail(s, SCI_ERR_ARG, "seg_nn: null pointer or lda below M");
    SCK(cudaSetDevice(s->device));
    if (s->nitems == 0) return SCI_OK;
    k_seg_nn<<<s->nitems, kSegThreads, 0, s->stream>>>(s->d_items, y, beta, k1, A1, lda1, c1, alpha1, k2, A2, lda2, c2,
                                                       alpha2, dg, shift);
    SCK(cudaGetLastError());
    return SCI_OK;
}

extern "C" const char *sci_seg_last_error(const sci_seg *s) { return s ? s->err.c_str() : "null segment set"; }
