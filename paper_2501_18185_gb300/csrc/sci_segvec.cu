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
//
// The projected matrices of those solvers (k x k, k <= 64) are diagonalised together by
// sci_syev_batched, one CTA per matrix (cyclic Jacobi, below).
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

// ---------------------------------------------------------------- batched eigensolver
// Eigenpairs of many small real symmetric matrices (the projected matrices G_s of the
// solvers), one CTA per matrix: the cyclic Jacobi method with the parallel (round-robin)
// ordering (Golub and Van Loan, Matrix Computations, Sec. 8.5).  A sweep is m - 1 steps
// (m = n rounded up to even); a step applies m/2 disjoint plane rotations at once, each
// chosen to zero its off-diagonal entry, as A <- J^T A J (rows, then columns) and V <- V J.
// Sweeps stop when the off-diagonal sum of squares falls below kJacobiTol^2 of the total,
// or after max_sweeps (then *not_converged is incremented).  The matrix and V live in
// shared memory (row stride n + 1).
constexpr int kJacobiThreads = 256;
constexpr int kJacobiNmax = 64;
constexpr double kJacobiTol = 1e-15;

__device__ __forceinline__ void jacobi_pair(int m, int step, int t, int &p, int &q)
{
    // circle method: player m-1 fixed, players 0..m-2 rotate
    int x, y;
    if (t == 0) {
        x = step;
        y = m - 1;
    } else {
        x = (step + t) % (m - 1);
        y = (step - t + (m - 1)) % (m - 1);
    }
    p = min(x, y);
    q = max(x, y);
}

__global__ void __launch_bounds__(kJacobiThreads)
k_syev_jacobi(int n, const double *__restrict__ A, int64_t lda, int64_t sA, double *__restrict__ w, int64_t sw,
              double *__restrict__ V, int64_t ldv, int64_t sV, int max_sweeps, int *not_converged)
{
    extern __shared__ double sm[];
    const int ld = n + 1;
    double *a = sm, *v = sm + n * ld;
    __shared__ double s_c[kJacobiNmax / 2], s_s[kJacobiNmax / 2];
    __shared__ int s_p[kJacobiNmax / 2], s_q[kJacobiNmax / 2];
    __shared__ double s_red[2][kJacobiThreads / 32];
    __shared__ int s_done;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *Ab = A + (int64_t)b * sA;
    for (int e = tid; e < n * n; e += kJacobiThreads) {
        const int i = e / n, j = e % n;
        a[i * ld + j] = 0.5 * (Ab[(int64_t)i * lda + j] + Ab[(int64_t)j * lda + i]);
        v[i * ld + j] = i == j ? 1.0 : 0.0;
    }
    const int m = (n + 1) & ~1, npair = m / 2;
    __syncthreads();
    bool converged = n <= 1;
    for (int sweep = 0; sweep < max_sweeps && !converged; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < n * n; e += kJacobiThreads) {
            const int i = e / n, j = e % n;
            const double x = a[i * ld + j] * a[i * ld + j];
            tot += x;
            if (i != j) off += x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (lane == 0) s_red[0][warp] = off, s_red[1][warp] = tot;
        __syncthreads();
        if (tid == 0) {
            double o2 = 0.0, t2 = 0.0;
            for (int k = 0; k < kJacobiThreads / 32; k++) o2 += s_red[0][k], t2 += s_red[1][k];
            s_done = o2 <= kJacobiTol * kJacobiTol * t2;
        }
        __syncthreads();
        converged = s_done;
        if (converged) break;
        for (int step = 0; step < m - 1; step++) {
            if (tid < npair) {
                int p, q;
                jacobi_pair(m, step, tid, p, q);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = a[p * ld + q];
                    if (apq != 0.0) {
                        const double tau = (a[q * ld + q] - a[p * ld + p]) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                s_p[tid] = p, s_q[tid] = q, s_c[tid] = c, s_s[tid] = s;
            }
            __syncthreads();
            // rows p, q of A (pairs with the padding index m - 1 = n, or no rotation, are skipped)
            for (int e = tid; e < npair * n; e += kJacobiThreads) {
                const int t = e / n, j = e % n, p = s_p[t], q = s_q[t];
                const double c = s_c[t], s = s_s[t];
                if (q >= n || s == 0.0) continue;
                const double x = a[p * ld + j], y = a[q * ld + j];
                a[p * ld + j] = c * x - s * y;
                a[q * ld + j] = s * x + c * y;
            }
            __syncthreads();
            // columns p, q of A and of V
            for (int e = tid; e < npair * n; e += kJacobiThreads) {
                const int t = e / n, i = e % n, p = s_p[t], q = s_q[t];
                const double c = s_c[t], s = s_s[t];
                if (q >= n || s == 0.0) continue;
                const double x = a[i * ld + p], y = a[i * ld + q];
                a[i * ld + p] = c * x - s * y;
                a[i * ld + q] = s * x + c * y;
                const double vx = v[i * ld + p], vy = v[i * ld + q];
                v[i * ld + p] = c * vx - s * vy;
                v[i * ld + q] = s * vx + c * vy;
            }
            __syncthreads();
        }
    }
    if (!converged && tid == 0 && not_converged) atomicAdd(not_converged, 1);
    // ascending order: eigenvalue j goes to the position of its rank (ties by index)
    for (int j = tid; j < n; j += kJacobiThreads) {
        const double lj = a[j * ld + j];
        int r = 0;
        for (int i = 0; i < n; i++) {
            const double li = a[i * ld + i];
            r += (li < lj) || (li == lj && i < j);
        }
        w[(int64_t)b * sw + r] = lj;
        for (int i = 0; i < n; i++) V[(int64_t)b * sV + (int64_t)i * ldv + r] = v[i * ld + j];
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

extern "C" int sci_syev_batched(int device, int nb, int n, const double *A, int64_t lda, int64_t strideA, double *w,
                                int64_t stridew, double *V, int64_t ldv, int64_t strideV, int max_sweeps,
                                int *not_converged, void *cuda_stream)
{
    if (nb < 0 || n < 0 || n > kJacobiNmax || max_sweeps < 1) return SCI_ERR_ARG;
    if (nb == 0 || n == 0) return SCI_OK;
    if (!A || !w || !V || lda < n || ldv < n || stridew < n || strideA < (int64_t)(n - 1) * lda + n ||
        strideV < (int64_t)(n - 1) * ldv + n)
        return SCI_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SCI_ERR_CUDA;
    const size_t smem = sizeof(double) * 2 * (size_t)n * (n + 1);
    // dynamic plus static shared memory above 48 KB needs the opt-in (the static part is
    // under 1 KB, so opt in from 40 KB of dynamic memory on)
    if (smem > 40 * 1024 &&
        cudaFuncSetAttribute(k_syev_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SCI_ERR_CUDA;
    k_syev_jacobi<<<nb, kJacobiThreads, smem, (cudaStream_t)cuda_stream>>>(n, A, lda, strideA, w, stridew, V, ldv, strideV,
                                                                         max_sweeps, not_converged);
    return cudaGetLastError() == cudaSuccess ? SCI_OK : SCI_ERR_CUDA;
}
