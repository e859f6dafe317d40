// Row ranges of sigma: the data path of a row-partitioned sigma over several processes.
//
// The paper parallelises over processes with the static data (integrals, the basis)
// replicated on every process and the results distributed, then merged (Sec. 3.1, the
// MPI dynamic scheduler).  Here each process keeps the whole determinant list and the
// integrals, computes the rows [row_begin, row_end) of sigma, and the rows are merged by
// one all-gather (in the Python layer, over torch.distributed).
//
// A row range narrows the bucket tables to what its rows need.  The rows of a bucket
// member are computed from every member of the bucket, so a range keeps each (N-2)- and
// (N-1)-hole bucket that holds at least one member in the range, whole and in the order
// of the full tables (largest buckets first, so the windows of the sigma kernels stay
// equal-size runs); the position and size fields of the entries stay valid unchanged.
// The sigma kernels then compute only the members whose determinant is in the range
// (RANGED instantiations in sci_sigma.cu).
//
// Row costs (sci_row_costs) count, per row, the connected determinants: the off-diagonal
// elements of that row of H, which set the row's share of the sigma work and balance
// the ranges.
//
// The same file builds the row order of the deterministic accumulation
// (sci_set_deterministic): each table's entries sorted by row with a stable radix sort (so
// a row's entries come in ascending table position), and for each entry its position in
// that order, where sigma stores the entry's row sum.
#include <cub/cub.cuh>

#include <algorithm>

#include "sci_internal.cuh"

#define SCI_CK(call)                                                 \
    do {                                                             \
        int _rc = sci_cuda_check(ctx, (call), #call);                \
        if (_rc != SCI_OK) return _rc;                               \
    } while (0)

namespace {

struct Tmp {
    void *p = nullptr;
    ~Tmp() { if (p) cudaFree(p); }
    template <typename T> T *as() { return static_cast<T *>(p); }
};

int grid_for(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// bucket start of entry p: (N-2) table from e_pos, (N-1) table from e_meta
__device__ __forceinline__ int64_t start2(const uint32_t *e_pos, int64_t p) { return p - sci::pos_off(e_pos[p]); }
__device__ __forceinline__ int64_t start1(const uint32_t *e_meta, int64_t p)
{
    return p - (int64_t)sci::meta_off(e_meta[p]);
}

// mark[bucket start] = 1 for every bucket with a member in [rb, re)
template <bool ONE>
__global__ void k_mark(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_posmeta, int64_t E,
                       int64_t rb, int64_t re, uint8_t *__restrict__ mark)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = e_idx[p];
        if (I >= rb && I < re) mark[ONE ? start1(e_posmeta, p) : start2(e_posmeta, p)] = 1;
    }
}

// keep[p] = 1 when the bucket of entry p is marked
template <bool ONE>
__global__ void k_keep(const uint32_t *__restrict__ e_posmeta, int64_t E, const uint8_t *__restrict__ mark,
                       uint32_t *__restrict__ keep)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x)
        keep[p] = mark[ONE ? start1(e_posmeta, p) : start2(e_posmeta, p)];
}

// the kept entries at their new positions (dst = exclusive prefix sum of keep)
template <typename A, typename B, typename C>
__global__ void k_compact(int64_t E, const uint32_t *__restrict__ keep, const uint32_t *__restrict__ dst,
                          const A *__restrict__ a, const B *__restrict__ b, const C *__restrict__ c, A *__restrict__ a2,
                          B *__restrict__ b2, C *__restrict__ c2)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[p]) continue;
        const uint32_t d = dst[p];
        a2[d] = a[p];
        b2[d] = b[p];
        c2[d] = c[p];
    }
}

// connected pairs (I, J) with I in [rb, re): doubles (disjoint members of the bucket)
// and singles (the other members), over a table; integer atomics, exact
__global__ void k_range_count2(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
                               const uint32_t *__restrict__ e_pos, int64_t E, int64_t rb, int64_t re,
                               unsigned long long *out)
{
    unsigned long long cnt = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = e_idx[p];
        if (I < rb || I >= re) continue;
        const uint32_t pos = e_pos[p];
        const int64_t bs = p - sci::pos_off(pos), be = bs + sci::pos_size(pos);
        const uint32_t cp = e_code[p];
        for (int64_t q = bs; q < be; q++) cnt += !sci::codes_overlap(e_code[q], cp);
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

__global__ void k_range_count1(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_meta, int64_t E,
                               int64_t rb, int64_t re, unsigned long long *out)
{
    unsigned long long cnt = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = e_idx[p];
        if (I >= rb && I < re) cnt += sci::meta_size(e_meta[p]) - 1;
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// per-row costs: cost[I] += disjoint members of each (N-2) bucket of I, and += the other
// members of each (N-1) bucket of I
__global__ void k_cost2(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
                        const uint32_t *__restrict__ e_pos, int64_t E, unsigned long long *__restrict__ cost)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pos = e_pos[p];
        const int64_t bs = p - sci::pos_off(pos), be = bs + sci::pos_size(pos);
        const uint32_t cp = e_code[p];
        unsigned long long cnt = 0;
        for (int64_t q = bs; q < be; q++) cnt += !sci::codes_overlap(e_code[q], cp);
        if (cnt) atomicAdd(cost + e_idx[p], cnt);
    }
}

__global__ void k_cost1(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_meta, int64_t E,
                        unsigned long long *__restrict__ cost)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = sci::meta_size(e_meta[p]) - 1;
        if (c) atomicAdd(cost + e_idx[p], c);
    }
}

// Narrow one table to the buckets with a member in [rb, re).  A: idx, B: code or S,
// C: pos or meta (the field that locates the bucket start).
// a spectator string of K words, moved as one entry
template <int K> struct Words {
    uint64_t w[K];
};

template <bool ONE, typename B>
int narrow(sci_ctx *ctx, int64_t E, const uint32_t *idx, const B *bfield, const uint32_t *posmeta, int64_t rb,
           int64_t re, uint32_t *&o_idx, B *&o_b, uint32_t *&o_pm, int64_t &o_n)
{
    cudaStream_t st = ctx->stream;
    o_n = 0;
    if (E == 0) return SCI_OK;
    Tmp mark, keep, dst, tmp;
    SCI_CK(cudaMalloc(&mark.p, (size_t)E));
    SCI_CK(cudaMalloc(&keep.p, (size_t)E * 4));
    SCI_CK(cudaMalloc(&dst.p, (size_t)E * 4));
    SCI_CK(cudaMemsetAsync(mark.p, 0, (size_t)E, st));
    k_mark<ONE><<<grid_for(E), 256, 0, st>>>(idx, posmeta, E, rb, re, mark.as<uint8_t>());
    k_keep<ONE><<<grid_for(E), 256, 0, st>>>(posmeta, E, mark.as<uint8_t>(), keep.as<uint32_t>());
    SCI_CK(cudaGetLastError());
    size_t tb = 0;
    SCI_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, keep.as<uint32_t>(), dst.as<uint32_t>(), (int)E, st));
    SCI_CK(cudaMalloc(&tmp.p, tb ? tb : 16));
    SCI_CK(cub::DeviceScan::ExclusiveSum(tmp.p, tb, keep.as<uint32_t>(), dst.as<uint32_t>(), (int)E, st));
    uint32_t last[2] = {0, 0};
    SCI_CK(cudaMemcpyAsync(&last[0], dst.as<uint32_t>() + (E - 1), 4, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaMemcpyAsync(&last[1], keep.as<uint32_t>() + (E - 1), 4, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    const int64_t n = (int64_t)last[0] + last[1];
    if (n == 0) return SCI_OK;
    SCI_CK(cudaMalloc(&o_idx, (size_t)n * 4));
    SCI_CK(cudaMalloc(&o_b, (size_t)n * sizeof(B)));
    SCI_CK(cudaMalloc(&o_pm, (size_t)n * 4));
    ctx->range_bytes += (size_t)n * (8 + sizeof(B));
    k_compact<uint32_t, B, uint32_t><<<grid_for(E), 256, 0, st>>>(E, keep.as<uint32_t>(), dst.as<uint32_t>(), idx,
                                                                 bfield, posmeta, o_idx, o_b, o_pm);
    SCI_CK(cudaGetLastError());
    SCI_CK(cudaStreamSynchronize(st));
    o_n = n;
    return SCI_OK;
}

template <typename T> void release(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

__global__ void k_iota(uint32_t *v, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        v[t] = (uint32_t)t;
}

__global__ void k_row_count(const uint32_t *__restrict__ idx, int64_t n, uint32_t *__restrict__ cnt)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + idx[t], 1u);
}

__global__ void k_invert(const uint32_t *__restrict__ ent, int64_t n, uint32_t *__restrict__ inv)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        inv[ent[t]] = (uint32_t)t;
}

// The row order of one table: ptr = exclusive prefix sum of the per-row counts (M + 1),
// inv[p] = the position of entry p among the entries sorted by row (a stable radix sort,
// so ascending table position within a row)
int row_index(sci_ctx *ctx, int64_t E, const uint32_t *e_idx, uint32_t *&ptr, uint32_t *&inv)
{
    cudaStream_t st = ctx->stream;
    const int64_t M = ctx->M;
    SCI_CK(cudaMalloc(&ptr, sizeof(uint32_t) * (M + 1)));
    SCI_CK(cudaMalloc(&inv, sizeof(uint32_t) * (E > 0 ? E : 1)));
    Tmp cnt, keys_out, vals_in, tmp, ent;
    SCI_CK(cudaMalloc(&ent.p, sizeof(uint32_t) * (E > 0 ? E : 1)));
    SCI_CK(cudaMalloc(&cnt.p, sizeof(uint32_t) * (M + 1)));
    SCI_CK(cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t) * (M + 1), st));
    if (E > 0) {
        k_row_count<<<grid_for(E), 256, 0, st>>>(e_idx, E, cnt.as<uint32_t>());
        SCI_CK(cudaMalloc(&keys_out.p, sizeof(uint32_t) * E));
        SCI_CK(cudaMalloc(&vals_in.p, sizeof(uint32_t) * E));
        k_iota<<<grid_for(E), 256, 0, st>>>(vals_in.as<uint32_t>(), E);
        SCI_CK(cudaGetLastError());
        int bits = 1;
        while (bits < 32 && ((int64_t)1 << bits) < M) bits++;
        size_t tb = 0;
        SCI_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, e_idx, keys_out.as<uint32_t>(), vals_in.as<uint32_t>(),
                                               ent.as<uint32_t>(), (int)E, 0, bits, st));
        SCI_CK(cudaMalloc(&tmp.p, tb ? tb : 16));
        SCI_CK(cub::DeviceRadixSort::SortPairs(tmp.p, tb, e_idx, keys_out.as<uint32_t>(), vals_in.as<uint32_t>(),
                                               ent.as<uint32_t>(), (int)E, 0, bits, st));
        k_invert<<<grid_for(E), 256, 0, st>>>(ent.as<uint32_t>(), E, inv);
        SCI_CK(cudaGetLastError());
    }
    size_t tb2 = 0;
    Tmp tmp2;
    SCI_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb2, cnt.as<uint32_t>(), ptr, (int)(M + 1), st));
    SCI_CK(cudaMalloc(&tmp2.p, tb2 ? tb2 : 16));
    SCI_CK(cub::DeviceScan::ExclusiveSum(tmp2.p, tb2, cnt.as<uint32_t>(), ptr, (int)(M + 1), st));
    SCI_CK(cudaStreamSynchronize(st));
    ctx->det_bytes += sizeof(uint32_t) * (M + 1 + E);
    return SCI_OK;
}

}  // namespace

void sci_free_det(sci_ctx *ctx)
{
    release(ctx->det_ptr2);
    release(ctx->det_inv2);
    release(ctx->det_ptr1);
    release(ctx->det_inv1);
    release(ctx->det_part2);
    release(ctx->det_part1);
    ctx->bytes_held -= std::min(ctx->bytes_held, ctx->det_bytes);
    ctx->det_bytes = 0;
    ctx->det_nvec = 0;
}

extern "C" int sci_set_deterministic(sci_ctx *ctx, int max_nvec)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "no determinants");
    if (max_nvec < 0) return sci_fail(ctx, SCI_ERR_ARG, "max_nvec < 0");
    if (ctx->ranged && max_nvec > 0) return sci_fail(ctx, SCI_ERR_STATE, "a row range is set");
    SCI_CK(cudaSetDevice(ctx->device));
    SCI_CK(cudaStreamSynchronize(ctx->stream));
    sci_free_det(ctx);
    if (max_nvec == 0) return SCI_OK;
    const size_t sc = ctx->cplx ? 16 : 8;
    int rc = row_index(ctx, ctx->e2, ctx->e2_idx, ctx->det_ptr2, ctx->det_inv2);
    if (rc == SCI_OK) rc = row_index(ctx, ctx->e1, ctx->e1_idx, ctx->det_ptr1, ctx->det_inv1);
    if (rc == SCI_OK) {
        const size_t b2 = sc * max_nvec * (size_t)std::max<int64_t>(ctx->e2, 1);
        const size_t b1 = sc * max_nvec * (size_t)std::max<int64_t>(ctx->e1, 1);
        if (cudaMalloc(&ctx->det_part2, b2) != cudaSuccess || cudaMalloc(&ctx->det_part1, b1) != cudaSuccess) {
            cudaGetLastError();
            rc = sci_fail(ctx, SCI_ERR_NOMEM, "deterministic sigma: per-entry buffers");
        } else {
            ctx->det_bytes += b1 + b2;
        }
    }
    if (rc != SCI_OK) {
        ctx->det_bytes = 0;  // not yet counted in bytes_held
        sci_free_det(ctx);
        return rc;
    }
    ctx->bytes_held += ctx->det_bytes;
    ctx->det_nvec = max_nvec;
    return SCI_OK;
}

void sci_free_range(sci_ctx *ctx)
{
    sci_free_split(ctx, true);
    release(ctx->r2_idx);
    release(ctx->r2_code);
    release(ctx->r2_pos);
    release(ctx->r1_idx);
    release(ctx->r1_S);
    release(ctx->r1_meta);
    ctx->bytes_held -= std::min(ctx->bytes_held, ctx->range_bytes);
    ctx->range_bytes = 0;
    ctx->ranged = 0;
    ctx->row_b = ctx->row_e = 0;
    ctx->r1 = ctx->r2 = ctx->range_pairs = ctx->range_pairs2 = ctx->range_pairs1 = 0;
}

extern "C" int sci_set_row_range(sci_ctx *ctx, int64_t row_begin, int64_t row_end)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "no determinants");
    if (row_begin < 0 || row_end > ctx->M || row_begin > row_end)
        return sci_fail(ctx, SCI_ERR_ARG, "row range outside [0, M]");
    if (ctx->det_nvec > 0 && !(row_begin == 0 && row_end == ctx->M))
        return sci_fail(ctx, SCI_ERR_STATE, "deterministic mode is on");
    SCI_CK(cudaSetDevice(ctx->device));
    SCI_CK(cudaStreamSynchronize(ctx->stream));  // no launch in flight reads the old tables
    sci_free_range(ctx);
    if (row_begin == 0 && row_end == ctx->M) return SCI_OK;  // the whole list: full tables
    int rc = narrow<false, uint32_t>(ctx, ctx->e2, ctx->e2_idx, ctx->e2_code, ctx->e2_pos, row_begin, row_end,
                                     ctx->r2_idx, ctx->r2_code, ctx->r2_pos, ctx->r2);
    if (rc == SCI_OK) {
        if (ctx->nwords == 4) {   // spectator strings of four words: 32 bytes per entry
            Words<4> *o = nullptr;
            rc = narrow<true, Words<4>>(ctx, ctx->e1, ctx->e1_idx, reinterpret_cast<const Words<4> *>(ctx->e1_S),
                                        ctx->e1_meta, row_begin, row_end, ctx->r1_idx, o, ctx->r1_meta, ctx->r1);
            ctx->r1_S = reinterpret_cast<uint64_t *>(o);
        } else if (ctx->nwords == 3) {   // spectator strings of three words: 24 bytes per entry
            Words<3> *o = nullptr;
            rc = narrow<true, Words<3>>(ctx, ctx->e1, ctx->e1_idx, reinterpret_cast<const Words<3> *>(ctx->e1_S),
                                        ctx->e1_meta, row_begin, row_end, ctx->r1_idx, o, ctx->r1_meta, ctx->r1);
            ctx->r1_S = reinterpret_cast<uint64_t *>(o);
        } else if (ctx->nwords == 2) {   // spectator strings of two words: 16 bytes per entry
            ulonglong2 *o = nullptr;
            rc = narrow<true, ulonglong2>(ctx, ctx->e1, ctx->e1_idx, reinterpret_cast<const ulonglong2 *>(ctx->e1_S),
                                          ctx->e1_meta, row_begin, row_end, ctx->r1_idx, o, ctx->r1_meta, ctx->r1);
            ctx->r1_S = reinterpret_cast<uint64_t *>(o);
        } else {
            rc = narrow<true, uint64_t>(ctx, ctx->e1, ctx->e1_idx, ctx->e1_S, ctx->e1_meta, row_begin, row_end,
                                        ctx->r1_idx, ctx->r1_S, ctx->r1_meta, ctx->r1);
        }
    }
    unsigned long long *cnt = nullptr, h[2] = {0, 0};
    if (rc == SCI_OK) rc = sci_cuda_check(ctx, cudaMalloc(&cnt, 16), "range pair count");
    if (rc == SCI_OK) {
        cudaStream_t st = ctx->stream;
        cudaMemsetAsync(cnt, 0, 16, st);
        if (ctx->r2 > 0)
            k_range_count2<<<grid_for(ctx->r2), 256, 0, st>>>(ctx->r2_idx, ctx->r2_code, ctx->r2_pos, ctx->r2,
                                                              row_begin, row_end, cnt);
        if (ctx->r1 > 0)
            k_range_count1<<<grid_for(ctx->r1), 256, 0, st>>>(ctx->r1_idx, ctx->r1_meta, ctx->r1, row_begin, row_end,
                                                              cnt + 1);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        rc = sci_cuda_check(ctx, e, "range pair count");
    }
    if (cnt) cudaFree(cnt);
    // the tiled prefix of the range tables (a subset of the full tables' buckets, in their
    // order, so the buckets left to the window kernels fit as they do there)
    if (rc == SCI_OK) rc = sci_table_split(ctx, true);
    if (rc != SCI_OK) {
        ctx->range_bytes = 0;  // not yet counted in bytes_held
        sci_free_range(ctx);
        return rc;
    }
    ctx->bytes_held += ctx->range_bytes;
    ctx->range_pairs = (int64_t)(h[0] + h[1]);
    ctx->range_pairs2 = (int64_t)h[0];
    ctx->range_pairs1 = (int64_t)h[1];
    ctx->row_b = row_begin;
    ctx->row_e = row_end;
    ctx->ranged = 1;
    return SCI_OK;
}

extern "C" int sci_row_costs(sci_ctx *ctx, int64_t *cost)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "no determinants");
    if (ctx->M == 0) return SCI_OK;
    if (!cost) return sci_fail(ctx, SCI_ERR_ARG, "cost is NULL");
    SCI_CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    unsigned long long *c = reinterpret_cast<unsigned long long *>(cost);
    SCI_CK(cudaMemsetAsync(c, 0, (size_t)ctx->M * 8, st));
    if (ctx->e2 > 0) k_cost2<<<grid_for(ctx->e2), 256, 0, st>>>(ctx->e2_idx, ctx->e2_code, ctx->e2_pos, ctx->e2, c);
    if (ctx->e1 > 0) k_cost1<<<grid_for(ctx->e1), 256, 0, st>>>(ctx->e1_idx, ctx->e1_meta, ctx->e1, c);
    return sci_cuda_check(ctx, cudaGetLastError(), "row cost kernels");
}
