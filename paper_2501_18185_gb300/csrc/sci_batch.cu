// Batched sigma over heterogeneous instances in one persistent launch.
//
// Many small Hamiltonians (each a sci_ctx with its own integrals and determinant list,
// real spin-orbital mode) are applied to their vectors by ONE kernel launch: the work of
// every instance is cut into items, and persistent CTAs (one wave over the GPU) take
// items from a global counter until the list is exhausted.  This is the GPU counterpart
// of the paper's dynamic task scheduling (Sec. 3.1: OpenMP schedule(dynamic, 1) over
// tasks, MPI chunks handed to idle workers).  The launch (a counter reset, a clear of
// sigma and the kernel) can be captured once in a CUDA graph and replayed.
//
// Two schedules, chosen per instance by the autotuner in sci_batch_plan():
//   TILE  the bucket walk of the single-instance kernels: items are windows of whole
//         (N-2)-hole buckets, chunks of (N-1)-table entries and chunks of diagonal rows;
//         results go to sigma by FP64 atomic adds.  Works for any determinant list.
//   WARP  warp per determinant, for full-CI instances: a warp enumerates all single and
//         double excitations of its row I, finds the index of each J by ranking its alpha
//         and beta strings in the combinatorial number system (the FCI list sorted as
//         uint64 is ordered by (beta rank, alpha rank)), evaluates H_IJ from the same
//         tables (pair table, reference Fock matrix and g_so corrections), reduces over
//         the warp and stores sigma_I: no atomics, no bucket tables read.
// Items are ordered by decreasing measured cost so that the tail of the wave is short.
// A per-instance flag array (sci_batch_set_active) lets a caller drop instances from
// later launches and graph replays: their items are taken from the counter and skipped.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "sci_bits.cuh"
#include "sci_bucket.cuh"
#include "sci_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCH = 512;          // table rows per TILE doubles window
constexpr int kSinglesChunk = kThreads;
constexpr int kDiagChunk = 4096;

enum ItemType : int { IT_DIAG = 0, IT_DOUBLES = 1, IT_SINGLES = 2, IT_WARP = 3 };

struct Inst {
    int64_t M, off;
    int n, norb, na, nb;
    uint64_t ref;
    int64_t nA;  // alpha strings of the FCI space (WARP)
    const uint64_t *keys;
    const double *hdiag, *tab, *fref, *g_so;
    const uint32_t *e2_idx, *e2_code, *e2_pos;
    int64_t e2;
    const uint32_t *e1_idx;
    const uint64_t *e1_S;
    const uint32_t *e1_meta;
    int64_t e1;
};

struct Item {
    int inst, type;
    int64_t a;
};

using sci::below;
using sci::kMaxPairs;
using sci::sflip;

// ---------------------------------------------------------------- TILE items
__device__ void tile_diag(const Inst &B, int64_t a, const double *C, double *S)
{
    const int64_t r0 = a * kDiagChunk, r1 = min(B.M, r0 + kDiagChunk);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) atomicAdd(S + B.off + r, B.hdiag[r] * C[B.off + r]);
}

__device__ void tile_doubles(const Inst &B, int64_t b, const double *C, double *S, unsigned char *smem)
{
    int64_t r0, r1;
    sci::window_of(B.e2_pos, B.e2, kCH, b, r0, r1);
    if (r0 >= r1) return;
    const int W = (int)(r1 - r0);
    double *s_c = reinterpret_cast<double *>(smem);
    uint2 *s_kc = reinterpret_cast<uint2 *>(smem + (size_t)W * sizeof(double));
    const sci::TabRule tr{0, B.n};
    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        const uint32_t code = B.e2_code[r0 + q];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        s_kc[q] = make_uint2(sci::col_code(code), colbase);
        s_c[q] = sflip(sci::code_par(code), C[B.off + B.e2_idx[r0 + q]]);
    }
    __syncthreads();
    for (int q0 = threadIdx.x; q0 < W; q0 += blockDim.x) {
        const uint32_t code = B.e2_code[r0 + q0], pos = B.e2_pos[r0 + q0];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        // the members other than the row itself (bucket position j + (j >= q0)): no FP64
        // instruction is issued for the row, and rows of one bucket size run equal counts
        const int bs = q0 - sci::pos_off(pos), je = bs + sci::pos_size(pos) - 1;
        const uint32_t rc = sci::row_code(code);
        const double *trow = B.tab + rowoff;
        double acc = 0.0;
        for (int j = bs; j < je; j++) {
            const int m = j + (j >= q0);
            const uint2 kc = s_kc[m];
            if (sci::disjoint(rc, kc.x)) acc = fma(__ldg(trow + kc.y), s_c[m], acc);
        }
        if (acc != 0.0) atomicAdd(S + B.off + B.e2_idx[r0 + q0], sflip(sci::code_par(code), acc));
    }
}

__device__ void tile_singles(const Inst &B, int64_t a, const double *C, double *S)
{
    const int64_t p = a * kSinglesChunk + threadIdx.x;
    if (p >= B.e1) return;
    const int norb = B.norb;
    const uint32_t meta = B.e1_meta[p];
    const int x = sci::meta_x(meta);
    const bool par = sci::meta_par(meta);
    const int64_t bs = p - (int64_t)sci::meta_off(meta), be = bs + (int64_t)sci::meta_size(meta);
    const uint64_t Sk = B.e1_S[p], part = Sk & ~B.ref, holes = B.ref & ~Sk;
    double acc = 0.0;
    for (int64_t q = bs; q < be; q++) {
        if (q == p) continue;
        const uint32_t mq = B.e1_meta[q];
        const int y = sci::meta_x(mq);
        double f = __ldg(B.fref + y * norb + x);
        for (uint64_t m = part; m; m &= m - 1) f += __ldg(B.g_so + ((int64_t)(__ffsll((long long)m) - 1) * norb + y) * norb + x);
        for (uint64_t m = holes; m; m &= m - 1) f -= __ldg(B.g_so + ((int64_t)(__ffsll((long long)m) - 1) * norb + y) * norb + x);
        acc = fma(f, sflip(sci::meta_par(mq), C[B.off + B.e1_idx[q]]), acc);
    }
    atomicAdd(S + B.off + B.e1_idx[p], sflip(par, acc));
}

// ---------------------------------------------------------------- WARP items
// The rank of a string in the combinatorial number system, sum_m C(p_m, m) over its set
// bits p_1 < p_2 < ... (m from 1), is its position among the strings of equal popcount in
// ascending numeric order, whatever the orbital count: one table of 2^kRankBits ranks
// serves every instance with up to kRankBits orbitals.
constexpr int kRankBits = 20;

__global__ void k_rank_table(uint32_t *rank)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < (1ll << kRankBits);
         s += (int64_t)gridDim.x * blockDim.x) {
        uint64_t r = 0;
        int m = 1;
        for (uint32_t x = (uint32_t)s; x; x &= x - 1, m++) {
            const int p = __ffs((int)x) - 1;  // C(p, m)
            uint64_t c = m <= p ? 1 : 0;
            for (int k = 1; k <= m && m <= p; k++) c = c * (uint64_t)(p - m + k) / (uint64_t)k;
            r += c;
        }
        rank[s] = (uint32_t)r;
    }
}


__device__ __forceinline__ int64_t fci_index(const Inst &B, uint64_t J, const uint32_t *__restrict__ rank)
{
    const uint32_t ja = (uint32_t)(J & ((1ull << B.n) - 1)), jb = (uint32_t)(J >> B.n);
    return (int64_t)__ldg(rank + jb) * B.nA + __ldg(rank + ja);
}

// H_IJ c_J for the double excitation I -> J with bra extras x < y (in I) and ket extras
// u < v (in J), spin-orbital indices
__device__ __forceinline__ double warp_double(const Inst &B, uint64_t key, int x, int y, int u, int v, const double *C,
                                              const uint32_t *__restrict__ rank)
{
    const uint64_t K = key & ~(1ull << x) & ~(1ull << y);
    const uint64_t J = K | (1ull << u) | (1ull << v);
    uint32_t rowoff, colbase, r2, cb2;
    const sci::TabRule tr{0, B.n};
    sci::pair_offsets(tr, x, y, rowoff, r2);
    sci::pair_offsets(tr, u, v, cb2, colbase);
    const bool ph = (below(K, x) + below(K, y) + below(K, u) + below(K, v)) & 1;
    return sflip(ph, __ldg(B.tab + rowoff + colbase) * C[B.off + fci_index(B, J, rank)]);
}

__device__ __forceinline__ double warp_single(const Inst &B, uint64_t key, int x, int u, const double *C,
                                              const uint32_t *__restrict__ rank)
{
    const uint64_t Sk = key & ~(1ull << x);
    const uint64_t J = Sk | (1ull << u);
    const int norb = B.norb;
    double f = __ldg(B.fref + u * norb + x);
    const uint64_t part = Sk & ~B.ref, holes = B.ref & ~Sk;
    for (uint64_t m = part; m; m &= m - 1) f += __ldg(B.g_so + ((int64_t)(__ffsll((long long)m) - 1) * norb + u) * norb + x);
    for (uint64_t m = holes; m; m &= m - 1) f -= __ldg(B.g_so + ((int64_t)(__ffsll((long long)m) - 1) * norb + u) * norb + x);
    const bool ph = (below(Sk, x) + below(Sk, u)) & 1;
    return sflip(ph, f * C[B.off + fci_index(B, J, rank)]);
}

// orb: this warp's lists [occupied alpha | virtual alpha | occupied beta | virtual beta]
// x 32 spin-orbital indices; pairs[P] = a | b << 8 with P = b(b-1)/2 + a, a < b
__device__ void warp_rows(const Inst &B, int64_t a, const double *C, double *S, const uint32_t *__restrict__ rank,
                          const uint16_t *pairs, uint8_t *orb)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = a * kWarps + warp;
    if (r >= B.M) return;
    const int n = B.n;
    const uint64_t key = B.keys[r];
    const uint32_t full = (uint32_t)((1ull << n) - 1);
    const uint32_t oa = (uint32_t)(key & full), ob = (uint32_t)(key >> n);
    const uint32_t va = full & ~oa, vb = full & ~ob;
    if (lane < n) {
        const uint32_t lm = (1u << lane) - 1;
        if ((oa >> lane) & 1) orb[__popc(oa & lm)] = (uint8_t)lane;
        else orb[32 + __popc(va & lm)] = (uint8_t)lane;
        if ((ob >> lane) & 1) orb[64 + __popc(ob & lm)] = (uint8_t)(n + lane);
        else orb[96 + __popc(vb & lm)] = (uint8_t)(n + lane);
    }
    __syncwarp();
    const int na = B.na, nb = B.nb, ua = n - na, ub = n - nb;
    // candidate classes: alpha singles, beta singles, alpha-alpha, beta-beta, alpha-beta
    const int c0 = na * ua, c1 = nb * ub;
    const int qa = ua * (ua - 1) / 2, qb = ub * (ub - 1) / 2;
    const int c2 = na * (na - 1) / 2 * qa, c3 = nb * (nb - 1) / 2 * qb;
    const int T = c0 + c1 + c2 + c3 + c0 * c1;
    double acc = 0.0;
    for (int t = lane; t < T; t += 32) {
        int s = t;
        if (s < c0) {                       // alpha single x -> u
            acc += warp_single(B, key, orb[s / ua], orb[32 + s % ua], C, rank);
            continue;
        }
        s -= c0;
        if (s < c1) {                       // beta single
            acc += warp_single(B, key, orb[64 + s / ub], orb[96 + s % ub], C, rank);
            continue;
        }
        s -= c1;
        if (s < c2 + c3) {                  // same-spin double
            const bool beta = s >= c2;
            if (beta) s -= c2;
            const int q = beta ? qb : qa;
            const uint8_t *occ = orb + (beta ? 64 : 0), *vir = orb + (beta ? 96 : 32);
            const uint16_t po = pairs[s / q], pv = pairs[s % q];
            acc += warp_double(B, key, occ[po & 0xFF], occ[po >> 8], vir[pv & 0xFF], vir[pv >> 8], C, rank);
            continue;
        }
        s -= c2 + c3;                       // alpha-beta double
        const int sa = s / c1, sb = s % c1;
        acc += warp_double(B, key, orb[sa / ua], orb[64 + sb / ub], orb[32 + sa % ua], orb[96 + sb % ub], C, rank);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) S[B.off + r] = fma(B.hdiag[r], C[B.off + r], acc);
}

// ---------------------------------------------------------------- the persistent kernel
__global__ void __launch_bounds__(kThreads)
k_batch(const Inst *__restrict__ insts, const Item *__restrict__ items, int nitems, int *counter,
        const double *__restrict__ C, double *__restrict__ S, const uint32_t *__restrict__ rank,
        const int *__restrict__ active)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint16_t pairs[kMaxPairs];
    __shared__ uint8_t orb[kWarps * 128];
    __shared__ int s_item;
    sci::fill_pair_table(pairs);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const Item I = items[it];
        if (!active[I.inst]) continue;   // the same for every thread of the CTA
        const Inst &B = insts[I.inst];
        switch (I.type) {
            case IT_DIAG: tile_diag(B, I.a, C, S); break;
            case IT_DOUBLES: tile_doubles(B, I.a, C, S, smem); break;
            case IT_SINGLES: tile_singles(B, I.a, C, S); break;
            default: warp_rows(B, I.a, C, S, rank, pairs, orb + (threadIdx.x >> 5) * 128); break;
        }
    }
}

int64_t binom_host(int a, int b)
{
    if (b < 0 || b > a) return 0;
    int64_t v = 1;
    for (int k = 1; k <= b; k++) v = v * (a - b + k) / k;
    return v;
}

}  // namespace

struct sci_batch {
    int device = 0;
    cudaStream_t user = nullptr;   // caller's stream
    cudaStream_t stream = nullptr; // own stream (graph capture needs a non-legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
    std::string err;
    std::vector<sci_ctx *> ctxs;
    std::vector<Inst> host;
    std::vector<int> sched;         // per instance: SCI_SCHED_TILE or SCI_SCHED_WARP
    std::vector<float> ms_tile, ms_warp;
    struct Tuned {
        int sched;
        float ms_tile, ms_warp;
    };
    std::map<std::tuple<int, int, int, int64_t>, Tuned> cache;  // autotuner decisions by shape
    Inst *d_inst = nullptr;
    Item *d_items = nullptr;
    int nitems = 0, items_cap = 0;
    int *d_counter = nullptr;
    uint32_t *d_rank = nullptr;  // combinatorial ranks of all strings of kRankBits bits
    int *d_active = nullptr;     // per instance: nonzero = computed
    int active_n = 0;
    std::vector<int> h_active;
    size_t smem = 0;
    int grid = 0;
    int64_t total_M = 0, total_pairs = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int bfail(sci_batch *b, int code, const std::string &m)
{
    b->err = m;
    return code;
}

#define BCK(x)                                                                 \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess) return bfail(b, SCI_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

// WARP needs a full-CI list (so that J is found by ranking) of at most kRankBits orbitals
bool warp_ok(const sci_ctx *c)
{
    return c->n <= kRankBits && binom_host(c->n, c->na) * binom_host(c->n, c->nb) == c->M;
}

// the items of one instance under one schedule, with a cost estimate per item
void items_of(const sci_batch *b, int i, int sched, std::vector<Item> &out)
{
    const Inst &B = b->host[i];
    if (sched == SCI_SCHED_WARP) {
        for (int64_t a = 0; a * kWarps < B.M; a++) out.push_back(Item{i, IT_WARP, a});
        return;
    }
    for (int64_t a = 0; a * kCH < B.e2; a++) out.push_back(Item{i, IT_DOUBLES, a});
    for (int64_t a = 0; a * kSinglesChunk < B.e1; a++) out.push_back(Item{i, IT_SINGLES, a});
    for (int64_t a = 0; a * kDiagChunk < B.M; a++) out.push_back(Item{i, IT_DIAG, a});
}

int upload_items(sci_batch *b, const std::vector<Item> &items)
{
    if ((int)items.size() > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        BCK(cudaMalloc(&b->d_items, sizeof(Item) * std::max<size_t>(1, items.size())));
        b->items_cap = (int)items.size();
    }
    if (!items.empty())
        BCK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    b->nitems = (int)items.size();
    return SCI_OK;
}

int launch(sci_batch *b, const double *C, double *S)
{
    if (!b->d_active || b->active_n != (int)b->host.size()) return bfail(b, SCI_ERR_STATE, "batch launch: no complete plan");
    BCK(cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream));
    if (b->total_M > 0) BCK(cudaMemsetAsync(S, 0, sizeof(double) * b->total_M, b->stream));
    k_batch<<<b->grid, kThreads, b->smem, b->stream>>>(b->d_inst, b->d_items, b->nitems, b->d_counter, C, S, b->d_rank,
                                                        b->d_active);
    BCK(cudaGetLastError());
    return SCI_OK;
}

}  // namespace

extern "C" int sci_batch_create(sci_batch **out, int device, void *cuda_stream)
{
    if (!out) return SCI_ERR_ARG;
    *out = nullptr;
    auto *b = new sci_batch();
    b->device = device;
    b->user = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess || cudaEventCreate(&b->t0) != cudaSuccess ||
        cudaEventCreate(&b->t1) != cudaSuccess || cudaMalloc(&b->d_counter, sizeof(int)) != cudaSuccess) {
        sci_batch_destroy(b);
        return SCI_ERR_CUDA;
    }
    *out = b;
    return SCI_OK;
}

extern "C" int sci_batch_destroy(sci_batch *b)
{
    if (!b) return SCI_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_rank) cudaFree(b->d_rank);
    if (b->d_active) cudaFree(b->d_active);
    for (cudaEvent_t e : {b->ev_in, b->ev_out, b->t0, b->t1})
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return SCI_OK;
}

extern "C" int sci_batch_add(sci_batch *b, sci_ctx *ctx)
{
    if (!b || !ctx) return SCI_ERR_ARG;
    if (!ctx->have_ints || !ctx->have_dets) return bfail(b, SCI_ERR_STATE, "batch_add: instance needs integrals and determinants");
    if (ctx->cplx || ctx->spinors) return bfail(b, SCI_ERR_ARG, "batch_add: real spin-orbital instances only");
    if (ctx->nwords != 1) return bfail(b, SCI_ERR_ARG, "batch_add: one-word keys only");
    if (ctx->device != b->device) return bfail(b, SCI_ERR_ARG, "batch_add: instance on another device");
    Inst B{};
    B.M = ctx->M;
    B.off = b->total_M;
    B.n = ctx->n, B.norb = ctx->norb, B.na = ctx->na, B.nb = ctx->nb;
    B.ref = ctx->ref;
    B.nA = binom_host(ctx->n, ctx->na);
    B.keys = ctx->keys;
    B.hdiag = ctx->hdiag;
    B.tab = static_cast<const double *>(ctx->tab);
    B.fref = static_cast<const double *>(ctx->fref);
    B.g_so = static_cast<const double *>(ctx->g_so);
    B.e2_idx = ctx->e2_idx, B.e2_code = ctx->e2_code, B.e2_pos = ctx->e2_pos, B.e2 = ctx->e2;
    B.e1_idx = ctx->e1_idx, B.e1_S = ctx->e1_S, B.e1_meta = ctx->e1_meta, B.e1 = ctx->e1;
    b->ctxs.push_back(ctx);
    b->host.push_back(B);
    b->sched.push_back(SCI_SCHED_TILE);
    b->ms_tile.push_back(-1.f);
    b->ms_warp.push_back(-1.f);
    b->total_M += ctx->M;
    b->total_pairs += ctx->pairs;
    return (int)b->host.size() - 1;
}

extern "C" int sci_batch_plan(sci_batch *b, int schedule, const double *C, double *S)
{
    if (!b) return SCI_ERR_ARG;
    if (schedule != SCI_SCHED_AUTO && schedule != SCI_SCHED_TILE && schedule != SCI_SCHED_WARP)
        return bfail(b, SCI_ERR_ARG, "batch_plan: schedule must be AUTO, TILE or WARP");
    if (schedule == SCI_SCHED_AUTO && b->total_M > 0 && (!C || !S))
        return bfail(b, SCI_ERR_ARG, "batch_plan: AUTO times the schedules on C -> S");
    BCK(cudaSetDevice(b->device));
    const int ni = (int)b->host.size();
    if (b->d_inst) cudaFree(b->d_inst);
    b->d_inst = nullptr;
    BCK(cudaMalloc(&b->d_inst, sizeof(Inst) * std::max(1, ni)));
    if (ni) BCK(cudaMemcpy(b->d_inst, b->host.data(), sizeof(Inst) * ni, cudaMemcpyHostToDevice));
    BCK(cudaStreamSynchronize(b->stream));
    if (b->active_n != ni) {
        if (b->d_active) cudaFree(b->d_active);
        b->d_active = nullptr;
        b->active_n = 0;
        BCK(cudaMalloc(&b->d_active, sizeof(int) * std::max(1, ni)));
        b->active_n = ni;
    }
    b->h_active.assign(std::max(1, ni), 1);
    BCK(cudaMemcpy(b->d_active, b->h_active.data(), sizeof(int) * std::max(1, ni), cudaMemcpyHostToDevice));
    if (!b->d_rank) {
        BCK(cudaMalloc(&b->d_rank, sizeof(uint32_t) << kRankBits));
        k_rank_table<<<1024, kThreads, 0, b->stream>>>(b->d_rank);
        BCK(cudaGetLastError());
        BCK(cudaStreamSynchronize(b->stream));
    }
    // shared memory for the largest TILE window; a grid of one wave
    int maxb = 1;
    for (auto *c : b->ctxs) maxb = std::max(maxb, c->maxb2);
    b->smem = (size_t)(kCH + maxb) * (sizeof(double) + sizeof(uint2));
    if (b->smem > 200 * 1024) return bfail(b, SCI_ERR_OVERFLOW, "batch_plan: largest bucket too large");
    if (b->smem > 48 * 1024) BCK(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    int per_sm = 0, sms = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, b->smem));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = std::max(1, per_sm) * sms;

    std::vector<float> cost(ni, 0.f);
    for (int i = 0; i < ni; i++) {
        const bool fci = warp_ok(b->ctxs[i]);
        if (schedule == SCI_SCHED_WARP && !fci)
            return bfail(b, SCI_ERR_ARG, "batch_plan: WARP needs full-CI instances of at most 20 orbitals");
        if (schedule != SCI_SCHED_AUTO) {
            b->sched[i] = schedule;
            continue;
        }
        const Inst &B = b->host[i];
        auto key = std::make_tuple(B.n, B.na, B.nb, B.M);
        auto hit = b->cache.find(key);
        if (hit != b->cache.end()) {
            b->sched[i] = hit->second.sched;
            b->ms_tile[i] = hit->second.ms_tile;
            b->ms_warp[i] = hit->second.ms_warp;
            continue;
        }
        // time each eligible schedule on this instance alone (one warm-up, three timed)
        float best = 1e30f;
        for (int s : {SCI_SCHED_TILE, SCI_SCHED_WARP}) {
            if (s == SCI_SCHED_WARP && !fci) continue;
            std::vector<Item> it;
            items_of(b, i, s, it);
            int rc = upload_items(b, it);
            if (rc) return rc;
            for (int rep = 0; rep < 4; rep++) {
                if (rep == 1) BCK(cudaEventRecord(b->t0, b->stream));
                BCK(cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream));
                BCK(cudaMemsetAsync(S + B.off, 0, sizeof(double) * B.M, b->stream));
                k_batch<<<b->grid, kThreads, b->smem, b->stream>>>(b->d_inst, b->d_items, b->nitems, b->d_counter, C, S,
                                                                    b->d_rank, b->d_active);
                BCK(cudaGetLastError());
            }
            BCK(cudaEventRecord(b->t1, b->stream));
            BCK(cudaEventSynchronize(b->t1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, b->t0, b->t1));
            ms /= 3.f;
            (s == SCI_SCHED_TILE ? b->ms_tile : b->ms_warp)[i] = ms;
            if (ms < best) best = ms, b->sched[i] = s;
        }
        b->cache[key] = sci_batch::Tuned{b->sched[i], b->ms_tile[i], b->ms_warp[i]};
    }
    // the full work list, costliest items first (cost: the instance's measured time, or
    // its pair count, spread over its items)
    std::vector<std::pair<float, Item>> all;
    for (int i = 0; i < ni; i++) {
        std::vector<Item> it;
        items_of(b, i, b->sched[i], it);
        float t = b->sched[i] == SCI_SCHED_WARP ? b->ms_warp[i] : b->ms_tile[i];
        if (t <= 0.f) t = 1e-9f * (float)(b->ctxs[i]->pairs + b->ctxs[i]->M);
        for (auto &x : it) all.push_back({t / (float)it.size(), x});
    }
    std::stable_sort(all.begin(), all.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<Item> items;
    items.reserve(all.size());
    for (auto &x : all) items.push_back(x.second);
    if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
    if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
    return upload_items(b, items);
}

extern "C" int sci_batch_sigma(sci_batch *b, const double *C, double *S)
{
    if (!b) return SCI_ERR_ARG;
    if (b->total_M > 0 && (!C || !S)) return bfail(b, SCI_ERR_ARG, "batch_sigma: C and S needed");
    if (!b->d_inst) return bfail(b, SCI_ERR_STATE, "batch_sigma: call sci_batch_plan first");
    BCK(cudaSetDevice(b->device));
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    int rc = launch(b, C, S);
    if (rc) return rc;
    BCK(cudaEventRecord(b->ev_out, b->stream));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return SCI_OK;
}

extern "C" int sci_batch_capture(sci_batch *b, const double *C, double *S)
{
    if (!b) return SCI_ERR_ARG;
    if (b->total_M > 0 && (!C || !S)) return bfail(b, SCI_ERR_ARG, "batch_capture: C and S needed");
    if (!b->d_inst) return bfail(b, SCI_ERR_STATE, "batch_capture: call sci_batch_plan first");
    BCK(cudaSetDevice(b->device));
    if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
    if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
    BCK(cudaStreamSynchronize(b->stream));
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch(b, C, S);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    BCK(e);
    b->graph = g;
    BCK(cudaGraphInstantiate(&b->exec, g, 0));
    return SCI_OK;
}

extern "C" int sci_batch_replay(sci_batch *b)
{
    if (!b) return SCI_ERR_ARG;
    if (!b->exec) return bfail(b, SCI_ERR_STATE, "batch_replay: nothing captured");
    BCK(cudaSetDevice(b->device));
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    BCK(cudaGraphLaunch(b->exec, b->stream));
    BCK(cudaEventRecord(b->ev_out, b->stream));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return SCI_OK;
}

extern "C" int sci_batch_set_active(sci_batch *b, const int32_t *active, int n)
{
    if (!b) return SCI_ERR_ARG;
    if (!b->d_active) return bfail(b, SCI_ERR_STATE, "batch_set_active: call sci_batch_plan first");
    if (!active || n != (int)b->host.size() || n != b->active_n) return bfail(b, SCI_ERR_ARG, "batch_set_active: one flag per instance");
    BCK(cudaSetDevice(b->device));
    for (int i = 0; i < n; i++) b->h_active[i] = active[i] != 0;
    // pageable source: the copy is staged before the call returns, so h_active may change after
    if (n) BCK(cudaMemcpyAsync(b->d_active, b->h_active.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->stream));
    return SCI_OK;
}

extern "C" int sci_batch_info(sci_batch *b, int i, int *schedule, float *ms_tile, float *ms_warp, int64_t *offset)
{
    if (!b || i < 0 || i >= (int)b->host.size()) return SCI_ERR_ARG;
    if (schedule) *schedule = b->sched[i];
    if (ms_tile) *ms_tile = b->ms_tile[i];
    if (ms_warp) *ms_warp = b->ms_warp[i];
    if (offset) *offset = b->host[i].off;
    return SCI_OK;
}

extern "C" int sci_batch_items(sci_batch *b, int64_t *out, int n)
{
    if (!b || !out || n < 1) return SCI_ERR_ARG;
    const int64_t v[4] = {b->nitems, b->grid, b->total_M, b->total_pairs};
    for (int k = 0; k < n && k < 4; k++) out[k] = v[k];
    return SCI_OK;
}

extern "C" const char *sci_batch_last_error(const sci_batch *b) { return b ? b->err.c_str() : "null batch"; }
