// sci_connections_noalloc: the connection export of sci_connections() for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc or cudaFree.  A process whose device memory is
// handed out by a pooling allocator (a framework's caching allocator, or a fixed arena
// sized to the card) has nothing left for the driver, so a late cudaMalloc fails or
// fragments the pool.  And cudaFree synchronises the whole device, which stalls every
// other stream of a caller that keeps several streams busy.  sci_connections() allocates
// a counter and a tuple buffer per call; this variant uses a fixed scratch array in the
// library's own device memory instead, and sorts on the host in the caller's arrays.
//
// Scratch: g_noalloc_scratch, a file-scope device array of kNoAllocBytes bytes: a 256-byte
// header whose first 8 bytes are the slot counter, then kNoAllocMaxPairs packed (I, J)
// pairs (uint64) and as many flag bytes.  Every call shares it and it keeps the last
// call's contents; the counter is cleared at the start of each call.  Calls that overlap
// on the GPU (two host threads, or two streams) race on it.
//
// When the scratch is committed.  The library is compiled per translation unit, so this
// file's device code (the array and the two kernels) is a module of its own, and the CUDA
// runtime loads modules lazily: the driver reserves the array's device memory only when
// the module is first touched.  A caller that cannot allocate must not meet that moment in
// the middle of its run, so sci_create() calls sci_noalloc_prepare(), which touches the
// module on the context's device (the array's address and both kernels' attributes).
// From the first sci_create() on a device until the process exits, that device holds the
// array; a later sci_connections_noalloc() call only reads the cached address.
#include <mutex>

#include "sci_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxPairs = SCI_NOALLOC_MAX_PAIRS;
constexpr size_t kHeader = 256;
constexpr size_t kNoAllocBytes = kHeader + (size_t)kNoAllocMaxPairs * 9;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

struct Scratch {
    unsigned long long *counter;
    uint64_t *pairs;   // (I << 32) | J
    uint8_t *flags;    // bit 0: degree 2; bit 1: phase -1
    int64_t cap;
};

Scratch carve(void *base)
{
    unsigned char *b = static_cast<unsigned char *>(base);
    Scratch s;
    s.counter = reinterpret_cast<unsigned long long *>(b);
    s.pairs = reinterpret_cast<uint64_t *>(b + kHeader);
    s.flags = b + kHeader + (size_t)kNoAllocMaxPairs * 8;
    s.cap = kNoAllocMaxPairs;
    return s;
}

__device__ __forceinline__ void put(Scratch s, uint32_t I, uint32_t J, int deg2, int neg)
{
    unsigned long long slot = atomicAdd(s.counter, 1ull);
    if ((int64_t)slot < s.cap) {
        s.pairs[slot] = ((uint64_t)I << 32) | J;
        s.flags[slot] = (uint8_t)(deg2 | (neg << 1));
    }
}

__global__ void k_conn2_noalloc(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
                                const uint32_t *__restrict__ e_pos, int64_t E, int64_t rb, int64_t re, Scratch s)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t I = e_idx[p];
        if (I < rb || I >= re) continue;
        const uint32_t pos = e_pos[p], code = e_code[p];
        int64_t bs = p - sci::pos_off(pos), be = bs + sci::pos_size(pos);
        int par = sci::code_par(code);
        for (int64_t q = bs; q < be; q++) {
            const uint32_t cq = e_code[q];
            if (sci::codes_overlap(cq, code)) continue;
            put(s, (uint32_t)I, e_idx[q], 1, par ^ (int)sci::code_par(cq));
        }
    }
}

__global__ void k_conn1_noalloc(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_meta, int64_t E,
                                int64_t rb, int64_t re, Scratch s)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t I = e_idx[p];
        if (I < rb || I >= re) continue;
        uint32_t meta = e_meta[p];
        int64_t bs = p - (int64_t)sci::meta_off(meta), be = bs + (int64_t)sci::meta_size(meta);
        int par = sci::meta_par(meta);
        for (int64_t q = bs; q < be; q++) {
            if (q == p) continue;
            put(s, (uint32_t)I, e_idx[q], 0, par ^ (int)sci::meta_par(e_meta[q]));
        }
    }
}

int grid_for(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// in-place heap sort of the parallel output arrays by (rows, J); no allocation
struct Out {
    int64_t *rows, *J;
    int8_t *deg, *ph;
    bool less(int64_t a, int64_t b) const { return rows[a] != rows[b] ? rows[a] < rows[b] : J[a] < J[b]; }
    void swap(int64_t a, int64_t b) const
    {
        int64_t t = rows[a]; rows[a] = rows[b]; rows[b] = t;
        t = J[a]; J[a] = J[b]; J[b] = t;
        if (deg) { int8_t u = deg[a]; deg[a] = deg[b]; deg[b] = u; }
        if (ph) { int8_t u = ph[a]; ph[a] = ph[b]; ph[b] = u; }
    }
    void sift(int64_t root, int64_t n) const
    {
        for (;;) {
            int64_t c = 2 * root + 1;
            if (c >= n) return;
            if (c + 1 < n && less(c, c + 1)) c++;
            if (!less(root, c)) return;
            swap(root, c);
            root = c;
        }
    }
    void sort(int64_t n) const
    {
        for (int64_t i = n / 2 - 1; i >= 0; i--) sift(i, n);
        for (int64_t e = n - 1; e > 0; e--) {
            swap(0, e);
            sift(0, e);
        }
    }
};

}  // namespace

// Once per device, with that device current: load this file's module (which commits the
// scratch array) and cache the array's device address.  Called by sci_create(); later
// calls on the same device return at once.
cudaError_t sci_noalloc_prepare(int device)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[device]) return cudaSuccess;
    void *addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_conn2_noalloc);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_conn1_noalloc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    g_scratch_addr[device] = addr;
    return cudaSuccess;
}

extern "C" int sci_connections_noalloc(sci_ctx *ctx, int64_t row_begin, int64_t row_end, int64_t *count,
                                       int64_t *rows, int64_t *J, int8_t *degree, int8_t *phase, int64_t cap)
{
    if (!ctx || !count) return SCI_ERR_ARG;
    if (!ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "no determinants");
    if (row_begin < 0 || row_end > ctx->M || row_begin > row_end || cap < 0)
        return sci_fail(ctx, SCI_ERR_ARG, "bad row range or capacity");
    if (cap > 0 && (!rows || !J)) return sci_fail(ctx, SCI_ERR_ARG, "rows and J are required (sorted in place)");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return sci_cuda_check(ctx, e, "cudaSetDevice");
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return sci_fail(ctx, SCI_ERR_ARG, "device index too large");

    // the scratch array's address, looked up by sci_create() on this device (a context
    // made by sci_create() always has it; the lookup here only repeats a failed one)
    e = sci_noalloc_prepare(ctx->device);
    if (e != cudaSuccess) return sci_cuda_check(ctx, e, "no-allocation scratch set-up");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        base = g_scratch_addr[ctx->device];
    }
    Scratch s = carve(base);
    cudaStream_t st = ctx->stream;
    e = cudaMemsetAsync(s.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return sci_cuda_check(ctx, e, "clear scratch counter");
    if (ctx->e2 > 0)
        k_conn2_noalloc<<<grid_for(ctx->e2), 256, 0, st>>>(ctx->e2_idx, ctx->e2_code, ctx->e2_pos, ctx->e2,
                                                           row_begin, row_end, s);
    if (ctx->e1 > 0)
        k_conn1_noalloc<<<grid_for(ctx->e1), 256, 0, st>>>(ctx->e1_idx, ctx->e1_meta, ctx->e1, row_begin, row_end, s);
    unsigned long long n = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, s.counter, sizeof(n), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return sci_cuda_check(ctx, e, "connection export");
    *count = (int64_t)n;
    if ((int64_t)n > kNoAllocMaxPairs)
        return sci_fail(ctx, SCI_ERR_OVERFLOW,
                        "more connections in the row range than the no-allocation scratch holds "
                        "(SCI_NOALLOC_MAX_PAIRS); split the range");
    if ((int64_t)n > cap) return sci_fail(ctx, SCI_ERR_OVERFLOW, "connection list exceeds cap");
    if (n == 0) return SCI_OK;
    // packed pairs into J, flag bytes into the front of rows, then unpack backwards so
    // that no flag byte is overwritten before it is read
    e = cudaMemcpyAsync(J, s.pairs, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rows, s.flags, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return sci_cuda_check(ctx, e, "copy connection list");
    const uint8_t *fl = reinterpret_cast<const uint8_t *>(rows);
    for (int64_t t = (int64_t)n - 1; t >= 0; t--) {
        uint8_t f = fl[t];
        uint64_t v = (uint64_t)J[t];
        if (degree) degree[t] = (f & 1) ? 2 : 1;
        if (phase) phase[t] = (f & 2) ? -1 : 1;
        J[t] = (int64_t)(v & 0xFFFFFFFFull);
        rows[t] = (int64_t)(v >> 32);
    }
    Out{rows, J, degree, phase}.sort((int64_t)n);
    return SCI_OK;
}
