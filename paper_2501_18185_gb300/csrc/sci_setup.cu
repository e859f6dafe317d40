// libsci setup: context, integral tables and the determinant bucket tables.
//
// Everything here runs once per Hamiltonian or per determinant space (the paper's
// "classify and sort pairs" steps of the batch evaluation scheme, Sec. 2.3); the hot
// path sigma = H c lives in sci_sigma.cu.  The radix sorts and scans of the setup use
// CUB (header-only, part of the CUDA toolkit).
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sci_internal.cuh"

using sci::zdbl;

// ------------------------------------------------------------------ error helpers
int sci_fail(sci_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int sci_cuda_check(sci_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SCI_OK;
    cudaGetLastError();  // clear non-sticky errors
    int code = (e == cudaErrorMemoryAllocation) ? SCI_ERR_NOMEM : SCI_ERR_CUDA;
    return sci_fail(ctx, code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SCI_CK(call)                                                 \
    do {                                                             \
        int _rc = sci_cuda_check(ctx, (call), #call);                \
        if (_rc != SCI_OK) return _rc;                               \
    } while (0)

namespace {

// device buffer owned by a scope (temporaries of the setup)
struct TmpBuf {
    void *p = nullptr;
    ~TmpBuf() { if (p) cudaFree(p); }
    template <typename T> T *as() { return static_cast<T *>(p); }
};

cudaError_t alloc_held(sci_ctx *ctx, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) ctx->bytes_held += bytes;
    return e;
}

template <typename T> void free_held(sci_ctx *ctx, T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
    (void)ctx;
}


// ------------------------------------------------------------------ scalar helpers
template <typename S> struct Sc;
template <> struct Sc<double> {
    __device__ static double zero() { return 0.0; }
    __device__ static double mul(double a, double b) { return a * b; }
    __device__ static double add(double a, double b) { return a + b; }
    __device__ static double sub(double a, double b) { return a - b; }
    __device__ static double re(double a) { return a; }
};
template <> struct Sc<zdbl> {
    __device__ static zdbl zero() { return zdbl{0.0, 0.0}; }
    __device__ static zdbl mul(zdbl a, zdbl b) { return zdbl{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
    __device__ static zdbl add(zdbl a, zdbl b) { return zdbl{a.x + b.x, a.y + b.y}; }
    __device__ static zdbl sub(zdbl a, zdbl b) { return zdbl{a.x - b.x, a.y - b.y}; }
    __device__ static double re(zdbl a) { return a.x; }
};

// ------------------------------------------------------------------ integral kernels
// (pq|rs) = sum_P L^P_pq L^P_rs, dense n^4
template <typename S>
__global__ void k_eri_from_chol(const S *__restrict__ L, int naux, int n, S *__restrict__ eri)
{
    int64_t n2 = (int64_t)n * n;
    int64_t total = n2 * n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t pq = t / n2, rs = t % n2;
        S acc = Sc<S>::zero();
        for (int P = 0; P < naux; P++) acc = Sc<S>::add(acc, Sc<S>::mul(L[P * n2 + pq], L[P * n2 + rs]));
        eri[t] = acc;
    }
}

struct OrbMap {
    int n, spinors;
    __device__ int spin(int p) const { return spinors ? 0 : (p >= n); }
    __device__ int sp(int p) const { return spinors ? p : (p >= n ? p - n : p); }
};

// spin-orbital integral from the spatial (or spinor) table
template <typename S>
__device__ S eri_so(const S *__restrict__ eri, OrbMap m, int p, int q, int r, int s)
{
    if (m.spin(p) != m.spin(q) || m.spin(r) != m.spin(s)) return Sc<S>::zero();
    int64_t n = m.n;
    return eri[((m.sp(p) * n + m.sp(q)) * n + m.sp(r)) * n + m.sp(s)];
}

template <typename S>
__global__ void k_small_tables(const S *__restrict__ h, const S *__restrict__ eri, OrbMap m, int norb,
                               S *__restrict__ h_so, S *__restrict__ jd, S *__restrict__ kd,
                               S *__restrict__ g_so)
{
    int64_t total = (int64_t)norb * norb * norb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(t / ((int64_t)norb * norb));
        int i = (int)((t / norb) % norb);
        int a = (int)(t % norb);
        // g_so[k][i][a] = (ai|kk) - (ak|ki)
        g_so[t] = Sc<S>::sub(eri_so(eri, m, a, i, k, k), eri_so(eri, m, a, k, k, i));
        if (k == 0) {
            // [i][a] tables
            int64_t u = (int64_t)i * norb + a;
            h_so[u] = (m.spin(i) == m.spin(a)) ? h[(int64_t)m.sp(i) * m.n + m.sp(a)] : Sc<S>::zero();
            jd[u] = eri_so(eri, m, i, i, a, a);
            kd[u] = eri_so(eri, m, i, a, a, i);
        }
    }
}

// real spin-orbital pair table: T (n^4) then W (NP^2)
__global__ void k_tab_real(const double *__restrict__ eri, int n, double *__restrict__ tab)
{
    int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
    int64_t NP = (int64_t)n * (n - 1) / 2;
    int64_t total = n4 + NP * NP;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n4) {
            // t = ((y'*n + x')*n + y)*n + x  ->  (x x'|y y')
            int x = (int)(t % n), y = (int)((t / n) % n), xp = (int)((t / n2) % n), yp = (int)(t / (n2 * n));
            tab[t] = eri[((int64_t)(x * n + xp) * n + y) * n + yp];
        } else {
            int64_t u = t - n4;
            int64_t col = u / NP, row = u % NP;   // col = P(i,j), row = P(a,b)
            int b = (int)((1 + sqrt(1.0 + 8.0 * row)) / 2);
            while (b * (b - 1) / 2 > row) b--;
            while ((b + 1) * b / 2 <= row) b++;
            int a = (int)(row - (int64_t)b * (b - 1) / 2);
            int j = (int)((1 + sqrt(1.0 + 8.0 * col)) / 2);
            while (j * (j - 1) / 2 > col) j--;
            while ((j + 1) * j / 2 <= col) j++;
            int i = (int)(col - (int64_t)j * (j - 1) / 2);
            // (ai|bj) - (aj|bi)
            tab[t] = eri[((int64_t)(a * n + i) * n + b) * n + j] - eri[((int64_t)(a * n + j) * n + b) * n + i];
        }
    }
}

// spinor pair table: W (NP^2), complex
__global__ void k_tab_spinor(const zdbl *__restrict__ eri, int n, zdbl *__restrict__ tab)
{
    int64_t NP = (int64_t)n * (n - 1) / 2;
    int64_t total = NP * NP;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t col = t / NP, row = t % NP;
        int b = (int)((1 + sqrt(1.0 + 8.0 * row)) / 2);
        while (b * (b - 1) / 2 > row) b--;
        while ((b + 1) * b / 2 <= row) b++;
        int a = (int)(row - (int64_t)b * (b - 1) / 2);
        int j = (int)((1 + sqrt(1.0 + 8.0 * col)) / 2);
        while (j * (j - 1) / 2 > col) j--;
        while ((j + 1) * j / 2 <= col) j++;
        int i = (int)(col - (int64_t)j * (j - 1) / 2);
        zdbl u = eri[((int64_t)(a * n + i) * n + b) * n + j];
        zdbl v = eri[((int64_t)(a * n + j) * n + b) * n + i];
        tab[t] = zdbl{u.x - v.x, u.y - v.y};
    }
}

// split doubles into (hi, lo) float pairs: hi = fl32(x), lo = fl32(x - hi)
__global__ void k_split_ds(const double *__restrict__ in, float2 *__restrict__ out, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double x = in[t];
        float hi = (float)x;
        out[t] = make_float2(hi, (float)(x - (double)hi));
    }
}

__global__ void k_to_f32(const double *__restrict__ in, float *__restrict__ out, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (float)in[t];
}

// ------------------------------------------------------------------ determinant kernels
struct KeyRule {
    int spinors, n, na, nb, N;
};

// Keys of KW 64-bit words (up to 64 KW spin-orbitals or spinors, word 0 holding orbitals
// 0..63: the paper's orbital configurations as arrays of 64-bit integers, Sec. 3.2)
template <int KW> struct Kw {
    uint64_t w[KW];
};
template <int KW> __device__ __forceinline__ Kw<KW> load_kw(const uint64_t *keys, int64_t I)
{
    Kw<KW> k;
#pragma unroll
    for (int t = 0; t < KW; t++) k.w[t] = keys[I * KW + t];
    return k;
}
// occupied orbitals of the key below orbital p
template <int KW> __device__ __forceinline__ int below_w(const Kw<KW> &k, int p)
{
    int c = 0;
#pragma unroll
    for (int t = 0; t < KW; t++) {
        const int q = p - 64 * t;
        if (q <= 0) break;
        c += __popcll(q >= 64 ? k.w[t] : (k.w[t] & ((1ull << q) - 1ull)));
    }
    return c;
}
template <int KW> __device__ __forceinline__ int popc_w(const Kw<KW> &k)
{
    int c = 0;
#pragma unroll
    for (int t = 0; t < KW; t++) c += __popcll(k.w[t]);
    return c;
}
// calls f(p) for every occupied orbital p of the key, ascending
template <int KW, typename F> __device__ __forceinline__ void for_bits_w(const Kw<KW> &k, F f)
{
#pragma unroll
    for (int t = 0; t < KW; t++)
        for (uint64_t m = k.w[t]; m; m &= m - 1) f(64 * t + __ffsll((long long)m) - 1);
}
// -1, 0, +1 as unsigned (64 KW)-bit integers
template <int KW> __device__ __forceinline__ int cmp_w(const Kw<KW> &a, const Kw<KW> &b)
{
#pragma unroll
    for (int t = KW - 1; t >= 0; t--)
        if (a.w[t] != b.w[t]) return a.w[t] < b.w[t] ? -1 : 1;
    return 0;
}

template <int KW>
__global__ void k_validate(const uint64_t *__restrict__ keys, int64_t M, KeyRule r, int *status)
{
    const int nbits = r.spinors ? r.n : 2 * r.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const Kw<KW> k = load_kw<KW>(keys, i);
        const int tot = popc_w(k);
        int bad = 0;
        if (r.spinors) {
            if (tot != r.N) bad |= sci::DEV_POPCOUNT;
        } else {
            const int na = below_w(k, r.n);
            if (na != r.na || below_w(k, 2 * r.n) - na != r.nb) bad |= sci::DEV_POPCOUNT;
        }
        if (tot != below_w(k, nbits)) bad |= sci::DEV_POPCOUNT;   // bits above the orbitals
        if (i > 0) {
            const int c = cmp_w(load_kw<KW>(keys, i - 1), k);
            if (c == 0) bad |= sci::DEV_DUPLICATE;
            else if (c > 0) bad |= sci::DEV_UNSORTED;
        }
        if (bad) atomicOr(status, bad);
    }
}

// H_II = sum_{i in occ} h_ii + 1/2 sum_{i,j in occ} [(ii|jj) - (ij|ji)]
template <typename S, int KW>
__global__ void k_diag(const uint64_t *__restrict__ keys, int64_t M, int norb, const S *__restrict__ h_so,
                       const S *__restrict__ jd, const S *__restrict__ kd, double *__restrict__ hdiag)
{
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < M; I += (int64_t)gridDim.x * blockDim.x) {
        const Kw<KW> k = load_kw<KW>(keys, I);
        double e1 = 0.0, e2 = 0.0;
        for_bits_w(k, [&](int i) {
            e1 += Sc<S>::re(h_so[i * norb + i]);
            for_bits_w(k, [&](int j) { e2 += Sc<S>::re(jd[i * norb + j]) - Sc<S>::re(kd[i * norb + j]); });
        });
        hdiag[I] = e1 + 0.5 * e2;
    }
}

// fref[i][a] = h_ai + sum_{k in ref} g_so[k][i][a]
template <typename S>
__global__ void k_fref(int norb, Kw<sci::kMaxWords> ref, const S *__restrict__ h_so, const S *__restrict__ g_so,
                       S *__restrict__ fref)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= norb * norb) return;
    int i = t / norb, a = t % norb;
    S f = h_so[a * norb + i];
    for_bits_w(ref, [&](int k) { f = Sc<S>::add(f, g_so[((int64_t)k * norb + i) * norb + a]); });
    fref[t] = f;
}

// every determinant emits its keys with `holes` occupied bits removed (1 or 2): the key
// words (word w at out_w + w * stride) and the value I | x << 32 | y << 40
template <int KW>
__global__ void k_emit(const uint64_t *__restrict__ keys, int64_t M, int holes, int per_det, uint64_t *__restrict__ out_w,
                       int64_t stride, uint64_t *__restrict__ out_vals)
{
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < M; I += (int64_t)gridDim.x * blockDim.x) {
        const Kw<KW> k = load_kw<KW>(keys, I);
        const int64_t base = I * per_det;
        int t = 0;
        auto put = [&](Kw<KW> e, uint64_t v) {
#pragma unroll
            for (int w = 0; w < KW; w++) out_w[w * stride + base + t] = e.w[w];
            out_vals[base + t] = v;
            t++;
        };
        for_bits_w(k, [&](int x) {
            Kw<KW> e = k;
            e.w[x >> 6] &= ~(1ull << (x & 63));
            if (holes == 1) {
                put(e, (uint64_t)I | ((uint64_t)x << 32));
                return;
            }
            for_bits_w(k, [&](int y) {
                if (y <= x) return;
                Kw<KW> f = e;
                f.w[y >> 6] &= ~(1ull << (y & 63));
                put(f, (uint64_t)I | ((uint64_t)x << 32) | ((uint64_t)y << 40));
            });
        });
    }
}

__global__ void k_iota_u32(uint32_t *a, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        a[t] = (uint32_t)t;
}

__global__ void k_size_keys(const uint32_t *__restrict__ counts, int64_t n, uint16_t *__restrict__ sk,
                            unsigned long long *kept, int *maxb)
{
    unsigned long long k = 0;
    int mx = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c = counts[t];
        sk[t] = (uint16_t)(0xFFFFu - min(c, 0xFFFFu));
        k += (c >= 2);
        mx = max(mx, (int)min(c, 0x7FFFFFFFu));
    }
    for (int o = 16; o; o >>= 1) {
        k += __shfl_down_sync(0xffffffffu, k, o);
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (k) atomicAdd(kept, k);
        atomicMax(maxb, mx);
    }
}

__global__ void k_gather_sizes(const uint32_t *__restrict__ order, const uint32_t *__restrict__ counts, int64_t n,
                               uint32_t *__restrict__ out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = counts[order[t]];
}



// warp per kept bucket: scatter members into the final doubles table.  Members of a
// bucket arrive in ascending determinant order, i.e. ascending (y, x); a y-group is the
// run of members with the same y.
template <int KW>
__global__ void k_fill2(const uint32_t *__restrict__ order, const uint32_t *__restrict__ counts,
                        const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ newoff,
                        const uint64_t *__restrict__ ukeys, const uint64_t *__restrict__ vals, int64_t kept,
                        uint32_t *__restrict__ e_idx, uint32_t *__restrict__ e_code, uint32_t *__restrict__ e_pos)
{
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = w; j < kept; j += nw) {
        uint32_t b = order[j];
        uint32_t size = counts[b], old = offsets[b], dst = newoff[j];
        const Kw<KW> K = load_kw<KW>(ukeys, b);
        for (uint32_t t = lane; t < size; t += 32) {
            uint64_t v = vals[old + t];
            int x = (int)((v >> 32) & 0xFF), y = (int)((v >> 40) & 0xFF);
            uint32_t gs = t, ge = t + 1;
            while (gs > 0 && (int)((vals[old + gs - 1] >> 40) & 0xFF) == y) gs--;
            while (ge < size && (int)((vals[old + ge] >> 40) & 0xFF) == y) ge++;
            int par = (below_w(K, x) + below_w(K, y)) & 1;
            e_idx[dst + t] = (uint32_t)(v & 0xFFFFFFFFull);
            // the y-group fields saturate (63, 127): no kernel reads them past that
            e_code[dst + t] = sci::make_code(x, y, par, (int)min(t - gs, 63u), (int)min(ge - gs, 127u));
            e_pos[dst + t] = t | (size << 16);
        }
    }
}

template <int KW>
__global__ void k_fill1(const uint32_t *__restrict__ order, const uint32_t *__restrict__ counts,
                        const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ newoff,
                        const uint64_t *__restrict__ ukeys, const uint64_t *__restrict__ vals, int64_t kept,
                        uint32_t *__restrict__ e_idx, uint64_t *__restrict__ e_S, uint32_t *__restrict__ e_meta)
{
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = w; j < kept; j += nw) {
        uint32_t b = order[j];
        uint32_t size = counts[b], old = offsets[b], dst = newoff[j];
        const Kw<KW> K = load_kw<KW>(ukeys, b);
        for (uint32_t t = lane; t < size; t += 32) {
            uint64_t v = vals[old + t];
            int x = (int)((v >> 32) & 0xFF);
            uint32_t par = (uint32_t)(below_w(K, x) & 1);
            e_idx[dst + t] = (uint32_t)(v & 0xFFFFFFFFull);
#pragma unroll
            for (int w = 0; w < KW; w++) e_S[(int64_t)(dst + t) * KW + w] = K.w[w];
            e_meta[dst + t] = sci::make_meta(x, (int)par, (int)t, (int)size);
        }
    }
}

int grid_for(int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

// Sort the emitted (key, value) pairs, group equal keys, drop singletons and return the
// kept buckets ordered by size (largest first).
struct Buckets {
    TmpBuf ukeys, counts, offsets, order, newoff, vals_sorted;
    int64_t kept = 0, entries = 0;
    int maxb = 0;
};

int order_runs(sci_ctx *ctx, int nruns, Buckets &B);

__global__ void k_gather_u64(const uint64_t *__restrict__ src, const uint32_t *__restrict__ idx, int64_t n,
                             uint64_t *__restrict__ dst)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = src[idx[t]];
}

__global__ void k_compose(const uint32_t *__restrict__ p1, const uint32_t *__restrict__ p2, int64_t n,
                          uint32_t *__restrict__ out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = p1[p2[t]];
}

// run starts of the sorted keys: any of the KW words (planar, stride n) differs from the
// previous key's
__global__ void k_run_flags_w(const uint64_t *__restrict__ words, int kw, int64_t n, uint32_t *__restrict__ flag)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f = t == 0;
        for (int w = 0; w < kw && !f; w++) f = words[w * n + t] != words[w * n + t - 1];
        flag[t] = f;
    }
}

__global__ void k_runs_w(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ rid,
                         const uint64_t *__restrict__ words, int kw, int64_t n, uint64_t *__restrict__ ukeys,
                         uint32_t *__restrict__ start)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        if (flag[t]) {
            const uint32_t r = rid[t];
            start[r] = (uint32_t)t;
            for (int w = 0; w < kw; w++) ukeys[kw * (int64_t)r + w] = words[w * n + t];
        }
}

__global__ void k_run_counts(const uint32_t *__restrict__ start, int64_t nruns, int64_t n, uint32_t *__restrict__ counts)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nruns; r += (int64_t)gridDim.x * blockDim.x)
        counts[r] = (uint32_t)((r + 1 < nruns ? (int64_t)start[r + 1] : n) - start[r]);
}

// Keys of KW > 1 words: emit, sort as (64 KW)-bit integers by KW stable radix passes (word
// 0 first, each pass on the previous permutation's order of the next word), and find the
// runs of equal keys.  Produces B.vals_sorted, B.ukeys ([nruns][KW]) and B.counts.
template <int KW>
int sort_runs_w(sci_ctx *ctx, int holes, int per_det, int64_t total, Buckets &B, int &nruns)
{
    cudaStream_t st = ctx->stream;
    const int64_t M = ctx->M;
    const int nitems = (int)total;
    TmpBuf words, vals, perm, perm_new, iota, pass_perm, kg, ks, sorted, flag, rid, start, tmp;
    SCI_CK(cudaMalloc(&words.p, total * 8 * KW));     // planar: word w of entry t at w * total + t
    SCI_CK(cudaMalloc(&vals.p, total * 8));
    SCI_CK(cudaMalloc(&perm.p, total * 4));
    SCI_CK(cudaMalloc(&perm_new.p, total * 4));
    SCI_CK(cudaMalloc(&iota.p, total * 4));
    SCI_CK(cudaMalloc(&pass_perm.p, total * 4));
    SCI_CK(cudaMalloc(&kg.p, total * 8));
    SCI_CK(cudaMalloc(&ks.p, total * 8));
    SCI_CK(cudaMalloc(&B.vals_sorted.p, total * 8));
    uint64_t *W = words.as<uint64_t>();
    k_emit<KW><<<grid_for(M), 256, 0, st>>>(ctx->keys, M, holes, per_det, W, total, vals.as<uint64_t>());
    k_iota_u32<<<grid_for(total), 256, 0, st>>>(perm.as<uint32_t>(), total);
    k_iota_u32<<<grid_for(total), 256, 0, st>>>(iota.as<uint32_t>(), total);
    SCI_CK(cudaGetLastError());
    size_t tb = 0;
    SCI_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, kg.as<uint64_t>(), ks.as<uint64_t>(), iota.as<uint32_t>(),
                                           pass_perm.as<uint32_t>(), nitems, 0, 64, st));
    SCI_CK(cudaMalloc(&tmp.p, std::max<size_t>(tb, 16)));
    for (int w = 0; w < KW; w++) {
        const int bits = std::max(1, std::min(64, ctx->norb - 64 * w));
        // word w in the current order, sorted stably; the order composes
        k_gather_u64<<<grid_for(total), 256, 0, st>>>(W + w * total, perm.as<uint32_t>(), total, kg.as<uint64_t>());
        SCI_CK(cub::DeviceRadixSort::SortPairs(tmp.p, tb, kg.as<uint64_t>(), ks.as<uint64_t>(), iota.as<uint32_t>(),
                                               pass_perm.as<uint32_t>(), nitems, 0, bits, st));
        k_compose<<<grid_for(total), 256, 0, st>>>(perm.as<uint32_t>(), pass_perm.as<uint32_t>(), total,
                                                   perm_new.as<uint32_t>());
        std::swap(perm.p, perm_new.p);
    }
    // the words and values in sorted order
    SCI_CK(cudaMalloc(&sorted.p, total * 8 * KW));
    uint64_t *SW = sorted.as<uint64_t>();
    for (int w = 0; w < KW; w++)
        k_gather_u64<<<grid_for(total), 256, 0, st>>>(W + w * total, perm.as<uint32_t>(), total, SW + w * total);
    k_gather_u64<<<grid_for(total), 256, 0, st>>>(vals.as<uint64_t>(), perm.as<uint32_t>(), total,
                                                  B.vals_sorted.as<uint64_t>());
    SCI_CK(cudaMalloc(&flag.p, total * 4));
    SCI_CK(cudaMalloc(&rid.p, total * 4));
    k_run_flags_w<<<grid_for(total), 256, 0, st>>>(SW, KW, total, flag.as<uint32_t>());
    SCI_CK(cudaGetLastError());
    size_t tb3 = 0;
    SCI_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb3, flag.as<uint32_t>(), rid.as<uint32_t>(), nitems, st));
    TmpBuf tmp3;
    SCI_CK(cudaMalloc(&tmp3.p, std::max<size_t>(tb3, 16)));
    SCI_CK(cub::DeviceScan::ExclusiveSum(tmp3.p, tb3, flag.as<uint32_t>(), rid.as<uint32_t>(), nitems, st));
    uint32_t last[2] = {0, 0};
    SCI_CK(cudaMemcpyAsync(&last[0], rid.as<uint32_t>() + (total - 1), 4, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaMemcpyAsync(&last[1], flag.as<uint32_t>() + (total - 1), 4, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    nruns = (int)(last[0] + last[1]);
    SCI_CK(cudaMalloc(&B.ukeys.p, (size_t)nruns * 8 * KW));
    SCI_CK(cudaMalloc(&B.counts.p, (size_t)nruns * 4));
    SCI_CK(cudaMalloc(&start.p, (size_t)nruns * 4));
    k_runs_w<<<grid_for(total), 256, 0, st>>>(flag.as<uint32_t>(), rid.as<uint32_t>(), SW, KW, total,
                                              B.ukeys.as<uint64_t>(), start.as<uint32_t>());
    k_run_counts<<<grid_for(nruns), 256, 0, st>>>(start.as<uint32_t>(), nruns, total, B.counts.as<uint32_t>());
    SCI_CK(cudaGetLastError());
    SCI_CK(cudaStreamSynchronize(st));
    return SCI_OK;
}

int build_buckets(sci_ctx *ctx, int holes, int per_det, Buckets &B)
{
    cudaStream_t st = ctx->stream;
    int64_t M = ctx->M;
    int64_t total = M * per_det;
    if (total >= (int64_t)1 << 31) return sci_fail(ctx, SCI_ERR_OVERFLOW, "too many bucket entries (>= 2^31)");
    if (total == 0) return SCI_OK;
    int nitems = (int)total;
    int nruns = 0;
    if (ctx->nwords > 1) {
        int rc = ctx->nwords == 2   ? sort_runs_w<2>(ctx, holes, per_det, total, B, nruns)
                 : ctx->nwords == 3 ? sort_runs_w<3>(ctx, holes, per_det, total, B, nruns)
                                    : sort_runs_w<4>(ctx, holes, per_det, total, B, nruns);
        if (rc != SCI_OK) return rc;
        return order_runs(ctx, nruns, B);
    }
    TmpBuf ka, kb, va;
    SCI_CK(cudaMalloc(&ka.p, total * 8));
    SCI_CK(cudaMalloc(&kb.p, total * 8));
    SCI_CK(cudaMalloc(&va.p, total * 8));
    SCI_CK(cudaMalloc(&B.vals_sorted.p, total * 8));
    k_emit<1><<<grid_for(M), 256, 0, st>>>(ctx->keys, M, holes, per_det, ka.as<uint64_t>(), total,
                                          va.as<uint64_t>());
    SCI_CK(cudaGetLastError());
    cub::DoubleBuffer<uint64_t> dk(ka.as<uint64_t>(), kb.as<uint64_t>());
    cub::DoubleBuffer<uint64_t> dv(va.as<uint64_t>(), B.vals_sorted.as<uint64_t>());
    int end_bit = ctx->norb;
    size_t tb = 0;
    SCI_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, dk, dv, nitems, 0, end_bit, st));
    {
        TmpBuf tmp;
        SCI_CK(cudaMalloc(&tmp.p, tb));
        SCI_CK(cub::DeviceRadixSort::SortPairs(tmp.p, tb, dk, dv, nitems, 0, end_bit, st));
    }
    // keep the sorted values; release the other value buffer
    if (dv.Current() != B.vals_sorted.as<uint64_t>()) std::swap(va.p, B.vals_sorted.p);
    cudaFree(va.p);
    va.p = nullptr;
    const uint64_t *sorted_keys = dk.Current();

    // run-length encode the sorted keys
    SCI_CK(cudaMalloc(&B.ukeys.p, total * 8));
    SCI_CK(cudaMalloc(&B.counts.p, total * 4));
    TmpBuf nruns_d;
    SCI_CK(cudaMalloc(&nruns_d.p, 8));
    tb = 0;
    SCI_CK(cub::DeviceRunLengthEncode::Encode(nullptr, tb, sorted_keys, B.ukeys.as<uint64_t>(),
                                              B.counts.as<uint32_t>(), nruns_d.as<int>(), nitems, st));
    {
        TmpBuf tmp;
        SCI_CK(cudaMalloc(&tmp.p, tb));
        SCI_CK(cub::DeviceRunLengthEncode::Encode(tmp.p, tb, sorted_keys, B.ukeys.as<uint64_t>(),
                                                  B.counts.as<uint32_t>(), nruns_d.as<int>(), nitems, st));
    }
    SCI_CK(cudaMemcpyAsync(&nruns, nruns_d.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    cudaFree(ka.p); ka.p = nullptr;
    cudaFree(kb.p); kb.p = nullptr;
    return order_runs(ctx, nruns, B);
}

// Given the runs of equal keys (B.counts, B.ukeys, B.vals_sorted), drop the singletons and
// order the kept buckets by size, largest first, with their new offsets.
int order_runs(sci_ctx *ctx, int nruns, Buckets &B)
{
    cudaStream_t st = ctx->stream;
    size_t tb = 0;
    // offsets of the runs in sorted order
    SCI_CK(cudaMalloc(&B.offsets.p, (size_t)nruns * 4));
    tb = 0;
    SCI_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, B.counts.as<uint32_t>(), B.offsets.as<uint32_t>(), nruns, st));
    {
        TmpBuf tmp;
        SCI_CK(cudaMalloc(&tmp.p, tb));
        SCI_CK(cub::DeviceScan::ExclusiveSum(tmp.p, tb, B.counts.as<uint32_t>(), B.offsets.as<uint32_t>(), nruns, st));
    }

    // order runs by size, largest first (stable: equal sizes keep key order)
    TmpBuf sk, sk2, ids, ids2, kept_d;
    SCI_CK(cudaMalloc(&sk.p, (size_t)nruns * 2));
    SCI_CK(cudaMalloc(&sk2.p, (size_t)nruns * 2));
    SCI_CK(cudaMalloc(&ids.p, (size_t)nruns * 4));
    SCI_CK(cudaMalloc(&ids2.p, (size_t)nruns * 4));
    SCI_CK(cudaMalloc(&kept_d.p, 16));
    SCI_CK(cudaMemsetAsync(kept_d.p, 0, 16, st));
    k_size_keys<<<grid_for(nruns), 256, 0, st>>>(B.counts.as<uint32_t>(), nruns, sk.as<uint16_t>(),
                                                 kept_d.as<unsigned long long>(),
                                                 (int *)(kept_d.as<char>() + 8));
    k_iota_u32<<<grid_for(nruns), 256, 0, st>>>(ids.as<uint32_t>(), nruns);
    SCI_CK(cudaGetLastError());
    cub::DoubleBuffer<uint16_t> dsk(sk.as<uint16_t>(), sk2.as<uint16_t>());
    cub::DoubleBuffer<uint32_t> dids(ids.as<uint32_t>(), ids2.as<uint32_t>());
    tb = 0;
    SCI_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, dsk, dids, nruns, 0, 16, st));
    {
        TmpBuf tmp;
        SCI_CK(cudaMalloc(&tmp.p, tb));
        SCI_CK(cub::DeviceRadixSort::SortPairs(tmp.p, tb, dsk, dids, nruns, 0, 16, st));
    }
    unsigned long long kept_h = 0;
    int maxb_h = 0;
    SCI_CK(cudaMemcpyAsync(&kept_h, kept_d.p, 8, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaMemcpyAsync(&maxb_h, kept_d.as<char>() + 8, 4, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    B.kept = (int64_t)kept_h;
    B.maxb = B.kept > 0 ? maxb_h : 0;
    // keep the order array
    if (dids.Current() == ids.as<uint32_t>()) std::swap(ids.p, B.order.p);
    else std::swap(ids2.p, B.order.p);
    if (B.kept == 0) return SCI_OK;

    // new offsets of the kept runs
    TmpBuf ksz;
    SCI_CK(cudaMalloc(&ksz.p, (size_t)B.kept * 4));
    SCI_CK(cudaMalloc(&B.newoff.p, (size_t)B.kept * 4));
    k_gather_sizes<<<grid_for(B.kept), 256, 0, st>>>(B.order.as<uint32_t>(), B.counts.as<uint32_t>(), B.kept,
                                                     ksz.as<uint32_t>());
    SCI_CK(cudaGetLastError());
    tb = 0;
    SCI_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, ksz.as<uint32_t>(), B.newoff.as<uint32_t>(), (int)B.kept, st));
    {
        TmpBuf tmp;
        SCI_CK(cudaMalloc(&tmp.p, tb));
        SCI_CK(cub::DeviceScan::ExclusiveSum(tmp.p, tb, ksz.as<uint32_t>(), B.newoff.as<uint32_t>(), (int)B.kept, st));
    }
    uint32_t last_off = 0, last_size = 0;
    SCI_CK(cudaMemcpyAsync(&last_off, B.newoff.as<uint32_t>() + (B.kept - 1), 4, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaMemcpyAsync(&last_size, ksz.as<uint32_t>() + (B.kept - 1), 4, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    B.entries = (int64_t)last_off + last_size;
    return SCI_OK;
}

// ------------------------------------------------------------------ tiled prefix
// The (N-2) table holds its buckets largest first, so the buckets of more than thr
// members are its first entries.  out[0] = the end of that prefix (written by the one
// entry where the sizes cross thr); out[1] counts entries where a bucket above thr follows
// one at or below it, which a table in size order never has.
__global__ void k_split_point(const uint32_t *__restrict__ e_pos, int64_t E, int thr, unsigned long long *out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const bool big = sci::pos_size(e_pos[p]) > thr;
        const bool next_big = p + 1 < E && sci::pos_size(e_pos[p + 1]) > thr;
        if (big && !next_big) out[0] = (unsigned long long)(p + 1);
        if (!big && next_big) atomicAdd(out + 1, 1ull);
    }
}

// tile starts: the entries at bucket offsets 0, kTileRows, 2 kTileRows, ...
__global__ void k_tile_flags(const uint32_t *__restrict__ e_pos, int64_t E, uint32_t *__restrict__ flag)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = sci::pos_off(e_pos[p]) % sci::kTileRows == 0;
}

__global__ void k_tile_fill(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ at, int64_t E,
                            uint32_t *__restrict__ tiles)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x)
        if (flag[p]) tiles[at[p]] = (uint32_t)p;
}

}  // namespace

void sci_free_split(sci_ctx *ctx, bool ranged)
{
    sci::TileSplit &sp = ranged ? ctx->rsplit2 : ctx->split2;
    if (sp.tiles) cudaFree(sp.tiles);
    sp = sci::TileSplit{};
}

namespace {
// the split at threshold thr: the end of the prefix of buckets above thr and the largest
// bucket after it
int split_point(sci_ctx *ctx, const uint32_t *e_pos, int64_t E, int thr, sci::Split &out)
{
    cudaStream_t st = ctx->stream;
    TmpBuf cnt;
    unsigned long long h[2] = {0, 0};
    SCI_CK(cudaMalloc(&cnt.p, 16));
    SCI_CK(cudaMemsetAsync(cnt.p, 0, 16, st));
    k_split_point<<<grid_for(E), 256, 0, st>>>(e_pos, E, thr, cnt.as<unsigned long long>());
    SCI_CK(cudaGetLastError());
    SCI_CK(cudaMemcpyAsync(h, cnt.p, 16, cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    if (h[1] != 0) return sci_fail(ctx, SCI_ERR_STATE, "internal: (N-2) buckets not in size order");
    out.big = (int64_t)h[0];
    out.maxb_small = 0;
    if (out.big < E) {
        uint32_t pos = 0;
        SCI_CK(cudaMemcpy(&pos, e_pos + out.big, 4, cudaMemcpyDeviceToHost));
        out.maxb_small = sci::pos_size(pos);
    }
    return SCI_OK;
}
}  // namespace

int sci_table_split(sci_ctx *ctx, bool ranged)
{
    sci_free_split(ctx, ranged);
    const uint32_t *e_pos = ranged ? ctx->r2_pos : ctx->e2_pos;
    const int64_t E = ranged ? ctx->r2 : ctx->e2;
    if (E == 0) return SCI_OK;
    cudaStream_t st = ctx->stream;
    sci::TileSplit sp;
    const int thr_wide = ctx->tile_user ? ctx->tile_b : std::min(ctx->tile_b, sci::kTileBucketWide);
    int rc = split_point(ctx, e_pos, E, ctx->tile_b, sp.base);
    if (rc == SCI_OK) rc = split_point(ctx, e_pos, E, thr_wide, sp.wide);
    if (rc != SCI_OK) return rc;
    const int64_t big = sp.wide.big;   // >= sp.base.big: the lower threshold tiles more
    if (big > 0) {
        TmpBuf flag, at, tmp;
        const int nitems = (int)big;
        SCI_CK(cudaMalloc(&flag.p, (size_t)big * 4));
        SCI_CK(cudaMalloc(&at.p, (size_t)big * 4));
        k_tile_flags<<<grid_for(big), 256, 0, st>>>(e_pos, big, flag.as<uint32_t>());
        size_t tb = 0;
        SCI_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, flag.as<uint32_t>(), at.as<uint32_t>(), nitems, st));
        SCI_CK(cudaMalloc(&tmp.p, std::max<size_t>(tb, 16)));
        SCI_CK(cub::DeviceScan::ExclusiveSum(tmp.p, tb, flag.as<uint32_t>(), at.as<uint32_t>(), nitems, st));
        uint32_t last[3] = {0, 0, 0};
        SCI_CK(cudaMemcpyAsync(&last[0], at.as<uint32_t>() + (big - 1), 4, cudaMemcpyDeviceToHost, st));
        SCI_CK(cudaMemcpyAsync(&last[1], flag.as<uint32_t>() + (big - 1), 4, cudaMemcpyDeviceToHost, st));
        if (sp.base.big < big)   // the tiles of the base prefix: those starting before its end
            SCI_CK(cudaMemcpyAsync(&last[2], at.as<uint32_t>() + sp.base.big, 4, cudaMemcpyDeviceToHost, st));
        SCI_CK(cudaStreamSynchronize(st));
        sp.wide.ntiles = (int64_t)last[0] + last[1];
        sp.base.ntiles = sp.base.big < big ? (int64_t)last[2] : sp.wide.ntiles;
        SCI_CK(cudaMalloc(&sp.tiles, (size_t)sp.wide.ntiles * 4));
        k_tile_fill<<<grid_for(big), 256, 0, st>>>(flag.as<uint32_t>(), at.as<uint32_t>(), big, sp.tiles);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFree(sp.tiles);
            return sci_cuda_check(ctx, e, "tile list");
        }
    }
    (ranged ? ctx->rsplit2 : ctx->split2) = sp;
    return SCI_OK;
}

namespace {

void free_dets(sci_ctx *ctx)
{
    sci_free_range(ctx);
    sci_free_det(ctx);
    sci_free_split(ctx, false);
    free_held(ctx, ctx->keys);
    free_held(ctx, ctx->hdiag);
    free_held(ctx, ctx->fref);
    free_held(ctx, ctx->c_ds);
    free_held(ctx, ctx->fref_ds);
    free_held(ctx, ctx->e2_idx);
    free_held(ctx, ctx->e2_code);
    free_held(ctx, ctx->e2_pos);
    free_held(ctx, ctx->e1_idx);
    free_held(ctx, ctx->e1_S);
    free_held(ctx, ctx->e1_meta);
    ctx->have_dets = 0;
    ctx->nwords = 1;
    ctx->ref_hi = ctx->ref_w2 = ctx->ref_w3 = 0;
    ctx->M = 0;
    ctx->e1 = ctx->e2 = ctx->nb1 = ctx->nb2 = 0;
    ctx->maxb1 = ctx->maxb2 = 0;
    ctx->pairs = ctx->pairs1 = ctx->pairs2 = 0;
}

void free_ints(sci_ctx *ctx)
{
    free_held(ctx, ctx->h_so);
    free_held(ctx, ctx->jd);
    free_held(ctx, ctx->kd);
    free_held(ctx, ctx->g_so);
    free_held(ctx, ctx->tab);
    free_held(ctx, ctx->tab32);
    free_held(ctx, ctx->tab_ds);
    free_held(ctx, ctx->g_ds);
    ctx->have_ints = 0;
}

size_t scalar_bytes(const sci_ctx *ctx) { return ctx->cplx ? 16 : 8; }

// diagonal and reference Fock matrix for the current integrals and determinants
int compute_diag_fref(sci_ctx *ctx)
{
    cudaStream_t st = ctx->stream;
    int norb = ctx->norb;
    if (!ctx->fref) SCI_CK(alloc_held(ctx, &ctx->fref, (size_t)norb * norb * scalar_bytes(ctx)));
    int nn = norb * norb;
    if (ctx->cplx) {
        k_fref<zdbl><<<(nn + 255) / 256, 256, 0, st>>>(norb, Kw<4>{{ctx->ref, ctx->ref_hi, ctx->ref_w2, ctx->ref_w3}},
                                                        (const zdbl *)ctx->h_so, (const zdbl *)ctx->g_so,
                                                        (zdbl *)ctx->fref);
        if (ctx->M > 0) {
            auto kd = ctx->nwords == 4   ? k_diag<zdbl, 4>
                      : ctx->nwords == 3 ? k_diag<zdbl, 3>
                      : ctx->nwords == 2 ? k_diag<zdbl, 2>
                                         : k_diag<zdbl, 1>;
            kd<<<grid_for(ctx->M), 256, 0, st>>>(ctx->keys, ctx->M, norb, (const zdbl *)ctx->h_so,
                                                 (const zdbl *)ctx->jd, (const zdbl *)ctx->kd, ctx->hdiag);
        }
    } else {
        k_fref<double><<<(nn + 255) / 256, 256, 0, st>>>(norb, Kw<4>{{ctx->ref, ctx->ref_hi, ctx->ref_w2, ctx->ref_w3}},
                                                          (const double *)ctx->h_so, (const double *)ctx->g_so,
                                                          (double *)ctx->fref);
        if (ctx->M > 0) {
            auto kd = ctx->nwords == 4   ? k_diag<double, 4>
                      : ctx->nwords == 3 ? k_diag<double, 3>
                      : ctx->nwords == 2 ? k_diag<double, 2>
                                         : k_diag<double, 1>;
            kd<<<grid_for(ctx->M), 256, 0, st>>>(ctx->keys, ctx->M, norb, (const double *)ctx->h_so,
                                                 (const double *)ctx->jd, (const double *)ctx->kd, ctx->hdiag);
        }
    }
    // paired-FP32 copy of fref for the paired-FP32 singles
    const int64_t nd = (int64_t)nn * (ctx->cplx ? 2 : 1);
    if (!ctx->fref_ds) SCI_CK(alloc_held(ctx, &ctx->fref_ds, (size_t)nd * 8));
    k_split_ds<<<grid_for(nd), 256, 0, st>>>((const double *)ctx->fref, (float2 *)ctx->fref_ds, nd);
    SCI_CK(cudaGetLastError());
    return SCI_OK;
}

// Symmetry checks of integrals given on the device: o[0] = max |x|, o[1] = max |a - b| over
// the pairs that the symmetry makes equal, by atomicMax on the bits of nonnegative doubles
// (their order as unsigned integers is that of the values).  A thread that meets a value
// that is not finite posts a NaN, whose bits sort above every number.
__device__ __forceinline__ void amax_bits(unsigned long long *o, double v, bool bad)
{
    const unsigned long long nan_bits = 0x7FF8000000000000ull;
    atomicMax(o, bad ? nan_bits : (unsigned long long)__double_as_longlong(fabs(v)));
}

__device__ __forceinline__ bool finite(double x) { return fabs(x) <= 1.7976931348623157e308; }

__global__ void k_chk_abs(const double *__restrict__ x, int64_t cnt, unsigned long long *o)
{
    double m = 0.0;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        m = fmax(m, fabs(x[t]));
        bad |= !finite(x[t]);
    }
    amax_bits(o, m, bad);
}

// h Hermitian: h_pq = conj(h_qp)
__global__ void k_chk_h(const double *__restrict__ h, int n, int sw, unsigned long long *o)
{
    double m = 0.0;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / n, q = t % n, a = p * n + q, b = q * n + p;
        m = fmax(m, fabs(h[a * sw] - h[b * sw]));
        if (sw == 2) m = fmax(m, fabs(h[a * sw + 1] + h[b * sw + 1]));
        bad |= !finite(h[a * sw]) || (sw == 2 && !finite(h[a * sw + 1]));
    }
    amax_bits(o, m, bad);
}

// (pq|rs) = (rs|pq) = conj((qp|sr))
__global__ void k_chk_eri(const double *__restrict__ e, int n, int sw, unsigned long long *o)
{
    const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
    double m = 0.0;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pq = t / n2, rs = t % n2, p = pq / n, q = pq % n, r = rs / n, s_ = rs % n;
        const int64_t b = rs * n2 + pq, c = (q * n + p) * n2 + s_ * n + r;
        m = fmax(m, fmax(fabs(e[t * sw] - e[b * sw]), fabs(e[t * sw] - e[c * sw])));
        if (sw == 2) m = fmax(m, fmax(fabs(e[t * sw + 1] - e[b * sw + 1]), fabs(e[t * sw + 1] + e[c * sw + 1])));
        bad |= !finite(e[t * sw]) || (sw == 2 && !finite(e[t * sw + 1]));
    }
    amax_bits(o, m, bad);
}

// each Cholesky vector Hermitian: L^P_pq = conj(L^P_qp)
__global__ void k_chk_chol(const double *__restrict__ L, int naux, int n, int sw, unsigned long long *o)
{
    const int64_t n2 = (int64_t)n * n;
    double m = 0.0;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)naux * n2;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t P = t / n2, pq = t % n2, p = pq / n, q = pq % n, b = P * n2 + q * n + p;
        m = fmax(m, fabs(L[t * sw] - L[b * sw]));
        if (sw == 2) m = fmax(m, fabs(L[t * sw + 1] + L[b * sw + 1]));
        bad |= !finite(L[t * sw]) || (sw == 2 && !finite(L[t * sw + 1]));
    }
    amax_bits(o, m, bad);
}

bool rel_close(double a, double b, double scale) { return std::fabs(a - b) <= 1e-10 * scale; }

}  // namespace

// ================================================================== public API
extern "C" int sci_create(sci_ctx **out, int device, void *cuda_stream)
{
    if (!out) return SCI_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return SCI_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return SCI_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SCI_ERR_CUDA;
    // commit the fixed scratch of sci_connections_noalloc() on this device now, so that
    // its callers, who cannot allocate, never meet a lazy module load later
    if (sci_noalloc_prepare(device) != cudaSuccess) return SCI_ERR_CUDA;
    sci_ctx *ctx = new sci_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (cudaMalloc(&ctx->status, sizeof(int)) != cudaSuccess || cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return SCI_ERR_NOMEM;
    }
    *out = ctx;
    return SCI_OK;
}

extern "C" int sci_destroy(sci_ctx *ctx)
{
    if (!ctx) return SCI_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_dets(ctx);
    free_ints(ctx);
    if (ctx->stage_c) cudaFree(ctx->stage_c);
    if (ctx->stage_s) cudaFree(ctx->stage_s);
    if (ctx->bv_part) cudaFree(ctx->bv_part);
    if (ctx->rdm_scratch) cudaFree(ctx->rdm_scratch);
    if (ctx->rdm_w) cudaFree(ctx->rdm_w);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
    return SCI_OK;
}

extern "C" int sci_set_stream(sci_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return SCI_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return SCI_OK;
}

namespace {
// the device-side form of the host symmetry checks below, for integrals given on the device
int check_ints_device(sci_ctx *ctx, int cplx, int n, const double *h, const double *eri, int naux, const double *chol)
{
    cudaStream_t st = ctx->stream;
    const int sw = cplx ? 2 : 1;
    const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
    TmpBuf o;
    SCI_CK(cudaMalloc(&o.p, 4 * sizeof(unsigned long long)));
    SCI_CK(cudaMemsetAsync(o.p, 0, 4 * sizeof(unsigned long long), st));
    unsigned long long *ob = o.as<unsigned long long>();
    k_chk_abs<<<grid_for(n2 * sw), 256, 0, st>>>(h, n2 * sw, ob);
    k_chk_h<<<grid_for(n2), 256, 0, st>>>(h, n, sw, ob + 1);
    if (eri) {
        k_chk_abs<<<grid_for(n4 * sw), 256, 0, st>>>(eri, n4 * sw, ob + 2);
        k_chk_eri<<<grid_for(n4), 256, 0, st>>>(eri, n, sw, ob + 3);
    } else {
        k_chk_abs<<<grid_for((int64_t)naux * n2 * sw), 256, 0, st>>>(chol, (int64_t)naux * n2 * sw, ob + 2);
        k_chk_chol<<<grid_for((int64_t)naux * n2), 256, 0, st>>>(chol, naux, n, sw, ob + 3);
    }
    SCI_CK(cudaGetLastError());
    unsigned long long r[4] = {0, 0, 0, 0};
    SCI_CK(cudaMemcpyAsync(r, ob, sizeof(r), cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    const unsigned long long inf_bits = 0x7FF0000000000000ull;
    if (r[0] >= inf_bits || r[1] >= inf_bits) return sci_fail(ctx, SCI_ERR_ARG, "h has a value that is not finite");
    if (r[2] >= inf_bits || r[3] >= inf_bits)
        return sci_fail(ctx, SCI_ERR_ARG, "the integrals have a value that is not finite");
    double v[4];
    std::memcpy(v, r, sizeof(v));
    if (!rel_close(v[1], 0.0, v[0] + 1e-300)) return sci_fail(ctx, SCI_ERR_ARG, "h is not Hermitian");
    if (!rel_close(v[3], 0.0, v[2] + 1e-300))
        return sci_fail(ctx, SCI_ERR_ARG, eri ? "eri lacks (pq|rs)=(rs|pq)=(qp|sr)^* symmetry"
                                              : "Cholesky vectors are not Hermitian");
    return SCI_OK;
}

// a device pointer of the context's device (or managed memory)
bool on_ctx_device(const sci_ctx *ctx, const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == ctx->device);
}

int set_ints(sci_ctx *ctx, int scalar, int mode, int n, const void *h, const void *eri, int naux, const void *chol,
             int on_device);
}  // namespace

extern "C" int sci_set_integrals(sci_ctx *ctx, int scalar, int mode, int n, const void *h, const void *eri,
                                 int naux, const void *chol)
{
    return set_ints(ctx, scalar, mode, n, h, eri, naux, chol, 0);
}

extern "C" int sci_set_integrals_ex(sci_ctx *ctx, int scalar, int mode, int n, const void *h, const void *eri,
                                    int naux, const void *chol, int on_device)
{
    return set_ints(ctx, scalar, mode, n, h, eri, naux, chol, on_device);
}

namespace {
int set_ints(sci_ctx *ctx, int scalar, int mode, int n, const void *h, const void *eri, int naux, const void *chol,
             int on_device)
{
    if (!ctx) return SCI_ERR_ARG;
    ctx->err.clear();
    if (scalar != SCI_REAL64 && scalar != SCI_COMPLEX128) return sci_fail(ctx, SCI_ERR_ARG, "bad scalar type");
    if (mode != SCI_SPIN_ORBITALS && mode != SCI_SPINORS) return sci_fail(ctx, SCI_ERR_ARG, "bad mode");
    if (mode == SCI_SPIN_ORBITALS && (n < 1 || n > 128)) return sci_fail(ctx, SCI_ERR_ARG, "spin-orbital mode needs 1 <= n <= 128");
    if (mode == SCI_SPINORS && (n < 1 || n > 256)) return sci_fail(ctx, SCI_ERR_ARG, "spinor mode needs 1 <= n <= 256");
    if (mode == SCI_SPIN_ORBITALS && scalar != SCI_REAL64)
        return sci_fail(ctx, SCI_ERR_ARG, "spin-orbital mode takes real integrals");
    if (!h) return sci_fail(ctx, SCI_ERR_ARG, "h is NULL");
    if ((eri == nullptr) == (chol == nullptr)) return sci_fail(ctx, SCI_ERR_ARG, "give exactly one of eri / chol");
    if (chol && naux < 1) return sci_fail(ctx, SCI_ERR_ARG, "naux < 1");
    SCI_CK(cudaSetDevice(ctx->device));
    const int cplx = scalar == SCI_COMPLEX128;
    const int sw = cplx ? 2 : 1;  // doubles per scalar
    const double *hd = (const double *)h;
    int64_t n2 = (int64_t)n * n, n4 = n2 * n2;

    if (on_device) {
        if (!on_ctx_device(ctx, h) || (eri && !on_ctx_device(ctx, eri)) || (chol && !on_ctx_device(ctx, chol)))
            return sci_fail(ctx, SCI_ERR_ARG, "on_device: h, eri and chol must be memory of the context's device");
        int rc = check_ints_device(ctx, cplx, n, hd, (const double *)eri, naux, (const double *)chol);
        if (rc != SCI_OK) return rc;
    } else {
    // ---- host-side symmetry checks (h Hermitian; (pq|rs) = (rs|pq) = (qp|sr)^*)
    double hs = 0;
    for (int64_t t = 0; t < n2 * sw; t++) hs = std::max(hs, std::fabs(hd[t]));
    for (int p = 0; p < n; p++)
        for (int q = 0; q < n; q++) {
            int64_t a = (int64_t)p * n + q, b = (int64_t)q * n + p;
            if (!rel_close(hd[a * sw], hd[b * sw], hs + 1e-300) ||
                (cplx && !rel_close(hd[a * sw + 1], -hd[b * sw + 1], hs + 1e-300)))
                return sci_fail(ctx, SCI_ERR_ARG, "h is not Hermitian");
        }
    if (eri) {
        const double *e = (const double *)eri;
        double es = 0;
        for (int64_t t = 0; t < n4 * sw; t++) es = std::max(es, std::fabs(e[t]));
        es += 1e-300;
        for (int p = 0; p < n; p++)
            for (int q = 0; q < n; q++)
                for (int r = 0; r < n; r++)
                    for (int s = 0; s < n; s++) {
                        int64_t a = ((int64_t)(p * n + q) * n + r) * n + s;
                        int64_t b = ((int64_t)(r * n + s) * n + p) * n + q;
                        int64_t c = ((int64_t)(q * n + p) * n + s) * n + r;
                        if (!rel_close(e[a * sw], e[b * sw], es) || !rel_close(e[a * sw], e[c * sw], es))
                            return sci_fail(ctx, SCI_ERR_ARG, "eri lacks (pq|rs)=(rs|pq)=(qp|sr)^* symmetry");
                        if (cplx && (!rel_close(e[a * sw + 1], e[b * sw + 1], es) ||
                                     !rel_close(e[a * sw + 1], -e[c * sw + 1], es)))
                            return sci_fail(ctx, SCI_ERR_ARG, "eri lacks (pq|rs)=(rs|pq)=(qp|sr)^* symmetry");
                    }
    } else {
        const double *L = (const double *)chol;
        double ls = 0;
        for (int64_t t = 0; t < (int64_t)naux * n2 * sw; t++) ls = std::max(ls, std::fabs(L[t]));
        ls += 1e-300;
        for (int P = 0; P < naux; P++)
            for (int p = 0; p < n; p++)
                for (int q = 0; q < n; q++) {
                    int64_t a = P * n2 + (int64_t)p * n + q, b = P * n2 + (int64_t)q * n + p;
                    if (!rel_close(L[a * sw], L[b * sw], ls) || (cplx && !rel_close(L[a * sw + 1], -L[b * sw + 1], ls)))
                        return sci_fail(ctx, SCI_ERR_ARG, "Cholesky vectors are not Hermitian");
                }
    }
    }

    int keep_dets = ctx->have_dets && ctx->have_ints && ctx->cplx == cplx && ctx->n == n &&
                    ctx->spinors == (mode == SCI_SPINORS);
    if (!keep_dets) free_dets(ctx);
    free_ints(ctx);
    ctx->cplx = cplx;
    ctx->spinors = mode == SCI_SPINORS;
    ctx->n = n;
    ctx->norb = ctx->spinors ? n : 2 * n;
    const size_t sb = cplx ? 16 : 8;
    cudaStream_t st = ctx->stream;

    // device copies of h and (pq|rs); integrals given on the device are read in place
    TmpBuf dh, deri, dl;
    const void *hsrc = h, *esrc = eri;
    if (!on_device) {
        SCI_CK(cudaMalloc(&dh.p, n2 * sb));
        SCI_CK(cudaMemcpyAsync(dh.p, h, n2 * sb, cudaMemcpyHostToDevice, st));
        hsrc = dh.p;
    }
    if (!(eri && on_device)) {
        SCI_CK(cudaMalloc(&deri.p, n4 * sb));
        esrc = deri.p;
    }
    if (eri) {
        if (!on_device) SCI_CK(cudaMemcpyAsync(deri.p, eri, n4 * sb, cudaMemcpyHostToDevice, st));
    } else {
        const void *lsrc = chol;
        if (!on_device) {
            SCI_CK(cudaMalloc(&dl.p, (size_t)naux * n2 * sb));
            SCI_CK(cudaMemcpyAsync(dl.p, chol, (size_t)naux * n2 * sb, cudaMemcpyHostToDevice, st));
            lsrc = dl.p;
        }
        if (cplx) k_eri_from_chol<zdbl><<<grid_for(n4), 256, 0, st>>>((const zdbl *)lsrc, naux, n, deri.as<zdbl>());
        else k_eri_from_chol<double><<<grid_for(n4), 256, 0, st>>>((const double *)lsrc, naux, n, deri.as<double>());
        SCI_CK(cudaGetLastError());
        SCI_CK(cudaStreamSynchronize(st));
    }
    int norb = ctx->norb;
    SCI_CK(alloc_held(ctx, &ctx->h_so, (size_t)norb * norb * sb));
    SCI_CK(alloc_held(ctx, &ctx->jd, (size_t)norb * norb * sb));
    SCI_CK(alloc_held(ctx, &ctx->kd, (size_t)norb * norb * sb));
    SCI_CK(alloc_held(ctx, &ctx->g_so, (size_t)norb * norb * norb * sb));
    OrbMap om{n, ctx->spinors};
    int64_t n3 = (int64_t)norb * norb * norb;
    if (cplx)
        k_small_tables<zdbl><<<grid_for(n3), 256, 0, st>>>((const zdbl *)hsrc, (const zdbl *)esrc, om, norb, (zdbl *)ctx->h_so,
                                                           (zdbl *)ctx->jd, (zdbl *)ctx->kd, (zdbl *)ctx->g_so);
    else
        k_small_tables<double><<<grid_for(n3), 256, 0, st>>>((const double *)hsrc, (const double *)esrc, om, norb,
                                                             (double *)ctx->h_so, (double *)ctx->jd, (double *)ctx->kd,
                                                             (double *)ctx->g_so);
    SCI_CK(cudaGetLastError());
    int64_t NP = (int64_t)n * (n - 1) / 2;
    if (ctx->spinors) {
        ctx->tab_elems = NP * NP;
        SCI_CK(alloc_held(ctx, &ctx->tab, (size_t)ctx->tab_elems * sb));
        if (cplx) {
            if (ctx->tab_elems > 0)
                k_tab_spinor<<<grid_for(ctx->tab_elems), 256, 0, st>>>((const zdbl *)esrc, n, (zdbl *)ctx->tab);
        } else {
            return sci_fail(ctx, SCI_ERR_ARG, "spinor mode takes complex integrals");
        }
    } else {
        ctx->tab_elems = n4 + NP * NP;
        SCI_CK(alloc_held(ctx, &ctx->tab, (size_t)ctx->tab_elems * sb));
        k_tab_real<<<grid_for(ctx->tab_elems), 256, 0, st>>>((const double *)esrc, n, (double *)ctx->tab);
        SCI_CK(alloc_held(ctx, (void **)&ctx->tab32, (size_t)ctx->tab_elems * 4));
        k_to_f32<<<grid_for(ctx->tab_elems), 256, 0, st>>>((const double *)ctx->tab, ctx->tab32, ctx->tab_elems);
    }
    // paired-FP32 copy of the pair table (complex: re and im parts each split)
    {
        int64_t nd = ctx->tab_elems * (cplx ? 2 : 1);
        SCI_CK(alloc_held(ctx, &ctx->tab_ds, (size_t)nd * 8));
        if (nd > 0) k_split_ds<<<grid_for(nd), 256, 0, st>>>((const double *)ctx->tab, (float2 *)ctx->tab_ds, nd);
        const int64_t ng = (int64_t)norb * norb * norb * (cplx ? 2 : 1);
        SCI_CK(alloc_held(ctx, &ctx->g_ds, (size_t)ng * 8));
        k_split_ds<<<grid_for(ng), 256, 0, st>>>((const double *)ctx->g_so, (float2 *)ctx->g_ds, ng);
    }
    SCI_CK(cudaGetLastError());
    ctx->have_ints = 1;
    if (ctx->have_dets) {
        int rc = compute_diag_fref(ctx);
        if (rc != SCI_OK) return rc;
    }
    SCI_CK(cudaStreamSynchronize(st));
    return SCI_OK;
}
}  // namespace

namespace {
int set_dets(sci_ctx *ctx, const uint64_t *keys, int nwords, int64_t M, int n_alpha, int n_beta, int keys_on_device);
}

extern "C" int sci_set_determinants(sci_ctx *ctx, const uint64_t *keys, int64_t M, int n_alpha, int n_beta,
                                    int keys_on_device)
{
    if (!ctx) return SCI_ERR_ARG;
    if (ctx->have_ints && ctx->norb > 64)
        return sci_fail(ctx, SCI_ERR_ARG, "more than 64 spin-orbitals: use sci_set_determinants_w with two to four words");
    return set_dets(ctx, keys, 1, M, n_alpha, n_beta, keys_on_device);
}

extern "C" int sci_set_determinants_w(sci_ctx *ctx, const uint64_t *keys, int nwords, int64_t M, int n_alpha,
                                      int n_beta, int keys_on_device)
{
    if (!ctx) return SCI_ERR_ARG;
    if (nwords < 1 || nwords > sci::kMaxWords) return sci_fail(ctx, SCI_ERR_ARG, "nwords must be 1 to 4");
    if (ctx->have_ints && ctx->norb > 64 * nwords)
        return sci_fail(ctx, SCI_ERR_ARG, "more spin-orbitals than the key words hold (64 per word)");
    return set_dets(ctx, keys, nwords, M, n_alpha, n_beta, keys_on_device);
}

extern "C" int sci_set_tile_threshold(sci_ctx *ctx, int members)
{
    if (!ctx) return SCI_ERR_ARG;
    ctx->err.clear();
    if (members < 0 || members > 0xFFFF) return sci_fail(ctx, SCI_ERR_ARG, "tile threshold outside [0, 65535]");
    SCI_CK(cudaSetDevice(ctx->device));
    SCI_CK(cudaStreamSynchronize(ctx->stream));   // no launch in flight reads the old tile lists
    const int old = ctx->tile_b, old_user = ctx->tile_user;
    ctx->tile_b = members == 0 ? sci::kTileBucket : members;
    ctx->tile_user = members != 0;
    if (!ctx->have_dets) return SCI_OK;
    int rc = sci_table_split(ctx, false);
    if (rc == SCI_OK && ctx->ranged) rc = sci_table_split(ctx, true);
    if (rc == SCI_OK && !sci_sigma_window_fits(ctx))
        rc = sci_fail(ctx, SCI_ERR_OVERFLOW, "buckets left to the window kernels do not fit shared memory");
    if (rc != SCI_OK) {   // back to the previous threshold, whose split was valid
        ctx->tile_b = old, ctx->tile_user = old_user;
        sci_table_split(ctx, false);
        if (ctx->ranged) sci_table_split(ctx, true);
    }
    return rc;
}

namespace {
int set_dets(sci_ctx *ctx, const uint64_t *keys, int nwords, int64_t M, int n_alpha, int n_beta, int keys_on_device)
{
    ctx->err.clear();
    if (!ctx->have_ints) return sci_fail(ctx, SCI_ERR_STATE, "set integrals before determinants");
    if (M < 0 || (M > 0 && !keys)) return sci_fail(ctx, SCI_ERR_ARG, "bad key array");
    if (M >= ((int64_t)1 << 31)) return sci_fail(ctx, SCI_ERR_OVERFLOW, "M >= 2^31");
    int N;
    if (ctx->spinors) {
        if (n_beta != -1 || n_alpha < 0 || n_alpha > ctx->n)
            return sci_fail(ctx, SCI_ERR_ARG, "spinor mode: n_alpha = N in [0, n], n_beta = -1");
        N = n_alpha;
    } else {
        if (n_alpha < 0 || n_beta < 0 || n_alpha > ctx->n || n_beta > ctx->n)
            return sci_fail(ctx, SCI_ERR_ARG, "electron counts out of range");
        N = n_alpha + n_beta;
    }
    SCI_CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    free_dets(ctx);
    ctx->M = M;
    ctx->na = n_alpha;
    ctx->nb = ctx->spinors ? -1 : n_beta;
    ctx->N = N;
    ctx->nwords = nwords;
    {
        // the reference: the lowest N spinors, or the lowest n_alpha alpha and n_beta beta
        // orbitals, over four words
        uint64_t r[4] = {0, 0, 0, 0};
        auto set = [&](int p) { r[p >> 6] |= 1ull << (p & 63); };
        if (ctx->spinors) {
            for (int p = 0; p < N; p++) set(p);
        } else {
            for (int p = 0; p < n_alpha; p++) set(p);
            for (int p = 0; p < n_beta; p++) set(ctx->n + p);
        }
        ctx->ref = r[0];
        ctx->ref_hi = r[1];
        ctx->ref_w2 = r[2];
        ctx->ref_w3 = r[3];
    }

    SCI_CK(alloc_held(ctx, (void **)&ctx->keys, (size_t)M * 8 * nwords));
    SCI_CK(alloc_held(ctx, (void **)&ctx->hdiag, (size_t)M * 8));
    SCI_CK(alloc_held(ctx, &ctx->c_ds, (size_t)M * 64));  // paired-FP32 coefficients, 64 B per determinant
    if (M > 0)
        SCI_CK(cudaMemcpyAsync(ctx->keys, keys, (size_t)M * 8 * nwords,
                               keys_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // K0: validation
    SCI_CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), st));
    if (M > 0) {
        KeyRule kr{ctx->spinors, ctx->n, n_alpha, n_beta, N};
        if (nwords == 4) k_validate<4><<<grid_for(M), 256, 0, st>>>(ctx->keys, M, kr, ctx->status);
        else if (nwords == 3) k_validate<3><<<grid_for(M), 256, 0, st>>>(ctx->keys, M, kr, ctx->status);
        else if (nwords == 2) k_validate<2><<<grid_for(M), 256, 0, st>>>(ctx->keys, M, kr, ctx->status);
        else k_validate<1><<<grid_for(M), 256, 0, st>>>(ctx->keys, M, kr, ctx->status);
        SCI_CK(cudaGetLastError());
    }
    int dev_status = 0;
    SCI_CK(cudaMemcpyAsync(&dev_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCI_CK(cudaStreamSynchronize(st));
    if (dev_status) {
        cudaMemsetAsync(ctx->status, 0, sizeof(int), st);
        free_dets(ctx);
        if (dev_status & sci::DEV_DUPLICATE) return sci_fail(ctx, SCI_ERR_DUPLICATE, "determinant list has duplicates");
        if (dev_status & sci::DEV_UNSORTED) return sci_fail(ctx, SCI_ERR_UNSORTED, "determinant list is not ascending");
        return sci_fail(ctx, SCI_ERR_POPCOUNT, "a key has the wrong electron count or stray bits");
    }
    int rc = compute_diag_fref(ctx);
    if (rc != SCI_OK) return rc;

    // (N-2)-hole buckets: doubles
    if (N >= 2) {
        Buckets B;
        rc = build_buckets(ctx, 2, N * (N - 1) / 2, B);
        if (rc != SCI_OK) { free_dets(ctx); return rc; }
        ctx->e2 = B.entries;
        ctx->nb2 = B.kept;
        ctx->maxb2 = B.maxb;
        SCI_CK(alloc_held(ctx, (void **)&ctx->e2_idx, (size_t)B.entries * 4));
        SCI_CK(alloc_held(ctx, (void **)&ctx->e2_code, (size_t)B.entries * 4));
        SCI_CK(alloc_held(ctx, (void **)&ctx->e2_pos, (size_t)B.entries * 4));
        if (B.kept > 0) {
            auto kf = nwords == 4 ? k_fill2<4> : nwords == 3 ? k_fill2<3> : nwords == 2 ? k_fill2<2> : k_fill2<1>;
            kf<<<grid_for(B.kept * 32), 256, 0, st>>>(B.order.as<uint32_t>(), B.counts.as<uint32_t>(),
                                                          B.offsets.as<uint32_t>(), B.newoff.as<uint32_t>(),
                                                          B.ukeys.as<uint64_t>(), B.vals_sorted.as<uint64_t>(), B.kept,
                                                          ctx->e2_idx, ctx->e2_code, ctx->e2_pos);
            SCI_CK(cudaGetLastError());
        }
        SCI_CK(cudaStreamSynchronize(st));
    }
    // (N-1)-hole buckets: singles
    if (N >= 1) {
        Buckets B;
        rc = build_buckets(ctx, 1, N, B);
        if (rc != SCI_OK) { free_dets(ctx); return rc; }
        ctx->e1 = B.entries;
        ctx->nb1 = B.kept;
        ctx->maxb1 = B.maxb;
        SCI_CK(alloc_held(ctx, (void **)&ctx->e1_idx, (size_t)B.entries * 4));
        SCI_CK(alloc_held(ctx, (void **)&ctx->e1_S, (size_t)B.entries * 8 * nwords));
        SCI_CK(alloc_held(ctx, (void **)&ctx->e1_meta, (size_t)B.entries * 4));
        if (B.kept > 0) {
            auto kf = nwords == 4 ? k_fill1<4> : nwords == 3 ? k_fill1<3> : nwords == 2 ? k_fill1<2> : k_fill1<1>;
            kf<<<grid_for(B.kept * 32), 256, 0, st>>>(B.order.as<uint32_t>(), B.counts.as<uint32_t>(),
                                                          B.offsets.as<uint32_t>(), B.newoff.as<uint32_t>(),
                                                          B.ukeys.as<uint64_t>(), B.vals_sorted.as<uint64_t>(), B.kept,
                                                          ctx->e1_idx, ctx->e1_S, ctx->e1_meta);
            SCI_CK(cudaGetLastError());
        }
        SCI_CK(cudaStreamSynchronize(st));
    }
    if (ctx->maxb2 > 0xFFFF || ctx->maxb1 > sci::kMaxBucket1) {
        free_dets(ctx);
        return sci_fail(ctx, SCI_ERR_OVERFLOW, "bucket larger than the table format allows");
    }
    // a list that sci_sigma() could not run is rejected here, not at every launch: the
    // largest bucket left to the window kernels (the buckets of more than tile_b members
    // go through the tiled kernel) must fit the shared-memory window of a one-vector
    // launch (always so at the default tile_b)
    rc = sci_table_split(ctx, false);
    if (rc != SCI_OK) { free_dets(ctx); return rc; }
    if (!sci_sigma_window_fits(ctx)) {
        free_dets(ctx);
        return sci_fail(ctx, SCI_ERR_OVERFLOW, "largest bucket does not fit the sigma kernel's shared-memory window");
    }
    ctx->have_dets = 1;
    int64_t p2 = 0, p1 = 0;
    rc = sci_count_pairs_device(ctx, &p2, &p1);
    if (rc != SCI_OK) { free_dets(ctx); return rc; }
    ctx->pairs2 = p2;
    ctx->pairs1 = p1;
    ctx->pairs = p1 + p2;
    return SCI_OK;
}
}  // namespace

extern "C" int sci_diagonal(sci_ctx *ctx, double *hdiag)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "no determinants");
    if (ctx->M > 0 && !hdiag) return sci_fail(ctx, SCI_ERR_ARG, "hdiag is NULL");
    if (ctx->M == 0) return SCI_OK;
    SCI_CK(cudaSetDevice(ctx->device));
    SCI_CK(cudaMemcpyAsync(hdiag, ctx->hdiag, (size_t)ctx->M * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return SCI_OK;
}

extern "C" int sci_sigma(sci_ctx *ctx, const void *C, void *S, int nvec, int prec)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_dets || !ctx->have_ints) return sci_fail(ctx, SCI_ERR_STATE, "integrals and determinants needed");
    if (nvec < 1) return sci_fail(ctx, SCI_ERR_ARG, "nvec < 1");
    if (prec != SCI_PREC_F64 && prec != SCI_PREC_F32_STORE_F64_ACC && prec != SCI_PREC_F64_DS)
        return sci_fail(ctx, SCI_ERR_ARG, "bad prec");
    if (prec == SCI_PREC_F32_STORE_F64_ACC && ctx->cplx)
        return sci_fail(ctx, SCI_ERR_ARG, "FP32 storage is available for real Hamiltonians only");
    if (ctx->det_nvec > 0 && nvec > ctx->det_nvec)
        return sci_fail(ctx, SCI_ERR_ARG, "nvec exceeds the deterministic mode's max_nvec");
    if (ctx->M == 0) return SCI_OK;
    if (!C || !S) return sci_fail(ctx, SCI_ERR_ARG, "C or S is NULL");
    SCI_CK(cudaSetDevice(ctx->device));
    return sci_launch_sigma(ctx, C, S, nvec, prec);
}

extern "C" int sci_sigma_host(sci_ctx *ctx, const void *C_host, void *S_host, int nvec, int prec)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_dets || !ctx->have_ints) return sci_fail(ctx, SCI_ERR_STATE, "integrals and determinants needed");
    if (nvec < 1) return sci_fail(ctx, SCI_ERR_ARG, "nvec < 1");
    if (ctx->M == 0) return SCI_OK;
    if (!C_host || !S_host) return sci_fail(ctx, SCI_ERR_ARG, "C or S is NULL");
    if (prec != SCI_PREC_F64 && prec != SCI_PREC_F32_STORE_F64_ACC && prec != SCI_PREC_F64_DS)
        return sci_fail(ctx, SCI_ERR_ARG, "bad prec");
    SCI_CK(cudaSetDevice(ctx->device));
    size_t sb = ctx->cplx ? 16 : 8;
    size_t cb = (size_t)ctx->M * nvec * (prec == SCI_PREC_F32_STORE_F64_ACC ? 4 : sb);
    size_t obytes = (size_t)ctx->M * nvec * sb;
    size_t need = std::max(cb, obytes);
    if (need > ctx->stage_bytes) {
        if (ctx->stage_c) cudaFree(ctx->stage_c);
        if (ctx->stage_s) cudaFree(ctx->stage_s);
        ctx->stage_c = ctx->stage_s = nullptr;
        ctx->stage_bytes = 0;
        SCI_CK(cudaMalloc(&ctx->stage_c, need));
        SCI_CK(cudaMalloc(&ctx->stage_s, need));
        ctx->stage_bytes = need;
    }
    SCI_CK(cudaMemcpyAsync(ctx->stage_c, C_host, cb, cudaMemcpyHostToDevice, ctx->stream));
    int rc = sci_sigma(ctx, ctx->stage_c, ctx->stage_s, nvec, prec);
    if (rc != SCI_OK) return rc;
    if (ctx->ranged) {  // only the rows sigma computed; the rest of S_host is left alone
        const size_t off = (size_t)ctx->row_b * nvec * sb, len = (size_t)(ctx->row_e - ctx->row_b) * nvec * sb;
        if (len > 0)
            SCI_CK(cudaMemcpyAsync((char *)S_host + off, (char *)ctx->stage_s + off, len, cudaMemcpyDeviceToHost,
                                   ctx->stream));
    } else {
        SCI_CK(cudaMemcpyAsync(S_host, ctx->stage_s, obytes, cudaMemcpyDeviceToHost, ctx->stream));
    }
    SCI_CK(cudaStreamSynchronize(ctx->stream));
    return SCI_OK;
}

extern "C" int sci_profile(sci_ctx *ctx, int enable)
{
    if (!ctx) return SCI_ERR_ARG;
    SCI_CK(cudaSetDevice(ctx->device));
    if (enable)
        for (auto &e : ctx->ev)
            if (!e) SCI_CK(cudaEventCreate(&e));
    ctx->profile = enable ? 1 : 0;
    return SCI_OK;
}

extern "C" int sci_kernel_times(sci_ctx *ctx, float *ms, int n)
{
    if (!ctx || !ms || n < 0 || n > 4) return SCI_ERR_ARG;
    if (!ctx->ev[4]) return sci_fail(ctx, SCI_ERR_STATE, "profiling was never enabled");
    SCI_CK(cudaSetDevice(ctx->device));
    SCI_CK(cudaEventSynchronize(ctx->ev[4]));
    for (int i = 0; i < n; i++) SCI_CK(cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]));
    return SCI_OK;
}

extern "C" int sci_connections(sci_ctx *ctx, int64_t row_begin, int64_t row_end, int64_t *count, int64_t *rows,
                               int64_t *J, int8_t *degree, int8_t *phase, int64_t cap)
{
    if (!ctx || !count) return SCI_ERR_ARG;
    if (!ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "no determinants");
    if (row_begin < 0 || row_end > ctx->M || row_begin > row_end || cap < 0)
        return sci_fail(ctx, SCI_ERR_ARG, "bad row range or capacity");
    SCI_CK(cudaSetDevice(ctx->device));
    return sci_connections_device(ctx, row_begin, row_end, count, rows, J, degree, phase, cap);
}

extern "C" int sci_count_pairs(sci_ctx *ctx, int64_t *pairs)
{
    if (!ctx || !pairs) return SCI_ERR_ARG;
    if (!ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "no determinants");
    *pairs = ctx->ranged ? ctx->range_pairs : ctx->pairs;
    return SCI_OK;
}

extern "C" int sci_info(sci_ctx *ctx, int64_t *out, int n)
{
    if (!ctx || !out || n < 0 || n > 10) return SCI_ERR_ARG;
    const bool r = ctx->ranged;
    int64_t v[10] = {ctx->M, r ? ctx->range_pairs : ctx->pairs, ctx->e2, ctx->nb2, ctx->e1, ctx->nb1,
                     std::max(ctx->maxb1, ctx->maxb2), (int64_t)ctx->bytes_held, r ? ctx->range_pairs2 : ctx->pairs2,
                     r ? ctx->range_pairs1 : ctx->pairs1};
    for (int i = 0; i < n; i++) out[i] = v[i];
    return SCI_OK;
}

extern "C" int sci_sync_status(sci_ctx *ctx)
{
    if (!ctx) return SCI_ERR_ARG;
    SCI_CK(cudaSetDevice(ctx->device));
    int s = 0;
    SCI_CK(cudaMemcpyAsync(&s, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SCI_CK(cudaStreamSynchronize(ctx->stream));
    if (s & sci::DEV_OVERFLOW) return sci_fail(ctx, SCI_ERR_OVERFLOW, "device reported an overflow");
    if (s) return sci_fail(ctx, SCI_ERR_CUDA, "device status word set");
    return SCI_OK;
}

extern "C" const char *sci_last_error(const sci_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}
