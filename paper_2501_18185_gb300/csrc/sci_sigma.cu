// libsci hot path: sigma = H c (Sec. 2.4, the diagonalisation paragraph).
//
// sigma_I = H_II c_I + sum_{J single of I} H_IJ c_J + sum_{J double of I} H_IJ c_J,
// each off-diagonal element evaluated on the fly from the two occupation strings by the
// Slater-Condon rules (Sec. 2.3: matrix-element categories with 0, 1, 2 differences).
//
// Connection finding is done once at setup by bucketing: two determinants are within a
// double excitation exactly when they share an (N-2)-electron sub-string K, and they
// share exactly one such K when they differ by a double excitation.  So the doubles of
// the whole space are the disjoint pairs inside the buckets of equal K.  For a bra
// I = K + {a,b} and a ket J = K + {i,j} (a<b, i<j):
//     H_IJ = (-1)^(pi_I + pi_J) [(ai|bj) - (aj|bi)],
//     pi_X = #(K below x) + #(K below y) for the extras {x,y} of X,
// since applying a_j, a_i, a+_a, a+_b to J passes pi_J + pi_I + 2 occupied orbitals.
// Singles are the pairs inside the buckets of equal (N-1)-electron S:
//     H_IJ = (-1)^(pi_I + pi_J) [h_ai + sum_{k in S} ((ai|kk) - (ak|ki))],
// evaluated as F^ref_ai plus the terms of the orbitals where S and the reference differ
// (the closed-shell reference simplification of Sec. 2.3).
//
// Kernel shape (bucket-major, no tensor cores: this is a sparse gather).  A CTA owns
// the whole buckets that start in its range of CH table rows (its window), and stages
// every member of them in shared memory: the member's ket code, its ket offset into the
// pair-integral table and its coefficients pre-multiplied by (-1)^pi.  Each thread owns
// a row and walks the members of its bucket (in the FP64 kernels, the members other than
// the row itself); lanes of a warp that share a bucket read the same member, or one of
// two neighbours (a shared-memory broadcast), and nearby pair-table entries (the table
// stores bra indices fastest).  A row's partial sum is added to sigma with one FP64
// atomic add per (bucket, member).  Buckets too large to stage beside a window (above
// the tile threshold) are walked by k_doubles_tiled instead: 256 members of one bucket as
// the rows of a CTA, the whole bucket streamed through shared memory in column tiles.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "sci_bucket.cuh"
#include "sci_ds.cuh"
#include "sci_internal.cuh"

using sci::zdbl;

namespace {

// ------------------------------------------------------------------ scalar ops
// Sign flips are integer XORs of the sign bit: on GB300 the FP64 pipe is the scarce
// resource (1.2 TFLOP/s), so no FP64 instruction is spent on a negation.
__device__ __forceinline__ double flip(bool f, double a)
{
    return __longlong_as_double(__double_as_longlong(a) ^ ((unsigned long long)f << 63));
}
__device__ __forceinline__ float flip(bool f, float a) { return __int_as_float(__float_as_int(a) ^ ((int)f << 31)); }
__device__ __forceinline__ zdbl flip(bool f, zdbl a) { return zdbl{flip(f, a.x), flip(f, a.y)}; }
__device__ __forceinline__ float2 flip(bool f, float2 a) { return make_float2(flip(f, a.x), flip(f, a.y)); }
__device__ __forceinline__ float4 flip(bool f, float4 a)
{
    return make_float4(flip(f, a.x), flip(f, a.y), flip(f, a.z), flip(f, a.w));
}

__device__ __forceinline__ void zero(double &a) { a = 0.0; }
__device__ __forceinline__ void zero(zdbl &a) { a = zdbl{0.0, 0.0}; }

// acc += t * c
__device__ __forceinline__ void fma_acc(double &acc, double t, double c) { acc = fma(t, c, acc); }
__device__ __forceinline__ void fma_acc(zdbl &acc, zdbl t, zdbl c)
{
    acc.x = fma(t.x, c.x, acc.x);
    acc.x = fma(-t.y, c.y, acc.x);
    acc.y = fma(t.x, c.y, acc.y);
    acc.y = fma(t.y, c.x, acc.y);
}

__device__ __forceinline__ void red_add(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add(zdbl *p, zdbl v)
{
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
// The same, not sent when the sum is zero (rows whose bucket holds only single
// excitations of them sum to exactly 0, and adding +-0 leaves sigma unchanged).  The
// test reads the bits on the integer pipe.  Used where the atomics are the bound (FP32
// storage at several vectors: -4% there); elsewhere the branch costs more than it saves.
__device__ __forceinline__ void red_add_nz(double *p, double v)
{
    if ((__double_as_longlong(v) << 1) != 0) atomicAdd(p, v);
}

template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ zdbl ldg<zdbl>(const zdbl *p)
{
    double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return zdbl{v.x, v.y};
}

using sci::col_code;
using sci::disjoint;
using sci::row_code;
using sci::window;

// acc type for a storage type
template <typename TS> struct AccOf { using type = double; };
template <> struct AccOf<zdbl> { using type = zdbl; };

constexpr int kThreads = 256;
constexpr int kUnroll = 4;
// Rows per CTA.  Eight 256-thread CTAs fit an SM; what shared memory leaves of the
// 256 KB L1 for caching decides the speed (measured on the 2M-determinant space:
// 5.20 ms at 768 rows, 5.34 at 1024, 7.63 at 1280, where L1 is nearly gone).
constexpr int kRowsPerCta = 768;
// The FP32-storage kernel at 8 vectors (the mixed Davidson's block) stages 40 bytes per
// window row, so its window rows and its CTAs per SM (registers) are set apart.  Measured
// on the 2M-determinant space (doubles kernel, 8 vectors): 768 rows at 64 registers (4
// CTAs/SM by shared memory and registers) 15.84 ms; 512 rows at 5 CTAs/SM (48 registers,
// no spills) 14.88 ms; 448 rows at 6 (40 registers) 15.17 ms; 384 rows 15.57 ms.
#ifndef SCI_F32_ROWS
#define SCI_F32_ROWS 512
#endif
#ifndef SCI_F32_MINB
#define SCI_F32_MINB 5
#endif

// ------------------------------------------------------------------ row ranges
// A RANGED launch walks the range tables of sci_set_row_range() and computes only the
// members whose determinant lies in [rr.rb, rr.re).  Its CTA lists those rows of its
// window, in window order, in shared memory (a ballot per warp and a prefix over the
// warps), so that the lanes of a warp still own neighbouring rows of equal-size buckets;
// a window with no such row returns before staging anything.  Returns the row count.
__device__ __forceinline__ int owned_rows(const uint32_t *__restrict__ e_idx, int64_t r0, int W, sci::RowRange rr,
                                          uint16_t *s_own)
{
    __shared__ int s_wcnt[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int total = 0;
    for (int base = 0; base < W; base += blockDim.x) {
        const int q = base + (int)threadIdx.x;
        bool own = false;
        if (q < W) {
            const int64_t I = e_idx[r0 + q];
            own = I >= rr.rb && I < rr.re;
        }
        const unsigned m = __ballot_sync(0xffffffffu, own);
        if (lane == 0) s_wcnt[wid] = __popc(m);
        __syncthreads();
        int off = total, tot = total;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            const int c = s_wcnt[w];
            off += w < wid ? c : 0;
            tot += c;
        }
        if (own) s_own[off + __popc(m & ((1u << lane) - 1u))] = (uint16_t)q;
        total = tot;
        __syncthreads();
    }
    return total;
}

// ------------------------------------------------------------------ sigma = diag * c
// rows [row0, row0 + nrows) of S = H_II C
template <typename TC, typename TA>
__global__ void k_sigma_init(const double *__restrict__ hdiag, const TC *__restrict__ C, TA *__restrict__ S,
                             int64_t row0, int64_t nrows, int nvec)
{
    const int64_t total = nrows * nvec;
    C += row0 * nvec;
    S += row0 * nvec;
    hdiag += row0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        double h = hdiag[t / nvec];
        TA s;
        zero(s);
        if constexpr (sizeof(TC) == sizeof(zdbl)) {
            zdbl c = C[t];
            s = TA{h * c.x, h * c.y};
        } else {
            s = (TA)(h * (double)C[t]);
        }
        S[t] = s;
    }
}

// ------------------------------------------------------------------ doubles (FP64)
// TS: storage type of tab and staged coefficients; TA: accumulator (FP64 / complex128).
// Shared memory per staged member: (ket code, ket table offset) as uint2, and its NV
// coefficients times (-1)^pi.
template <typename TS, typename TC, int NV, bool RANGED, bool STORE = false>
__global__ void __launch_bounds__(kThreads)
k_doubles(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code, const uint32_t *__restrict__ e_pos,
          int64_t E, int CH, sci::TabRule tr, const TS *__restrict__ tab, const TC *__restrict__ C, int nvec, int v0,
          typename AccOf<TS>::type *__restrict__ Sout, sci::RowRange rr, const uint32_t *__restrict__ slot)
{
    using TA = typename AccOf<TS>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t r0, r1;
    window(e_pos, E, CH, r0, r1);
    if (r0 >= r1) return;
    const int W = (int)(r1 - r0);
    TS *s_c = reinterpret_cast<TS *>(smem);
    const size_t cbytes = ((size_t)W * NV * sizeof(TS) + 15) & ~(size_t)15;
    uint2 *s_kc = reinterpret_cast<uint2 *>(smem + cbytes);
    uint16_t *s_own = reinterpret_cast<uint16_t *>(smem + cbytes + (size_t)W * sizeof(uint2));
    int nrows = W;
    if constexpr (RANGED) {
        nrows = owned_rows(e_idx, r0, W, rr, s_own);
        if (nrows == 0) return;
    }

    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        const int64_t g = r0 + q;
        const uint32_t idx = e_idx[g], code = e_code[g];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        s_kc[q] = make_uint2(col_code(code), colbase);
        const bool par = sci::code_par(code);
#pragma unroll
        for (int v = 0; v < NV; v++) s_c[q * NV + v] = flip(par, (TS)C[(int64_t)idx * nvec + v0 + v]);
    }
    __syncthreads();

    for (int t_ = threadIdx.x; t_ < nrows; t_ += blockDim.x) {
        const int q0 = RANGED ? (int)s_own[t_] : t_;
        const uint32_t code = e_code[r0 + q0], pos = e_pos[r0 + q0];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        const int bs = q0 - sci::pos_off(pos), je = bs + sci::pos_size(pos) - 1;
        const uint32_t rc = row_code(code);
        const TS *trow = tab + rowoff;
        TA acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) zero(acc[v]);
        // the members other than the row itself: j in [bs, je) stands for bucket position
        // j + (j >= q0), so rows of equal bucket size (windows hold buckets of one size,
        // largest first) run the same trip count and no FP64 FMA is spent on the row (one
        // in 3.5 members on average).  Groups of kUnroll members: a group with no double
        // of this row (single excitations of it) is skipped, and so is the whole warp's
        // work when no lane has one; otherwise up to kUnroll table loads are in flight per
        // thread and a non-double member contributes t = 0
        int j = bs;
        for (; j + kUnroll <= je; j += kUnroll) {
            uint2 kc[kUnroll];
            TS t[kUnroll];
            unsigned vm = 0;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                kc[u] = s_kc[j + u + (j + u >= q0)];
                vm |= (unsigned)disjoint(rc, kc[u].x) << u;
            }
            if (vm == 0) continue;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                zero(t[u]);
                if (vm & (1u << u)) t[u] = ldg(trow + kc[u].y);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++)
#pragma unroll
                for (int v = 0; v < NV; v++) fma_acc(acc[v], t[u], s_c[(j + u + (j + u >= q0)) * NV + v]);
        }
        for (; j < je; j++) {
            const int m = j + (j >= q0);
            const uint2 kc = s_kc[m];
            if (!disjoint(rc, kc.x)) continue;
            const TS t = ldg(trow + kc.y);
#pragma unroll
            for (int v = 0; v < NV; v++) fma_acc(acc[v], t, s_c[m * NV + v]);
        }
        const bool par = sci::code_par(code);
        if constexpr (STORE) {   // the row sum to this entry's slot (summed per row later)
#pragma unroll
            for (int v = 0; v < NV; v++) Sout[(int64_t)slot[r0 + q0] * nvec + v0 + v] = flip(par, acc[v]);
        } else {
            const uint32_t idx = e_idx[r0 + q0];
#pragma unroll
            for (int v = 0; v < NV; v++) red_add(Sout + (int64_t)idx * nvec + v0 + v, flip(par, acc[v]));
        }
    }
}

// ------------------------------------------------------------------ doubles, paired FP32
// The same bucket walk with the products and per-row sums in "double-single" arithmetic
// on the FP32 pipes: an FP64 value x is carried as hi + lo with hi = fl32(x) and
// lo = fl32(x - hi).  For t = th + tl and c = ch + cl the product is
//     p = fl(th*ch),  e = (th*ch - p) + th*cl + tl*ch      (exact first term via FMA;
// the dropped tl*cl is ~2^-48 of |tc|), and the sum (hi, lo) takes p by TwoSum
// (Knuth) with e and the rounding error folded into lo.  lo is renormalised into hi every
// kUnroll pairs.  The row sum leaves the kernel as fp64(hi) + fp64(lo) through the same
// FP64 atomic add as the FP64 path.
using sci::Ds;
using sci::ds_fma;
using sci::ds_renorm;
using sci::ds_value;
using sci::ds_zero;
using sci::f2d_int;

__device__ __forceinline__ float2 ds_split(double x)
{
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

__device__ __forceinline__ float2 ds_split(float x) { return make_float2(x, 0.f); }

// split the vector group C[:, v0:v0+G] into paired floats, once per sigma call (so the
// staging in the bucket kernel, which touches each coefficient many times, only copies)
template <typename TC>
__global__ void k_split_c(const TC *__restrict__ C, int64_t M, int nvec, int v0, int G, float2 *__restrict__ out)
{
    const int64_t total = M * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = ds_split(C[(t / G) * nvec + v0 + t % G]);
}

// a += t * c for FP32 t and c: the product is exact as p + e (e by FMA), the sum is
// compensated as in ds_fma
__device__ __forceinline__ void ds_fma1(Ds &a, float t, float c)
{
    const float p = t * c;
    const float e = fmaf(t, c, -p);
    const float s = a.hi + p;
    const float bv = s - a.hi;
    const float err = (a.hi - (s - bv)) + (p - bv);
    a.lo += err + e;
    a.hi = s;
}

// FP32 storage: the pair table rounded to FP32 (tab32) and FP32 coefficients, exact
// products, compensated bucket sums, FP64 accumulation into sigma
template <int NV, bool RANGED, bool STORE = false>
__global__ void __launch_bounds__(kThreads, NV >= 8 ? SCI_F32_MINB : 1)
k_doubles_f32(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
              const uint32_t *__restrict__ e_pos, int64_t E, int CH, sci::TabRule tr,
              const float *__restrict__ tab32, const float *__restrict__ C, int nvec, int v0,
              double *__restrict__ Sout, sci::RowRange rr, const uint32_t *__restrict__ slot)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t r0, r1;
    window(e_pos, E, CH, r0, r1);
    if (r0 >= r1) return;
    const int W = (int)(r1 - r0);
    float *s_c = reinterpret_cast<float *>(smem);
    const size_t cbytes = ((size_t)W * NV * sizeof(float) + 15) & ~(size_t)15;
    uint2 *s_kc = reinterpret_cast<uint2 *>(smem + cbytes);
    uint16_t *s_own = reinterpret_cast<uint16_t *>(smem + cbytes + (size_t)W * sizeof(uint2));
    int nrows = W;
    if constexpr (RANGED) {
        nrows = owned_rows(e_idx, r0, W, rr, s_own);
        if (nrows == 0) return;
    }

    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        const int64_t g = r0 + q;
        const uint32_t idx = e_idx[g], code = e_code[g];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        s_kc[q] = make_uint2(col_code(code), colbase);
        const bool par = sci::code_par(code);
#pragma unroll
        for (int v = 0; v < NV; v++) s_c[q * NV + v] = flip(par, C[(int64_t)idx * nvec + v0 + v]);
    }
    __syncthreads();

    for (int t_ = threadIdx.x; t_ < nrows; t_ += blockDim.x) {
        const int q0 = RANGED ? (int)s_own[t_] : t_;
        const uint32_t code = e_code[r0 + q0], pos = e_pos[r0 + q0];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        const int bs = q0 - sci::pos_off(pos), be = bs + sci::pos_size(pos);
        const uint32_t rc = row_code(code);
        const float *trow = tab32 + rowoff;
        Ds acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) ds_zero(acc[v]);
        // all members, the row itself included (t = 0): this kernel is bound by its FP64
        // atomics, and the aligned walk keeps lanes of one bucket on the same member
        int j = bs;
        for (; j + kUnroll <= be; j += kUnroll) {
            uint2 kc[kUnroll];
            float t[kUnroll];
            unsigned vm = 0;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                kc[u] = s_kc[j + u];
                vm |= (unsigned)disjoint(rc, kc[u].x) << u;
            }
            if (vm == 0) continue;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                t[u] = 0.f;
                if (vm & (1u << u)) t[u] = __ldg(trow + kc[u].y);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++)
#pragma unroll
                for (int v = 0; v < NV; v++) ds_fma1(acc[v], t[u], s_c[(j + u) * NV + v]);
#pragma unroll
            for (int v = 0; v < NV; v++) ds_renorm(acc[v]);
        }
        for (; j < be; j++) {
            const uint2 kc = s_kc[j];
            if (!disjoint(rc, kc.x)) continue;
            const float t = __ldg(trow + kc.y);
#pragma unroll
            for (int v = 0; v < NV; v++) ds_fma1(acc[v], t, s_c[j * NV + v]);
        }
        const bool par = sci::code_par(code);
        if constexpr (STORE) {
#pragma unroll
            for (int v = 0; v < NV; v++) Sout[(int64_t)slot[r0 + q0] * nvec + v0 + v] = flip(par, ds_value(acc[v]));
        } else {
            const uint32_t idx = e_idx[r0 + q0];
#pragma unroll
            for (int v = 0; v < NV; v++) red_add_nz(Sout + (int64_t)idx * nvec + v0 + v, flip(par, ds_value(acc[v])));
        }
    }
}

__global__ void k_split_cz(const zdbl *__restrict__ C, int64_t M, int nvec, int v0, int G, float4 *__restrict__ out)
{
    const int64_t total = M * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const zdbl c = C[(t / G) * nvec + v0 + t % G];
        const float2 re = ds_split(c.x), im = ds_split(c.y);
        out[t] = make_float4(re.x, re.y, im.x, im.y);
    }
}

// real: tab2 is the (hi, lo) split of the pair table, C2 the split vector group
template <int NV, bool RANGED, bool STORE = false>
__global__ void __launch_bounds__(kThreads)
k_doubles_ds(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
             const uint32_t *__restrict__ e_pos, int64_t E, int CH, sci::TabRule tr,
             const float2 *__restrict__ tab2, const float2 *__restrict__ C2, int nvec, int v0,
             double *__restrict__ Sout, sci::RowRange rr, const uint32_t *__restrict__ slot)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t r0, r1;
    window(e_pos, E, CH, r0, r1);
    if (r0 >= r1) return;
    const int W = (int)(r1 - r0);
    float2 *s_c = reinterpret_cast<float2 *>(smem);
    const size_t cbytes = ((size_t)W * NV * sizeof(float2) + 15) & ~(size_t)15;
    uint2 *s_kc = reinterpret_cast<uint2 *>(smem + cbytes);
    uint16_t *s_own = reinterpret_cast<uint16_t *>(smem + cbytes + (size_t)W * sizeof(uint2));
    int nrows = W;
    if constexpr (RANGED) {
        nrows = owned_rows(e_idx, r0, W, rr, s_own);
        if (nrows == 0) return;
    }

    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        const int64_t g = r0 + q;
        const uint32_t idx = e_idx[g], code = e_code[g];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        s_kc[q] = make_uint2(col_code(code), colbase);
        const bool par = sci::code_par(code);
#pragma unroll
        for (int v = 0; v < NV; v++) s_c[q * NV + v] = flip(par, C2[(int64_t)idx * NV + v]);
    }
    __syncthreads();

    for (int t_ = threadIdx.x; t_ < nrows; t_ += blockDim.x) {
        const int q0 = RANGED ? (int)s_own[t_] : t_;
        const uint32_t code = e_code[r0 + q0], pos = e_pos[r0 + q0];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        const int bs = q0 - sci::pos_off(pos), be = bs + sci::pos_size(pos);
        const uint32_t rc = row_code(code);
        const float2 *trow = tab2 + rowoff;
        Ds acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) ds_zero(acc[v]);
        // all members, the row itself included (it contributes t = 0): lanes of one bucket
        // then read the same member and neighbouring table entries at every step, which
        // this LSU-bound kernel needs more than the skipped arithmetic
        int j = bs;
        for (; j + kUnroll <= be; j += kUnroll) {
            uint2 kc[kUnroll];
            float2 t[kUnroll];
            unsigned vm = 0;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                kc[u] = s_kc[j + u];
                vm |= (unsigned)disjoint(rc, kc[u].x) << u;
            }
            if (vm == 0) continue;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                t[u] = make_float2(0.f, 0.f);
                if (vm & (1u << u)) t[u] = __ldg(trow + kc[u].y);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++)
#pragma unroll
                for (int v = 0; v < NV; v++) ds_fma(acc[v], t[u], s_c[(j + u) * NV + v]);
#pragma unroll
            for (int v = 0; v < NV; v++) ds_renorm(acc[v]);
        }
        for (; j < be; j++) {
            const uint2 kc = s_kc[j];
            if (!disjoint(rc, kc.x)) continue;
            const float2 t = __ldg(trow + kc.y);
#pragma unroll
            for (int v = 0; v < NV; v++) ds_fma(acc[v], t, s_c[j * NV + v]);
        }
        const bool par = sci::code_par(code);
        if constexpr (STORE) {
#pragma unroll
            for (int v = 0; v < NV; v++) Sout[(int64_t)slot[r0 + q0] * nvec + v0 + v] = flip(par, ds_value(acc[v]));
        } else {
            const uint32_t idx = e_idx[r0 + q0];
#pragma unroll
            for (int v = 0; v < NV; v++) red_add(Sout + (int64_t)idx * nvec + v0 + v, flip(par, ds_value(acc[v])));
        }
    }
}

// complex: tab4 holds (re_hi, re_lo, im_hi, im_lo); C4 the split vector group
template <int NV, bool RANGED, bool STORE = false>
__global__ void __launch_bounds__(kThreads)
k_doubles_dsz(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
              const uint32_t *__restrict__ e_pos, int64_t E, int CH, sci::TabRule tr,
              const float4 *__restrict__ tab4, const float4 *__restrict__ C4, int nvec, int v0, zdbl *__restrict__ Sout,
              sci::RowRange rr, const uint32_t *__restrict__ slot)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t r0, r1;
    window(e_pos, E, CH, r0, r1);
    if (r0 >= r1) return;
    const int W = (int)(r1 - r0);
    float4 *s_c = reinterpret_cast<float4 *>(smem);
    const size_t cbytes = ((size_t)W * NV * sizeof(float4) + 15) & ~(size_t)15;
    uint2 *s_kc = reinterpret_cast<uint2 *>(smem + cbytes);
    uint16_t *s_own = reinterpret_cast<uint16_t *>(smem + cbytes + (size_t)W * sizeof(uint2));
    int nrows = W;
    if constexpr (RANGED) {
        nrows = owned_rows(e_idx, r0, W, rr, s_own);
        if (nrows == 0) return;
    }

    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        const int64_t g = r0 + q;
        const uint32_t idx = e_idx[g], code = e_code[g];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        s_kc[q] = make_uint2(col_code(code), colbase);
        const bool par = sci::code_par(code);
#pragma unroll
        for (int v = 0; v < NV; v++) s_c[q * NV + v] = flip(par, C4[(int64_t)idx * NV + v]);
    }
    __syncthreads();

    for (int t_ = threadIdx.x; t_ < nrows; t_ += blockDim.x) {
        const int q0 = RANGED ? (int)s_own[t_] : t_;
        const uint32_t code = e_code[r0 + q0], pos = e_pos[r0 + q0];
        uint32_t rowoff, colbase;
        sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
        const int bs = q0 - sci::pos_off(pos), je = bs + sci::pos_size(pos) - 1;
        const uint32_t rc = row_code(code);
        const float4 *trow = tab4 + rowoff;
        Ds ar[NV], ai[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) ds_zero(ar[v]), ds_zero(ai[v]);
        int nused = 0;
        // the members other than the row itself (bucket position j + (j >= q0))
        for (int j = bs; j < je; j++) {
            const int m = j + (j >= q0);
            const uint2 kc = s_kc[m];
            if (!disjoint(rc, kc.x)) continue;
            const float4 t = __ldg(trow + kc.y);
            const float2 tr_ = make_float2(t.x, t.y), ti = make_float2(t.z, t.w);
            const float2 mti = make_float2(-t.z, -t.w);
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const float4 c = s_c[m * NV + v];
                const float2 cr = make_float2(c.x, c.y), ci = make_float2(c.z, c.w);
                ds_fma(ar[v], tr_, cr);
                ds_fma(ar[v], mti, ci);
                ds_fma(ai[v], tr_, ci);
                ds_fma(ai[v], ti, cr);
            }
            if ((++nused & 3) == 0)
#pragma unroll
                for (int v = 0; v < NV; v++) ds_renorm(ar[v]), ds_renorm(ai[v]);
        }
        const bool par = sci::code_par(code);
        if constexpr (STORE) {
#pragma unroll
            for (int v = 0; v < NV; v++)
                Sout[(int64_t)slot[r0 + q0] * nvec + v0 + v] = flip(par, zdbl{ds_value(ar[v]), ds_value(ai[v])});
        } else {
            const uint32_t idx = e_idx[r0 + q0];
#pragma unroll
            for (int v = 0; v < NV; v++)
                red_add(Sout + (int64_t)idx * nvec + v0 + v, flip(par, zdbl{ds_value(ar[v]), ds_value(ai[v])}));
        }
    }
}

// ------------------------------------------------------------------ doubles, tiled
// (N-2) buckets of more than tile_b members (sci_set_tile_threshold) are too large to
// stage whole beside a window, so they run here.  A CTA takes kTileRows consecutive
// members of one bucket as its rows (one per thread) and streams the bucket's members
// through shared memory in column tiles, each staged once per CTA; every thread walks a
// column tile against its row as the window kernels walk a bucket (disjointness test, one
// table load per double, the FMAs), so a row sums the same products.  The row itself and
// its single excitations fail the disjointness test and add nothing.  All threads of a
// CTA share the bucket, so trip counts are uniform and the barriers are CTA-wide.
// The arithmetic is a policy: staged element SC, table element TT, accumulator ACC,
// output TO, input coefficients CI; how a coefficient is read, multiplied in,
// renormalised (paired FP32) and written out.
template <typename TS, typename TC> struct PolF64 {   // FP64 / complex128 (the k_doubles arithmetic)
    using SC = TS;
    using TT = TS;
    using ACC = typename AccOf<TS>::type;
    using TO = ACC;
    using CI = TC;
    __device__ static SC load(const CI *C, int64_t i) { return (SC)C[i]; }
    __device__ static TT table(const TT *p) { return ldg(p); }
    __device__ static void clear(ACC &a) { zero(a); }
    __device__ static void mul_add(ACC &a, TT t, SC c) { fma_acc(a, t, c); }
    __device__ static void renorm(ACC &) {}
    __device__ static TO value(const ACC &a) { return a; }
    __device__ static void add_out(TO *p, TO v) { red_add(p, v); }
};
struct PolDS {   // paired FP32, real (the k_doubles_ds arithmetic)
    using SC = float2;
    using TT = float2;
    using ACC = Ds;
    using TO = double;
    using CI = float2;
    __device__ static SC load(const CI *C, int64_t i) { return C[i]; }
    __device__ static TT table(const TT *p) { return __ldg(p); }
    __device__ static void clear(ACC &a) { ds_zero(a); }
    __device__ static void mul_add(ACC &a, TT t, SC c) { ds_fma(a, t, c); }
    __device__ static void renorm(ACC &a) { ds_renorm(a); }
    __device__ static TO value(const ACC &a) { return ds_value(a); }
    __device__ static void add_out(TO *p, TO v) { red_add(p, v); }
};
struct PolF32 {   // FP32 storage, paired-FP32 sums (the k_doubles_f32 arithmetic)
    using SC = float;
    using TT = float;
    using ACC = Ds;
    using TO = double;
    using CI = float;
    __device__ static SC load(const CI *C, int64_t i) { return C[i]; }
    __device__ static TT table(const TT *p) { return __ldg(p); }
    __device__ static void clear(ACC &a) { ds_zero(a); }
    __device__ static void mul_add(ACC &a, TT t, SC c);
    __device__ static void renorm(ACC &a) { ds_renorm(a); }
    __device__ static TO value(const ACC &a) { return ds_value(a); }
    __device__ static void add_out(TO *p, TO v) { red_add_nz(p, v); }
};
__device__ __forceinline__ void PolF32::mul_add(Ds &a, float t, float c) { ds_fma1(a, t, c); }
struct DsZ {
    Ds r, i;
};
struct PolDSZ {   // paired FP32, complex (the k_doubles_dsz arithmetic)
    using SC = float4;
    using TT = float4;
    using ACC = DsZ;
    using TO = zdbl;
    using CI = float4;
    __device__ static SC load(const CI *C, int64_t i) { return C[i]; }
    __device__ static TT table(const TT *p) { return __ldg(p); }
    __device__ static void clear(ACC &a) { ds_zero(a.r), ds_zero(a.i); }
    __device__ static void mul_add(ACC &a, TT t, SC c)
    {
        const float2 tr_ = make_float2(t.x, t.y), ti = make_float2(t.z, t.w), mti = make_float2(-t.z, -t.w);
        const float2 cr = make_float2(c.x, c.y), ci = make_float2(c.z, c.w);
        ds_fma(a.r, tr_, cr);
        ds_fma(a.r, mti, ci);
        ds_fma(a.i, tr_, ci);
        ds_fma(a.i, ti, cr);
    }
    __device__ static void renorm(ACC &a) { ds_renorm(a.r), ds_renorm(a.i); }
    __device__ static TO value(const ACC &a) { return zdbl{ds_value(a.r), ds_value(a.i)}; }
    __device__ static void add_out(TO *p, TO v) { red_add(p, v); }
};

// shared memory of the tiled kernel: at most this, which needs no opt-in
constexpr size_t kTiledSmem = 48 * 1024;

// C holds coefficient v of determinant I at C[I * cstride + coff + v].  With few tiles
// (a handful of very large buckets) the columns of a bucket are also split: CTA row y of
// the grid (gridDim.y = nsplit) takes the y-th of nsplit equal runs of column tiles and
// adds its partial row sums atomically (nsplit = 1 in the deterministic mode, where one
// CTA writes a slot).
template <class P, int NV, bool RANGED, bool STORE>
__global__ void __launch_bounds__(kThreads)
k_doubles_tiled(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
                const uint32_t *__restrict__ e_pos, const uint32_t *__restrict__ tiles, int64_t ntiles, int TCOL,
                sci::TabRule tr, const typename P::TT *__restrict__ tab, const typename P::CI *__restrict__ C,
                int cstride, int coff, int nvec, int v0, typename P::TO *__restrict__ Sout, sci::RowRange rr,
                const uint32_t *__restrict__ slot)
{
    const int nsplit = STORE ? 1 : (int)gridDim.y;
    using SC = typename P::SC;
    using TT = typename P::TT;
    using ACC = typename P::ACC;
    extern __shared__ __align__(16) unsigned char smem[];
    SC *s_c = reinterpret_cast<SC *>(smem);
    uint2 *s_kc = reinterpret_cast<uint2 *>(smem + (((size_t)TCOL * NV * sizeof(SC) + 15) & ~(size_t)15));
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = tiles[t];
        const uint32_t pos0 = e_pos[r0];
        const int64_t bs = r0 - sci::pos_off(pos0);
        const int bsize = sci::pos_size(pos0);
        // this CTA's column tiles: [c_lo, c_hi) in members of the bucket
        const int nct = (bsize + TCOL - 1) / TCOL, per_split = (nct + nsplit - 1) / nsplit;
        const int c_lo = (int)blockIdx.y * per_split * TCOL, c_hi = min(bsize, c_lo + per_split * TCOL);
        if (c_lo >= c_hi) continue;   // uniform over the CTA
        const int64_t row = r0 + threadIdx.x;
        bool active = row < bs + bsize;
        if (RANGED && active) {
            const int64_t I = e_idx[row];
            active = I >= rr.rb && I < rr.re;
        }
        if (!__syncthreads_or(active)) continue;   // no row of this tile is computed
        uint32_t rc = 0;
        const TT *trow = tab;
        bool par = false;
        if (active) {
            const uint32_t code = e_code[row];
            uint32_t rowoff, colbase;
            sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
            rc = row_code(code);
            trow = tab + rowoff;
            par = sci::code_par(code);
        }
        ACC acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) P::clear(acc[v]);
        for (int cs = c_lo; cs < c_hi; cs += TCOL) {
            const int n = min(TCOL, c_hi - cs);
            __syncthreads();   // every thread is done with the previous column tile
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                const int64_t g = bs + cs + q;
                const uint32_t idx = e_idx[g], code = e_code[g];
                uint32_t rowoff, colbase;
                sci::pair_offsets(tr, sci::code_x(code), sci::code_y(code), rowoff, colbase);
                s_kc[q] = make_uint2(col_code(code), colbase);
                const bool pq = sci::code_par(code);
#pragma unroll
                for (int v = 0; v < NV; v++) s_c[q * NV + v] = flip(pq, P::load(C, (int64_t)idx * cstride + coff + v));
            }
            __syncthreads();
            if (!active) continue;
            int j = 0;
            for (; j + kUnroll <= n; j += kUnroll) {
                uint2 kc[kUnroll];
                TT tv[kUnroll];
                unsigned vm = 0;
#pragma unroll
                for (int u = 0; u < kUnroll; u++) {
                    kc[u] = s_kc[j + u];
                    vm |= (unsigned)disjoint(rc, kc[u].x) << u;
                }
                if (vm == 0) continue;
#pragma unroll
                for (int u = 0; u < kUnroll; u++) {
                    tv[u] = TT{};
                    if (vm & (1u << u)) tv[u] = P::table(trow + kc[u].y);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; u++)
#pragma unroll
                    for (int v = 0; v < NV; v++) P::mul_add(acc[v], tv[u], s_c[(j + u) * NV + v]);
#pragma unroll
                for (int v = 0; v < NV; v++) P::renorm(acc[v]);
            }
            for (; j < n; j++) {
                const uint2 kc = s_kc[j];
                if (!disjoint(rc, kc.x)) continue;
                const TT tv = P::table(trow + kc.y);
#pragma unroll
                for (int v = 0; v < NV; v++) P::mul_add(acc[v], tv, s_c[j * NV + v]);
            }
#pragma unroll
            for (int v = 0; v < NV; v++) P::renorm(acc[v]);
        }
        if (active) {
            if constexpr (STORE) {
#pragma unroll
                for (int v = 0; v < NV; v++) Sout[(int64_t)slot[row] * nvec + v0 + v] = flip(par, P::value(acc[v]));
            } else {
                const uint32_t idx = e_idx[row];
#pragma unroll
                for (int v = 0; v < NV; v++) P::add_out(Sout + (int64_t)idx * nvec + v0 + v, flip(par, P::value(acc[v])));
            }
        }
    }
}

// ------------------------------------------------------------------ singles
template <typename TS, typename TC, int NV, bool RANGED, bool STORE = false, int KW = 1>
__global__ void __launch_bounds__(kThreads)
k_singles(const uint32_t *__restrict__ e_idx, const uint64_t *__restrict__ e_S, const uint32_t *__restrict__ e_meta,
          int64_t E, int norb, sci::RefW ref, const TS *__restrict__ fref, const TS *__restrict__ g_so,
          const TC *__restrict__ C, int nvec, int v0, typename AccOf<TS>::type *__restrict__ Sout, sci::RowRange rr, const uint32_t *__restrict__ slot)
{
    using TA = typename AccOf<TS>::type;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (RANGED) {
            const int64_t I = e_idx[p];
            if (I < rr.rb || I >= rr.re) continue;
        }
        const uint32_t meta = e_meta[p];
        const int a = sci::meta_x(meta);
        const bool par = sci::meta_par(meta);
        const int64_t bs = p - (int64_t)sci::meta_off(meta);
        const int64_t be = bs + (int64_t)sci::meta_size(meta);
        uint64_t part[KW], holes[KW];   // S \ ref and ref \ S, word w holding orbitals 64w..64w+63
#pragma unroll
        for (int w_ = 0; w_ < KW; w_++) {
            const uint64_t Sw = e_S[p * KW + w_], rw = ref.w[w_];
            part[w_] = Sw & ~rw, holes[w_] = rw & ~Sw;
        }
        TA acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) zero(acc[v]);
        for (int64_t q = bs; q < be; q++) {
            if (q == p) continue;
            const uint32_t mq = e_meta[q];
            const int i = sci::meta_x(mq);
            const bool parq = sci::meta_par(mq);
            const uint32_t idxq = e_idx[q];
            TS f = ldg(fref + i * norb + a);
#pragma unroll
            for (int w_ = 0; w_ < KW; w_++)
            for (uint64_t m = part[w_]; m; m &= m - 1) {
                int k = 64 * w_ + __ffsll((long long)m) - 1;
                TS g = ldg(g_so + ((int64_t)k * norb + i) * norb + a);
                if constexpr (sizeof(TS) == sizeof(zdbl)) { f.x += g.x; f.y += g.y; } else { f += g; }
            }
#pragma unroll
            for (int w_ = 0; w_ < KW; w_++)
            for (uint64_t m = holes[w_]; m; m &= m - 1) {
                int k = 64 * w_ + __ffsll((long long)m) - 1;
                TS g = ldg(g_so + ((int64_t)k * norb + i) * norb + a);
                if constexpr (sizeof(TS) == sizeof(zdbl)) { f.x -= g.x; f.y -= g.y; } else { f -= g; }
            }
#pragma unroll
            for (int v = 0; v < NV; v++) fma_acc(acc[v], f, flip(parq, C[(int64_t)idxq * nvec + v0 + v]));
        }
        if constexpr (STORE) {
#pragma unroll
            for (int v = 0; v < NV; v++) Sout[(int64_t)slot[p] * nvec + v0 + v] = flip(par, acc[v]);
        } else {
            const uint32_t idx = e_idx[p];
#pragma unroll
            for (int v = 0; v < NV; v++) red_add(Sout + (int64_t)idx * nvec + v0 + v, flip(par, acc[v]));
        }
    }
}

// ------------------------------------------------------------------ singles, paired FP32
// F^S_ai = F^ref_ai + sum_{k in S\ref} g_ai(k) - sum_{k in ref\S} g_ai(k) summed in
// paired FP32 from split copies of fref and g_so, then multiplied into the row sum like
// the doubles.  C2/C4 is the split vector group (row stride NV).
using sci::ds_add;

template <int NV, bool RANGED, bool STORE = false, int KW = 1>
__global__ void __launch_bounds__(kThreads)
k_singles_ds(const uint32_t *__restrict__ e_idx, const uint64_t *__restrict__ e_S, const uint32_t *__restrict__ e_meta,
             int64_t E, int norb, sci::RefW ref, const float2 *__restrict__ fref2, const float2 *__restrict__ g2,
             const float2 *__restrict__ C2, int nvec, int v0, double *__restrict__ Sout, sci::RowRange rr, const uint32_t *__restrict__ slot)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (RANGED) {
            const int64_t I = e_idx[p];
            if (I < rr.rb || I >= rr.re) continue;
        }
        const uint32_t meta = e_meta[p];
        const int a = sci::meta_x(meta);
        const bool par = sci::meta_par(meta);
        const int64_t bs = p - (int64_t)sci::meta_off(meta);
        const int64_t be = bs + (int64_t)sci::meta_size(meta);
        uint64_t part[KW], holes[KW];   // S \ ref and ref \ S, word w holding orbitals 64w..64w+63
#pragma unroll
        for (int w_ = 0; w_ < KW; w_++) {
            const uint64_t Sw = e_S[p * KW + w_], rw = ref.w[w_];
            part[w_] = Sw & ~rw, holes[w_] = rw & ~Sw;
        }
        Ds acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) ds_zero(acc[v]);
        for (int64_t q = bs; q < be; q++) {
            if (q == p) continue;
            const uint32_t mq = e_meta[q];
            const int i = sci::meta_x(mq);
            const bool parq = sci::meta_par(mq);
            const uint32_t idxq = e_idx[q];
            const float2 f0 = __ldg(fref2 + i * norb + a);
            Ds f{f0.x, f0.y};
#pragma unroll
            for (int w_ = 0; w_ < KW; w_++)
            for (uint64_t m = part[w_]; m; m &= m - 1) {
                const int k = 64 * w_ + __ffsll((long long)m) - 1;
                ds_add(f, __ldg(g2 + ((int64_t)k * norb + i) * norb + a));
            }
#pragma unroll
            for (int w_ = 0; w_ < KW; w_++)
            for (uint64_t m = holes[w_]; m; m &= m - 1) {
                const int k = 64 * w_ + __ffsll((long long)m) - 1;
                ds_add(f, flip(true, __ldg(g2 + ((int64_t)k * norb + i) * norb + a)));
            }
            ds_renorm(f);
            const float2 fv = make_float2(f.hi, f.lo);
#pragma unroll
            for (int v = 0; v < NV; v++) ds_fma(acc[v], fv, flip(parq, C2[(int64_t)idxq * NV + v]));
        }
        if constexpr (STORE) {
#pragma unroll
            for (int v = 0; v < NV; v++) Sout[(int64_t)slot[p] * nvec + v0 + v] = flip(par, ds_value(acc[v]));
        } else {
            const uint32_t idx = e_idx[p];
#pragma unroll
            for (int v = 0; v < NV; v++) red_add(Sout + (int64_t)idx * nvec + v0 + v, flip(par, ds_value(acc[v])));
        }
    }
}

template <int NV, bool RANGED, bool STORE = false, int KW = 1>
__global__ void __launch_bounds__(kThreads)
k_singles_dsz(const uint32_t *__restrict__ e_idx, const uint64_t *__restrict__ e_S,
              const uint32_t *__restrict__ e_meta, int64_t E, int norb, sci::RefW ref,
              const float4 *__restrict__ fref4, const float4 *__restrict__ g4, const float4 *__restrict__ C4,
              int nvec, int v0, zdbl *__restrict__ Sout, sci::RowRange rr, const uint32_t *__restrict__ slot)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (RANGED) {
            const int64_t I = e_idx[p];
            if (I < rr.rb || I >= rr.re) continue;
        }
        const uint32_t meta = e_meta[p];
        const int a = sci::meta_x(meta);
        const bool par = sci::meta_par(meta);
        const int64_t bs = p - (int64_t)sci::meta_off(meta);
        const int64_t be = bs + (int64_t)sci::meta_size(meta);
        uint64_t part[KW], holes[KW];   // S \ ref and ref \ S, word w holding orbitals 64w..64w+63
#pragma unroll
        for (int w_ = 0; w_ < KW; w_++) {
            const uint64_t Sw = e_S[p * KW + w_], rw = ref.w[w_];
            part[w_] = Sw & ~rw, holes[w_] = rw & ~Sw;
        }
        Ds ar[NV], ai[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) ds_zero(ar[v]), ds_zero(ai[v]);
        for (int64_t q = bs; q < be; q++) {
            if (q == p) continue;
            const uint32_t mq = e_meta[q];
            const int i = sci::meta_x(mq);
            const bool parq = sci::meta_par(mq);
            const uint32_t idxq = e_idx[q];
            const float4 f0 = __ldg(fref4 + i * norb + a);
            Ds fr{f0.x, f0.y}, fi{f0.z, f0.w};
#pragma unroll
            for (int w_ = 0; w_ < KW; w_++)
            for (uint64_t m = part[w_]; m; m &= m - 1) {
                const int k = 64 * w_ + __ffsll((long long)m) - 1;
                const float4 g = __ldg(g4 + ((int64_t)k * norb + i) * norb + a);
                ds_add(fr, make_float2(g.x, g.y));
                ds_add(fi, make_float2(g.z, g.w));
            }
#pragma unroll
            for (int w_ = 0; w_ < KW; w_++)
            for (uint64_t m = holes[w_]; m; m &= m - 1) {
                const int k = 64 * w_ + __ffsll((long long)m) - 1;
                const float4 g = flip(true, __ldg(g4 + ((int64_t)k * norb + i) * norb + a));
                ds_add(fr, make_float2(g.x, g.y));
                ds_add(fi, make_float2(g.z, g.w));
            }
            ds_renorm(fr);
            ds_renorm(fi);
            const float2 tr_ = make_float2(fr.hi, fr.lo), ti = make_float2(fi.hi, fi.lo);
            const float2 mti = make_float2(-fi.hi, -fi.lo);
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const float4 c = flip(parq, C4[(int64_t)idxq * NV + v]);
                const float2 cr = make_float2(c.x, c.y), ci = make_float2(c.z, c.w);
                ds_fma(ar[v], tr_, cr);
                ds_fma(ar[v], mti, ci);
                ds_fma(ai[v], tr_, ci);
                ds_fma(ai[v], ti, cr);
            }
        }
        if constexpr (STORE) {
#pragma unroll
            for (int v = 0; v < NV; v++) Sout[(int64_t)slot[p] * nvec + v0 + v] = flip(par, zdbl{ds_value(ar[v]), ds_value(ai[v])});
        } else {
            const uint32_t idx = e_idx[p];
#pragma unroll
            for (int v = 0; v < NV; v++)
                red_add(Sout + (int64_t)idx * nvec + v0 + v, flip(par, zdbl{ds_value(ar[v]), ds_value(ai[v])}));
        }
    }
}

int grid_for(int64_t n, int threads = kThreads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// Rows per CTA (CH) so that the staged window, at most CH + maxb - 1 members, fits the
// shared-memory budget; small windows first (more resident CTAs per SM), larger ones
// only when the buckets need them.
int choose_rows(int maxb, size_t bytes_per_entry, size_t &smem, int max_rows = kRowsPerCta)
{
    const size_t budgets[3] = {48 * 1024, 100 * 1024, 200 * 1024};
    for (size_t budget : budgets) {
        int64_t ch = (int64_t)(budget / bytes_per_entry) - (int64_t)maxb - 8;
        if (ch >= 512 || (budget == budgets[2] && ch >= 64)) {
            ch = std::min<int64_t>(ch, max_rows);
            ch = std::max<int64_t>(64, ch & ~(int64_t)63);
            smem = (size_t)(ch + maxb) * bytes_per_entry + 64;
            return (int)ch;
        }
    }
    return -1;
}

sci::TabRule tab_rule(const sci_ctx *ctx) { return sci::TabRule{ctx->spinors, ctx->n}; }

// The tables a sigma launch walks and the rows it computes: the full tables (every row),
// or the range tables of sci_set_row_range() (rows [row_b, row_e)).
// The (N-2) entries [0, sp.big) are the buckets of the tiled kernel (tile starts in
// tiles[0, sp.ntiles)); the window kernels walk [sp.big, e2), whose largest bucket is
// sp.maxb_small.  A launch takes the wide split when it stages kWideRowBytes or more per
// window row.
struct Tabs {
    const uint32_t *e2_idx, *e2_code, *e2_pos;
    int64_t e2;
    const uint32_t *e1_idx;
    const uint64_t *e1_S;
    const uint32_t *e1_meta;
    int64_t e1;
    sci::RowRange rr;
    const sci::TileSplit *ts;
    const uint32_t *tiles() const { return ts->tiles; }
    const sci::Split &split(size_t row_bytes) const
    {
        return row_bytes >= sci::kWideRowBytes ? ts->wide : ts->base;
    }
    int maxb_small() const { return ts->base.maxb_small; }   // the larger of the two
};

Tabs tabs_of(const sci_ctx *ctx)
{
    if (ctx->ranged)
        return Tabs{ctx->r2_idx, ctx->r2_code, ctx->r2_pos, ctx->r2, ctx->r1_idx, ctx->r1_S, ctx->r1_meta, ctx->r1,
                    sci::RowRange{ctx->row_b, ctx->row_e}, &ctx->rsplit2};
    return Tabs{ctx->e2_idx, ctx->e2_code, ctx->e2_pos, ctx->e2, ctx->e1_idx, ctx->e1_S, ctx->e1_meta, ctx->e1,
                sci::RowRange{0, ctx->M}, &ctx->split2};
}

// the tiled kernel over the buckets of [0, sp.big) (nothing when there are none)
template <class P, bool RG, bool ST, int NV>
int launch_tiled(sci_ctx *ctx, const Tabs &T, const sci::Split &sp, const typename P::TT *tab,
                 const typename P::CI *C, int cstride, int coff, int nvec, int v0, typename P::TO *S)
{
    if (sp.ntiles == 0) return SCI_OK;
    const size_t per = NV * sizeof(typename P::SC) + sizeof(uint2);
    int tcol = (int)std::min<size_t>(1024, (kTiledSmem - 16) / per) & ~31;
    const size_t smem = (((size_t)tcol * NV * sizeof(typename P::SC) + 15) & ~(size_t)15) + (size_t)tcol * sizeof(uint2);
    const int64_t grid = std::min<int64_t>(sp.ntiles, 152 * 16);
    // few tiles: split the columns too, up to the column tiles of the largest bucket, for
    // about 8 CTAs per SM (not in the deterministic mode, whose slots have one writer)
    int nsplit = 1;
    if (!ST && sp.ntiles < 152 * 8) {
        const int64_t want = (152 * 8 + sp.ntiles - 1) / sp.ntiles;
        const int64_t most = (ctx->maxb2 + tcol - 1) / tcol;
        nsplit = (int)std::max<int64_t>(1, std::min<int64_t>({want, most, 65535}));
    }
    k_doubles_tiled<P, NV, RG, ST><<<dim3((unsigned)grid, (unsigned)nsplit), kThreads, smem, ctx->stream>>>(
        T.e2_idx, T.e2_code, T.e2_pos, T.tiles(), sp.ntiles, tcol, tab_rule(ctx), tab, C, cstride, coff, nvec, v0, S,
        T.rr, ST ? ctx->det_inv2 : nullptr);
    return sci_cuda_check(ctx, cudaGetLastError(), "k_doubles_tiled launch");
}

// staged bytes per window row: NV coefficients, the (code, offset) pair, and in a RANGED
// launch the row's slot in the owned-row list
template <bool RG> constexpr size_t row_extra() { return RG ? 8 + sizeof(uint16_t) : 8; }

template <bool RG, bool ST, typename TS, typename TC, int NV>
int launch_doubles(sci_ctx *ctx, const Tabs &T, const TS *tab, const TC *C, typename AccOf<TS>::type *S, int nvec,
                   int v0)
{
    if (T.e2 == 0) return SCI_OK;
    const size_t per = NV * sizeof(TS) + row_extra<RG>();
    const sci::Split &sp = T.split(per);
    int rc = launch_tiled<PolF64<TS, TC>, RG, ST, NV>(ctx, T, sp, tab, C, nvec, v0, nvec, v0, S);
    const int64_t b = sp.big, E = T.e2 - b;
    if (rc != SCI_OK || E == 0) return rc;
    size_t smem = 0;
    int ch = choose_rows(sp.maxb_small, per, smem);
    if (ch < 0) return sci_fail(ctx, SCI_ERR_OVERFLOW, "bucket too large for shared memory");
    auto kern = k_doubles<TS, TC, NV, RG, ST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return sci_cuda_check(ctx, e, "cudaFuncSetAttribute");
    int64_t blocks = (E + ch - 1) / ch;
    kern<<<(unsigned)blocks, kThreads, smem, ctx->stream>>>(T.e2_idx + b, T.e2_code + b, T.e2_pos + b, E, ch,
                                                          tab_rule(ctx), tab, C, nvec, v0, S, T.rr,
                                                          ST ? ctx->det_inv2 + b : nullptr);
    return sci_cuda_check(ctx, cudaGetLastError(), "k_doubles launch");
}

// paired-FP32 doubles: real (float2 table, float2 staged c) or complex (float4 / float4)
template <bool RG, bool ST, bool CPLX, int NV>
int launch_doubles_ds(sci_ctx *ctx, const Tabs &T, const void *C, void *S, int nvec, int v0)
{
    if (T.e2 == 0) return SCI_OK;
    const size_t per = NV * (CPLX ? sizeof(float4) : sizeof(float2)) + row_extra<RG>();
    const sci::Split &sp = T.split(per);
    const int64_t b = sp.big, E = T.e2 - b;
    size_t smem = 0;
    int ch = E > 0 ? choose_rows(sp.maxb_small, per, smem) : 0;
    if (ch < 0) return sci_fail(ctx, SCI_ERR_OVERFLOW, "bucket too large for shared memory");
    cudaError_t e;
    // the vector group, split into paired floats in the context's c_ds buffer
    // (64 bytes per determinant: up to 8 real or 4 complex coefficients)
    if constexpr (CPLX)
        k_split_cz<<<grid_for(ctx->M * NV), kThreads, 0, ctx->stream>>>((const zdbl *)C, ctx->M, nvec, v0, NV,
                                                                        (float4 *)ctx->c_ds);
    else
        k_split_c<<<grid_for(ctx->M * NV), kThreads, 0, ctx->stream>>>((const double *)C, ctx->M, nvec, v0, NV,
                                                                       (float2 *)ctx->c_ds);
    int rc;
    if constexpr (CPLX)
        rc = launch_tiled<PolDSZ, RG, ST, NV>(ctx, T, sp, (const float4 *)ctx->tab_ds, (const float4 *)ctx->c_ds, NV,
                                              0, nvec, v0, (zdbl *)S);
    else
        rc = launch_tiled<PolDS, RG, ST, NV>(ctx, T, sp, (const float2 *)ctx->tab_ds, (const float2 *)ctx->c_ds, NV,
                                             0, nvec, v0, (double *)S);
    if (rc != SCI_OK || E == 0) return rc;
    const int64_t blocks = (E + ch - 1) / ch;
    const uint32_t *slot = ST ? ctx->det_inv2 + b : nullptr;
    if constexpr (CPLX) {
        auto kern = k_doubles_dsz<NV, RG, ST>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return sci_cuda_check(ctx, e, "cudaFuncSetAttribute");
        kern<<<(unsigned)blocks, kThreads, smem, ctx->stream>>>(T.e2_idx + b, T.e2_code + b, T.e2_pos + b, E, ch,
                                                              tab_rule(ctx), (const float4 *)ctx->tab_ds,
                                                              (const float4 *)ctx->c_ds, nvec, v0, (zdbl *)S, T.rr, slot);
    } else {
        auto kern = k_doubles_ds<NV, RG, ST>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return sci_cuda_check(ctx, e, "cudaFuncSetAttribute");
        kern<<<(unsigned)blocks, kThreads, smem, ctx->stream>>>(T.e2_idx + b, T.e2_code + b, T.e2_pos + b, E, ch,
                                                              tab_rule(ctx), (const float2 *)ctx->tab_ds,
                                                              (const float2 *)ctx->c_ds, nvec, v0, (double *)S, T.rr, slot);
    }
    return sci_cuda_check(ctx, cudaGetLastError(), "k_doubles_ds launch");
}

template <bool RG, bool ST, bool CPLX>
int ds_groups(sci_ctx *ctx, const Tabs &T, const void *C, void *S, int nvec)
{
    int rc = SCI_OK;
    const size_t unit = CPLX ? sizeof(float4) : sizeof(float2);
    for (int v0 = 0; v0 < nvec && rc == SCI_OK;) {
        int left = nvec - v0;
        int g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        if (CPLX && g > 4) g = 4;
        size_t smem_probe = 0;
        while (g > 1 && choose_rows(T.maxb_small(), g * unit + row_extra<RG>(), smem_probe) < 0) g >>= 1;
        switch (g) {
        case 8: rc = launch_doubles_ds<RG, ST, CPLX, 8>(ctx, T, C, S, nvec, v0); break;
        case 4: rc = launch_doubles_ds<RG, ST, CPLX, 4>(ctx, T, C, S, nvec, v0); break;
        case 2: rc = launch_doubles_ds<RG, ST, CPLX, 2>(ctx, T, C, S, nvec, v0); break;
        default: rc = launch_doubles_ds<RG, ST, CPLX, 1>(ctx, T, C, S, nvec, v0); break;
        }
        v0 += g;
    }
    return rc;
}

// FP32-storage doubles (SCI_PREC_F32_STORE_F64_ACC)
template <bool RG, bool ST, int NV>
int launch_doubles_f32(sci_ctx *ctx, const Tabs &T, const float *C, double *S, int nvec, int v0)
{
    if (T.e2 == 0) return SCI_OK;
    const size_t per = NV * sizeof(float) + row_extra<RG>();
    const sci::Split &sp = T.split(per);
    int rc = launch_tiled<PolF32, RG, ST, NV>(ctx, T, sp, ctx->tab32, C, nvec, v0, nvec, v0, S);
    const int64_t b = sp.big, E = T.e2 - b;
    if (rc != SCI_OK || E == 0) return rc;
    size_t smem = 0;
    int ch = choose_rows(sp.maxb_small, per, smem, NV >= 8 ? SCI_F32_ROWS : kRowsPerCta);
    if (ch < 0) return sci_fail(ctx, SCI_ERR_OVERFLOW, "bucket too large for shared memory");
    int64_t blocks = (E + ch - 1) / ch;
    auto kern = k_doubles_f32<NV, RG, ST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return sci_cuda_check(ctx, e, "cudaFuncSetAttribute");
    kern<<<(unsigned)blocks, kThreads, smem, ctx->stream>>>(T.e2_idx + b, T.e2_code + b, T.e2_pos + b, E, ch,
                                                          tab_rule(ctx), ctx->tab32, C, nvec, v0, S, T.rr,
                                                          ST ? ctx->det_inv2 + b : nullptr);
    return sci_cuda_check(ctx, cudaGetLastError(), "k_doubles_f32 launch");
}

template <bool RG, bool ST>
int f32_groups(sci_ctx *ctx, const Tabs &T, const float *C, double *S, int nvec)
{
    int rc = SCI_OK;
    for (int v0 = 0; v0 < nvec && rc == SCI_OK;) {
        int left = nvec - v0;
        int g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        size_t smem_probe = 0;
        while (g > 1 && choose_rows(T.maxb_small(), g * sizeof(float) + row_extra<RG>(), smem_probe) < 0) g >>= 1;
        switch (g) {
        case 8: rc = launch_doubles_f32<RG, ST, 8>(ctx, T, C, S, nvec, v0); break;
        case 4: rc = launch_doubles_f32<RG, ST, 4>(ctx, T, C, S, nvec, v0); break;
        case 2: rc = launch_doubles_f32<RG, ST, 2>(ctx, T, C, S, nvec, v0); break;
        default: rc = launch_doubles_f32<RG, ST, 1>(ctx, T, C, S, nvec, v0); break;
        }
        v0 += g;
    }
    return rc;
}

// paired-FP32 singles; real coefficients may come in as double or float; keys of one to
// four words (KW)
template <bool RG, bool ST, bool CPLX, int NV, typename TC, int KW>
int launch_singles_ds_w(sci_ctx *ctx, const Tabs &T, const void *C, void *S, int nvec, int v0)
{
    const int g = grid_for(T.e1);
    if constexpr (CPLX) {
        k_split_cz<<<grid_for(ctx->M * NV), kThreads, 0, ctx->stream>>>((const zdbl *)C, ctx->M, nvec, v0, NV,
                                                                        (float4 *)ctx->c_ds);
        k_singles_dsz<NV, RG, ST, KW><<<g, kThreads, 0, ctx->stream>>>(
            T.e1_idx, T.e1_S, T.e1_meta, T.e1, ctx->norb, ref_words(ctx), (const float4 *)ctx->fref_ds,
            (const float4 *)ctx->g_ds, (const float4 *)ctx->c_ds, nvec, v0, (zdbl *)S, T.rr,
            ST ? ctx->det_inv1 : nullptr);
    } else {
        k_split_c<TC><<<grid_for(ctx->M * NV), kThreads, 0, ctx->stream>>>((const TC *)C, ctx->M, nvec, v0, NV,
                                                                           (float2 *)ctx->c_ds);
        k_singles_ds<NV, RG, ST, KW><<<g, kThreads, 0, ctx->stream>>>(
            T.e1_idx, T.e1_S, T.e1_meta, T.e1, ctx->norb, ref_words(ctx), (const float2 *)ctx->fref_ds,
            (const float2 *)ctx->g_ds, (const float2 *)ctx->c_ds, nvec, v0, (double *)S, T.rr,
            ST ? ctx->det_inv1 : nullptr);
    }
    return sci_cuda_check(ctx, cudaGetLastError(), "k_singles_ds launch");
}

template <bool RG, bool ST, bool CPLX, int NV, typename TC = double>
int launch_singles_ds(sci_ctx *ctx, const Tabs &T, const void *C, void *S, int nvec, int v0)
{
    if (T.e1 == 0) return SCI_OK;
    if (ctx->nwords == 4) return launch_singles_ds_w<RG, ST, CPLX, NV, TC, 4>(ctx, T, C, S, nvec, v0);
    if (ctx->nwords == 3) return launch_singles_ds_w<RG, ST, CPLX, NV, TC, 3>(ctx, T, C, S, nvec, v0);
    if (ctx->nwords == 2) return launch_singles_ds_w<RG, ST, CPLX, NV, TC, 2>(ctx, T, C, S, nvec, v0);
    return launch_singles_ds_w<RG, ST, CPLX, NV, TC, 1>(ctx, T, C, S, nvec, v0);
}

template <bool RG, bool ST, bool CPLX, typename TC = double>
int ds_singles_groups(sci_ctx *ctx, const Tabs &T, const void *C, void *S, int nvec)
{
    int rc = SCI_OK;
    for (int v0 = 0; v0 < nvec && rc == SCI_OK;) {
        int left = nvec - v0;
        int g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        if (CPLX && g > 4) g = 4;
        switch (g) {
        case 8: rc = launch_singles_ds<RG, ST, CPLX, 8, TC>(ctx, T, C, S, nvec, v0); break;
        case 4: rc = launch_singles_ds<RG, ST, CPLX, 4, TC>(ctx, T, C, S, nvec, v0); break;
        case 2: rc = launch_singles_ds<RG, ST, CPLX, 2, TC>(ctx, T, C, S, nvec, v0); break;
        default: rc = launch_singles_ds<RG, ST, CPLX, 1, TC>(ctx, T, C, S, nvec, v0); break;
        }
        v0 += g;
    }
    return rc;
}

template <bool RG, bool ST, typename TS, typename TC, int NV>
int launch_singles(sci_ctx *ctx, const Tabs &T, const TC *C, typename AccOf<TS>::type *S, int nvec, int v0)
{
    if (T.e1 == 0) return SCI_OK;
    auto kern = ctx->nwords == 4   ? k_singles<TS, TC, NV, RG, ST, 4>
                : ctx->nwords == 3 ? k_singles<TS, TC, NV, RG, ST, 3>
                : ctx->nwords == 2 ? k_singles<TS, TC, NV, RG, ST, 2>
                                   : k_singles<TS, TC, NV, RG, ST, 1>;
    kern<<<grid_for(T.e1), kThreads, 0, ctx->stream>>>(T.e1_idx, T.e1_S, T.e1_meta, T.e1, ctx->norb, ref_words(ctx),
                                                       (const TS *)ctx->fref, (const TS *)ctx->g_so, C,
                                                       nvec, v0, S, T.rr, ST ? ctx->det_inv1 : nullptr);
    return sci_cuda_check(ctx, cudaGetLastError(), "k_singles launch");
}

template <bool RG, bool ST, typename TS, typename TC>
int sigma_groups(sci_ctx *ctx, const Tabs &T, const TS *tab, const TC *C, typename AccOf<TS>::type *S, int nvec)
{
    int rc = SCI_OK;
    for (int v0 = 0; v0 < nvec && rc == SCI_OK;) {
        int left = nvec - v0;
        int g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        if (sizeof(TS) == 16 && g > 4) g = 4;
        size_t smem_probe = 0;  // shrink the vector group until its window fits
        while (g > 1 && choose_rows(T.maxb_small(), g * sizeof(TS) + row_extra<RG>(), smem_probe) < 0) g >>= 1;
        switch (g) {
        case 8: rc = launch_doubles<RG, ST, TS, TC, 8>(ctx, T, tab, C, S, nvec, v0); break;
        case 4: rc = launch_doubles<RG, ST, TS, TC, 4>(ctx, T, tab, C, S, nvec, v0); break;
        case 2: rc = launch_doubles<RG, ST, TS, TC, 2>(ctx, T, tab, C, S, nvec, v0); break;
        default: rc = launch_doubles<RG, ST, TS, TC, 1>(ctx, T, tab, C, S, nvec, v0); break;
        }
        v0 += g;
    }
    return rc;
}

template <bool RG, bool ST, typename TS, typename TC>
int singles_groups(sci_ctx *ctx, const Tabs &T, const TC *C, typename AccOf<TS>::type *S, int nvec)
{
    int rc = SCI_OK;
    for (int v0 = 0; v0 < nvec && rc == SCI_OK;) {
        int left = nvec - v0;
        int g = left >= 4 ? 4 : left >= 2 ? 2 : 1;
        switch (g) {
        case 4: rc = launch_singles<RG, ST, TS, TC, 4>(ctx, T, C, S, nvec, v0); break;
        case 2: rc = launch_singles<RG, ST, TS, TC, 2>(ctx, T, C, S, nvec, v0); break;
        default: rc = launch_singles<RG, ST, TS, TC, 1>(ctx, T, C, S, nvec, v0); break;
        }
        v0 += g;
    }
    return rc;
}

// ------------------------------------------------------------------ pair counting
__global__ void k_count2(const uint32_t *__restrict__ e_code, const uint32_t *__restrict__ e_pos, int64_t E,
                         unsigned long long *out)
{
    unsigned long long cnt = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pos = e_pos[p];
        const int64_t bs = p - sci::pos_off(pos), be = bs + sci::pos_size(pos);
        const uint32_t cp = e_code[p];
        for (int64_t q = bs; q < be; q++) cnt += !sci::codes_overlap(e_code[q], cp);
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

__global__ void k_count1(const uint32_t *__restrict__ e_meta, int64_t E, unsigned long long *out)
{
    unsigned long long cnt = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x)
        cnt += sci::meta_size(e_meta[p]) - 1;
    for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// ------------------------------------------------------------------ connection export
struct ConnOut {
    int64_t *row, *col;
    int8_t *deg, *ph;
    int64_t cap;
    unsigned long long *counter;
};

__device__ __forceinline__ void conn_put(ConnOut o, int64_t r, int64_t c, int d, int ph)
{
    unsigned long long s = atomicAdd(o.counter, 1ull);
    if ((int64_t)s < o.cap) {
        o.row[s] = r;
        o.col[s] = c;
        o.deg[s] = (int8_t)d;
        o.ph[s] = (int8_t)ph;
    }
}

__global__ void k_conn2(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code,
                        const uint32_t *__restrict__ e_pos, int64_t E, int64_t rb, int64_t re, ConnOut o)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = e_idx[p];
        if (I < rb || I >= re) continue;
        const uint32_t pos = e_pos[p], code = e_code[p];
        const int64_t bs = p - sci::pos_off(pos), be = bs + sci::pos_size(pos);
        const int par = sci::code_par(code);
        for (int64_t q = bs; q < be; q++) {
            const uint32_t cq = e_code[q];
            if (sci::codes_overlap(cq, code)) continue;
            conn_put(o, I, e_idx[q], 2, (par ^ (int)sci::code_par(cq)) ? -1 : 1);
        }
    }
}

__global__ void k_conn1(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_meta, int64_t E, int64_t rb,
                        int64_t re, ConnOut o)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t I = e_idx[p];
        if (I < rb || I >= re) continue;
        uint32_t meta = e_meta[p];
        int64_t bs = p - (int64_t)sci::meta_off(meta), be = bs + (int64_t)sci::meta_size(meta);
        int par = sci::meta_par(meta);
        for (int64_t q = bs; q < be; q++) {
            if (q == p) continue;
            int parq = sci::meta_par(e_meta[q]);
            conn_put(o, I, e_idx[q], 1, (par ^ parq) ? -1 : 1);
        }
    }
}

inline void mark(sci_ctx *ctx, int i)
{
    if (ctx->profile) cudaEventRecord(ctx->ev[i], ctx->stream);
}

}  // namespace

#define SCI_CK(call)                                                 \
    do {                                                             \
        int _rc = sci_cuda_check(ctx, (call), #call);                \
        if (_rc != SCI_OK) return _rc;                               \
    } while (0)

// whether the largest (N-2) bucket fits the staging window of a one-vector launch in the
// context's scalar mode, row-range launches included (wider vector groups shrink until
// they fit, down to one vector)
bool sci_sigma_window_fits(const sci_ctx *ctx)
{
    size_t smem = 0;
    const size_t per = (ctx->cplx ? sizeof(zdbl) : sizeof(double)) + row_extra<true>();
    return ctx->e2 == ctx->split2.base.big || choose_rows(ctx->split2.base.maxb_small, per, smem) >= 0;
}

namespace {

// Deterministic accumulation: S_I = H_II C_I + the row sums the double- and single-
// excitation kernels stored for row I's bucket entries.  They store them in row order (the
// slot of an entry is its position among the entries sorted by row), so row I's sums are
// the contiguous segment [ptr[I], ptr[I + 1]).  One warp per row: lane l adds the segment's
// elements l, l + 32, ..., then the lanes are combined by a fixed butterfly of shuffles,
// so the result does not depend on scheduling.
__device__ __forceinline__ void add_to(double &a, double b) { a += b; }
__device__ __forceinline__ void add_to(zdbl &a, zdbl b) { a.x += b.x, a.y += b.y; }
__device__ __forceinline__ double shfl_xor(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ zdbl shfl_xor(zdbl a, int o)
{
    return zdbl{__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)};
}
__device__ __forceinline__ double diag_times(double h, double c) { return h * c; }
__device__ __forceinline__ double diag_times(double h, float c) { return h * (double)c; }
__device__ __forceinline__ zdbl diag_times(double h, zdbl c) { return zdbl{h * c.x, h * c.y}; }

// Lanes per row of k_row_sums.  A row holds ~C(N,2)/2 + N slots on average (about 100 on
// the 20-electron spaces), so four lanes per row keep the lanes busy and the butterfly at
// two levels; a warp per row spent more FP64 adds on its butterfly and on padding than on
// the slots (2M-determinant space, one vector: 1.97 ms with a warp per row, FP64 pipe 83%
// busy in ncu; 0.80 ms with four lanes).
constexpr int kRowLanes = 4;

template <typename TC, typename TA, int NV>
__global__ void __launch_bounds__(kThreads)
k_row_sums(int64_t M, int nvec, int v0, const double *__restrict__ hdiag, const TC *__restrict__ C,
           const uint32_t *__restrict__ ptr2, const TA *__restrict__ part2, const uint32_t *__restrict__ ptr1,
           const TA *__restrict__ part1, TA *__restrict__ S)
{
    constexpr int G = kRowLanes, RPW = 32 / G;   // lanes per row, rows per warp
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    // warp-uniform loop (the butterfly needs every lane); a lane past M adds nothing
    for (int64_t Ib = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / 32 * RPW; Ib < M; Ib += warps * RPW) {
        const int64_t I = Ib + lane / G;
        TA acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) zero(acc[v]);
        if (I < M) {
            // the row's doubles slots, then its singles slots: lane gl adds slots gl, gl + G,
            // ... in order, four loads in flight per step, each add predicated on its slot
            for (int tab = 0; tab < 2; tab++) {
                const uint32_t *ptr = tab ? ptr1 : ptr2;
                const TA *part = tab ? part1 : part2;
                const uint32_t end = ptr[I + 1];
                for (uint32_t t0 = ptr[I] + gl; t0 < end; t0 += 4 * G) {
                    TA x[4][NV];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const uint32_t t = t0 + G * u;
                        const TA *src = part + (int64_t)t * nvec + v0;
#pragma unroll
                        for (int v = 0; v < NV; v++) {
                            zero(x[u][v]);
                            if (t < end) x[u][v] = src[v];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (t0 + G * u < end)
#pragma unroll
                            for (int v = 0; v < NV; v++) add_to(acc[v], x[u][v]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < NV; v++)
#pragma unroll
            for (int o = G / 2; o; o >>= 1) add_to(acc[v], shfl_xor(acc[v], o));
        if (I < M) {
            // lane gl writes vectors gl, gl + G, ...: H_II c_I plus the row sum
#pragma unroll
            for (int v = 0; v < NV; v++)
                if (v % G == gl) {
                    TA out = diag_times(hdiag[I], C[I * nvec + v0 + v]);
                    add_to(out, acc[v]);
                    S[I * nvec + v0 + v] = out;
                }
        }
    }
}

template <typename TC, typename TA>
int row_sums(sci_ctx *ctx, const TC *C, TA *S, int nvec)
{
    const int64_t M = ctx->M;
    const int grid = grid_for(M * kRowLanes);
    auto go = [&](auto kern, int v0) {
        kern<<<grid, kThreads, 0, ctx->stream>>>(M, nvec, v0, ctx->hdiag, C, ctx->det_ptr2, (const TA *)ctx->det_part2,
                                                 ctx->det_ptr1, (const TA *)ctx->det_part1, S);
    };
    for (int v0 = 0; v0 < nvec;) {
        const int left = nvec - v0;
        const int g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        switch (g) {
        case 8: go(k_row_sums<TC, TA, 8>, v0); break;
        case 4: go(k_row_sums<TC, TA, 4>, v0); break;
        case 2: go(k_row_sums<TC, TA, 2>, v0); break;
        default: go(k_row_sums<TC, TA, 1>, v0); break;
        }
        v0 += g;
    }
    return sci_cuda_check(ctx, cudaGetLastError(), "k_row_sums launch");
}

// one sigma launch sequence over the tables T (RG: the rows of a row range only; ST: the
// deterministic accumulation, row sums stored in the entries' slots, then per-row sums)
template <bool RG, bool ST>
int launch_sigma(sci_ctx *ctx, const Tabs &T, const void *C, void *S_out, int nvec, int prec)
{
    // with ST the double- and single-excitation kernels write the slots, not S
    void *S = ST ? ctx->det_part2 : S_out;
    void *S1 = ST ? ctx->det_part1 : S_out;
    cudaStream_t st = ctx->stream;
    const int64_t row0 = T.rr.rb, nrows = T.rr.re - T.rr.rb;
    int rc;
    mark(ctx, 0);
    if (ctx->cplx) {
        const zdbl *Cz = (const zdbl *)C;
        zdbl *Sz = (zdbl *)S;
        if (!ST && nrows > 0)
            k_sigma_init<zdbl, zdbl><<<grid_for(nrows * nvec), kThreads, 0, st>>>(ctx->hdiag, Cz, Sz, row0, nrows, nvec);
        SCI_CK(cudaGetLastError());
        mark(ctx, 1);
        rc = prec == SCI_PREC_F64_DS ? ds_groups<RG, ST, true>(ctx, T, C, S, nvec)
                                     : sigma_groups<RG, ST, zdbl, zdbl>(ctx, T, (const zdbl *)ctx->tab, Cz, Sz, nvec);
        mark(ctx, 2);
        if (rc == SCI_OK)
            rc = prec == SCI_PREC_F64_DS ? ds_singles_groups<RG, ST, true>(ctx, T, C, S1, nvec)
                                         : singles_groups<RG, ST, zdbl, zdbl>(ctx, T, Cz, (zdbl *)S1, nvec);
        mark(ctx, 3);
        if (ST && rc == SCI_OK) rc = row_sums<zdbl, zdbl>(ctx, Cz, (zdbl *)S_out, nvec);
        mark(ctx, 4);
        return rc;
    }
    double *Sd = (double *)S;
    if (prec == SCI_PREC_F64 || prec == SCI_PREC_F64_DS) {
        const double *Cd = (const double *)C;
        if (!ST && nrows > 0)
            k_sigma_init<double, double><<<grid_for(nrows * nvec), kThreads, 0, st>>>(ctx->hdiag, Cd, Sd, row0, nrows,
                                                                                       nvec);
        SCI_CK(cudaGetLastError());
        mark(ctx, 1);
        rc = prec == SCI_PREC_F64_DS ? ds_groups<RG, ST, false>(ctx, T, C, S, nvec)
                                     : sigma_groups<RG, ST, double, double>(ctx, T, (const double *)ctx->tab, Cd, Sd, nvec);
        mark(ctx, 2);
        if (rc == SCI_OK)
            rc = prec == SCI_PREC_F64_DS ? ds_singles_groups<RG, ST, false>(ctx, T, C, S1, nvec)
                                         : singles_groups<RG, ST, double, double>(ctx, T, Cd, (double *)S1, nvec);
        mark(ctx, 3);
        if (ST && rc == SCI_OK) rc = row_sums<double, double>(ctx, Cd, (double *)S_out, nvec);
        mark(ctx, 4);
        return rc;
    }
    const float *Cf = (const float *)C;
    if (!ST && nrows > 0)
        k_sigma_init<float, double><<<grid_for(nrows * nvec), kThreads, 0, st>>>(ctx->hdiag, Cf, Sd, row0, nrows, nvec);
    SCI_CK(cudaGetLastError());
    mark(ctx, 1);
    rc = f32_groups<RG, ST>(ctx, T, Cf, Sd, nvec);
    mark(ctx, 2);
    if (rc == SCI_OK) rc = ds_singles_groups<RG, ST, false, float>(ctx, T, C, S1, nvec);
    mark(ctx, 3);
    if (ST && rc == SCI_OK) rc = row_sums<float, double>(ctx, Cf, (double *)S_out, nvec);
    mark(ctx, 4);
    return rc;
}

}  // namespace

int sci_launch_sigma(sci_ctx *ctx, const void *C, void *S, int nvec, int prec, bool whole_list)
{
    if (whole_list || !ctx->ranged) {
        const bool ranged = ctx->ranged;
        ctx->ranged = 0;   // tabs_of: the full tables
        const Tabs T = tabs_of(ctx);
        ctx->ranged = ranged;
        if (ctx->det_nvec > 0 && nvec <= ctx->det_nvec) return launch_sigma<false, true>(ctx, T, C, S, nvec, prec);
        return launch_sigma<false, false>(ctx, T, C, S, nvec, prec);
    }
    return launch_sigma<true, false>(ctx, tabs_of(ctx), C, S, nvec, prec);
}

int sci_count_pairs_device(sci_ctx *ctx, int64_t *pairs2, int64_t *pairs1)
{
    cudaStream_t st = ctx->stream;
    unsigned long long *d = nullptr;
    SCI_CK(cudaMalloc(&d, 16));
    cudaMemsetAsync(d, 0, 16, st);
    if (ctx->e2 > 0) k_count2<<<grid_for(ctx->e2), kThreads, 0, st>>>(ctx->e2_code, ctx->e2_pos, ctx->e2, d);
    if (ctx->e1 > 0) k_count1<<<grid_for(ctx->e1), kThreads, 0, st>>>(ctx->e1_meta, ctx->e1, d + 1);
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    SCI_CK(e);
    *pairs2 = (int64_t)h[0];
    *pairs1 = (int64_t)h[1];
    return SCI_OK;
}

int sci_connections_device(sci_ctx *ctx, int64_t row_begin, int64_t row_end, int64_t *count, int64_t *rows,
                           int64_t *J, int8_t *degree, int8_t *phase, int64_t cap)
{
    cudaStream_t st = ctx->stream;
    unsigned long long *counter = nullptr;
    SCI_CK(cudaMalloc(&counter, 8));
    // pass 1: count
    ConnOut o{nullptr, nullptr, nullptr, nullptr, 0, counter};
    cudaMemsetAsync(counter, 0, 8, st);
    if (ctx->e2 > 0)
        k_conn2<<<grid_for(ctx->e2), kThreads, 0, st>>>(ctx->e2_idx, ctx->e2_code, ctx->e2_pos, ctx->e2, row_begin,
                                                         row_end, o);
    if (ctx->e1 > 0)
        k_conn1<<<grid_for(ctx->e1), kThreads, 0, st>>>(ctx->e1_idx, ctx->e1_meta, ctx->e1, row_begin, row_end, o);
    unsigned long long n = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, counter, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(counter); return sci_cuda_check(ctx, e, "connection count"); }
    *count = (int64_t)n;
    if ((int64_t)n > cap) { cudaFree(counter); return sci_fail(ctx, SCI_ERR_OVERFLOW, "connection list exceeds cap"); }
    if (n == 0) { cudaFree(counter); return SCI_OK; }
    // pass 2: fill
    void *buf = nullptr;
    e = cudaMalloc(&buf, n * 18);
    if (e != cudaSuccess) { cudaFree(counter); return sci_cuda_check(ctx, e, "connection buffer"); }
    o.row = (int64_t *)buf;
    o.col = o.row + n;
    o.deg = (int8_t *)(o.col + n);
    o.ph = o.deg + n;
    o.cap = (int64_t)n;
    cudaMemsetAsync(counter, 0, 8, st);
    if (ctx->e2 > 0)
        k_conn2<<<grid_for(ctx->e2), kThreads, 0, st>>>(ctx->e2_idx, ctx->e2_code, ctx->e2_pos, ctx->e2, row_begin,
                                                         row_end, o);
    if (ctx->e1 > 0)
        k_conn1<<<grid_for(ctx->e1), kThreads, 0, st>>>(ctx->e1_idx, ctx->e1_meta, ctx->e1, row_begin, row_end, o);
    std::vector<int64_t> hr(n), hc(n);
    std::vector<int8_t> hd(n), hp(n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr.data(), o.row, n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), o.col, n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), o.deg, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), o.ph, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    cudaFree(counter);
    SCI_CK(e);
    std::vector<int64_t> perm(n);
    for (size_t t = 0; t < n; t++) perm[t] = (int64_t)t;
    std::sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) {
        return hr[a] != hr[b] ? hr[a] < hr[b] : hc[a] < hc[b];
    });
    for (size_t t = 0; t < n; t++) {
        int64_t s = perm[t];
        if (rows) rows[t] = hr[s];
        if (J) J[t] = hc[s];
        if (degree) degree[t] = hd[s];
        if (phase) phase[t] = hp[s];
    }
    return SCI_OK;
}
