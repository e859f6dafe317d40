// Internal declarations of libsci (sigma = H c for selected CI on sm_103a).
//
// Data layout in device memory (all owned by the context):
//   keys[M]            uint64 determinant keys, ascending.
//   hdiag[M]           FP64 diagonal H_II (Sec. 2.1, Eq. decompositionH: H_1^0 + H_2^0).
//   tab                pair-integral table read by the double-excitation kernel.  Real
//                      spin-orbital mode: [ T | W ] with
//                        T[y'][x'][y][x] = (x x'|y y')  (alpha x<-x', beta y<-y')
//                        W[P(i,j)][P(a,b)] = (ai|bj) - (aj|bi), a<b, i<j same spin,
//                      spinor mode: W only (complex), P(a,b) = b(b-1)/2 + a.
//                      The bra (row) indices are the fast ones so that lanes that own
//                      consecutive rows of one bucket read consecutive addresses.
//   g_so[k][i][a]      (ai|kk) - (ak|ki) over spin-orbitals/spinors (singles).
//   fref[i][a]         h_ai + sum_{k in ref} g_so[k][i][a]: the Fock matrix of the
//                      reference determinant ref (lowest orbitals), the closed-shell
//                      reference trick of Sec. 2.3.
//   Doubles table "B2" (structure of arrays over E2 entries): every determinant D
//     emits the (N-2)-electron keys K = D minus two occupied bits; entries sharing K
//     form a bucket and are within a double excitation of each other.  Buckets of size
//     1 are dropped; the rest are stored contiguously, largest first.  12 bytes each:
//       e2_idx[p]     determinant index of the member
//       e2_code[p]    bits 0-7 x, bits 8-15 y: the two extra orbitals x < y of the
//                     member (D = K | 2^x | 2^y); bit 16 the phase parity
//                     #(K below x) + #(K below y); bits 17-22 the member's position
//                     inside its y-group (members of the bucket with the same y);
//                     bits 23-29 the y-group size
//       e2_pos[p]     bits 0-15 position inside the bucket, bits 16-31 bucket size
//     Table offsets are derived from (x, y) by pair_offsets().
//   Singles table "B1": the same with (N-1)-electron keys S = D minus one bit.
//       e1_idx[p], e1_S[p] (the bucket key S), e1_meta[p]: bits 0-6 extra orbital,
//       bit 7 parity, bits 8-19 position in bucket, bits 20-31 bucket size.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sci.h"

namespace sci {

struct zdbl {
    double x, y;
};

enum DevErr : int {
    DEV_UNSORTED = 1,
    DEV_DUPLICATE = 2,
    DEV_POPCOUNT = 4,
    DEV_OVERFLOW = 8,
};

// fields of an (N-2)-table code word and position word
__host__ __device__ __forceinline__ int code_x(uint32_t c) { return (int)(c & 0xFFu); }
__host__ __device__ __forceinline__ int code_y(uint32_t c) { return (int)((c >> 8) & 0xFFu); }
__host__ __device__ __forceinline__ bool code_par(uint32_t c) { return (c >> 16) & 1u; }
__host__ __device__ __forceinline__ int code_gofs(uint32_t c) { return (int)((c >> 17) & 0x3Fu); }
__host__ __device__ __forceinline__ int code_gsize(uint32_t c) { return (int)((c >> 23) & 0x7Fu); }
__host__ __device__ __forceinline__ uint32_t make_code(int x, int y, int par, int gofs, int gsize)
{
    return (uint32_t)x | ((uint32_t)y << 8) | ((uint32_t)par << 16) | ((uint32_t)gofs << 17) | ((uint32_t)gsize << 23);
}
__host__ __device__ __forceinline__ int pos_off(uint32_t p) { return (int)(p & 0xFFFFu); }
__host__ __device__ __forceinline__ int pos_size(uint32_t p) { return (int)(p >> 16); }
// fields of an (N-1)-table meta word: the member's extra orbital x (8 bits, up to 255
// orbitals), the parity of its position, its offset in the bucket (11 bits) and the bucket
// size (12 bits)
__host__ __device__ __forceinline__ int meta_x(uint32_t m) { return (int)(m & 0xFFu); }
__host__ __device__ __forceinline__ bool meta_par(uint32_t m) { return (m >> 8) & 1u; }
__host__ __device__ __forceinline__ int meta_off(uint32_t m) { return (int)((m >> 9) & 0x7FFu); }
__host__ __device__ __forceinline__ int meta_size(uint32_t m) { return (int)(m >> 20); }
__host__ __device__ __forceinline__ uint32_t make_meta(int x, int par, int off, int size)
{
    return (uint32_t)x | ((uint32_t)par << 8) | ((uint32_t)off << 9) | ((uint32_t)size << 20);
}
constexpr int kMaxBucket1 = 2047;   // the largest (N-1) bucket the meta word holds
// 64-bit words of an occupation string at most: 256 spin-orbitals or spinors, the most the
// 8-bit orbital fields of the bucket codes hold
constexpr int kMaxWords = 4;
// the reference string, word w holding orbitals 64w .. 64w + 63
struct RefW {
    uint64_t w[kMaxWords];
};
// (N-2) buckets of more members than this go through the tiled sigma kernel by default.
// Measured on 2M-determinant spaces (doubles kernel, FP64, one vector): buckets of up to
// 1,089 (80 spin-orbitals) 12.04 ms all in windows, 9.12 ms with those above 512 tiled;
// up to 4,489 (140 spin-orbitals) 25.8 ms at 2048, 20.2 ms at 512; a space whose buckets
// stay below 512 (30 orbitals, up to 441) is unchanged, and tiling it at 256 costs 2%.
constexpr int kTileBucket = 512;
constexpr int kTileRows = 256;      // rows of a tile of the tiled kernel (one per thread)
// launches that stage 64 bytes or more per window row (8 real vectors) tile from this
// size instead (measured on the 30-orbital 2M space, buckets up to 441: FP64 x 8
// 39.75 -> 38.66 ms, paired FP32 x 8 25.97 -> 22.52 ms; narrower launches lose 0-6%)
constexpr int kTileBucketWide = 384;
constexpr size_t kWideRowBytes = 64;

// The split of an (N-2) table at one threshold: entries [0, big) are the buckets above it
// (the table holds buckets largest first), their tiles are the first ntiles of the tile
// list, and maxb_small is the largest bucket left to the window kernels.
struct Split {
    int64_t big = 0, ntiles = 0;
    int maxb_small = 0;
};
// tile starts (table order) of the buckets above the lower of the two thresholds, and the
// splits at the context's threshold (base) and at the wide-launch threshold (wide)
struct TileSplit {
    uint32_t *tiles = nullptr;
    Split base, wide;
};
// whether two members of a bucket share an extra orbital (then they are a single
// excitation of each other, not a double); valid for orbitals up to 255
__host__ __device__ __forceinline__ bool codes_overlap(uint32_t a, uint32_t b)
{
    const int xa = code_x(a), ya = code_y(a), xb = code_x(b), yb = code_y(b);
    return xa == xb || xa == yb || ya == xb || ya == yb;
}

// Rows whose sigma a launch computes: [rb, re) (sci_set_row_range), every row otherwise.
struct RowRange {
    int64_t rb, re;
};

// Layout of the pair-integral table (see tab above).
struct TabRule {
    int spinors, n;
};

// bra (row) offset and ket (column) base of a member with extra orbitals x < y
__host__ __device__ __forceinline__ void pair_offsets(TabRule r, int x, int y, uint32_t &rowoff, uint32_t &colbase)
{
    if (r.spinors) {
        const uint32_t NP = (uint32_t)(r.n * (r.n - 1) / 2);
        const uint32_t p = (uint32_t)(y * (y - 1) / 2 + x);
        rowoff = p;
        colbase = p * NP;
        return;
    }
    const int n = r.n;
    const uint32_t n2 = (uint32_t)(n * n);
    if (x < n && y >= n) {  // alpha-beta
        const uint32_t u = (uint32_t)((y - n) * n + x);
        rowoff = u;
        colbase = u * n2;
    } else {                // same spin
        const int a = x >= n ? x - n : x, b = y >= n ? y - n : y;
        const uint32_t NP = (uint32_t)(n * (n - 1) / 2);
        const uint32_t p = (uint32_t)(b * (b - 1) / 2 + a);
        rowoff = p;
        colbase = n2 * n2 + p * NP;
    }
}

}  // namespace sci

struct sci_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // Hamiltonian
    int have_ints = 0;
    int cplx = 0;     // 1: complex128 scalars
    int spinors = 0;  // 1: spinor mode
    int n = 0;        // spatial orbitals or spinors
    int norb = 0;     // bits in a key: 2n or n
    void *h_so = nullptr;   // [norb][norb], spin-orbital h (scalar)
    void *jd = nullptr;     // [norb][norb] (ii|jj)
    void *kd = nullptr;     // [norb][norb] (ij|ji)
    void *g_so = nullptr;   // [norb][norb][norb]
    void *tab = nullptr;    // pair table (scalar)
    float *tab32 = nullptr; // FP32 copy of tab (real mode)
    void *tab_ds = nullptr; // tab split into (hi, lo) floats: float2 (real) / float4 (complex)
    void *c_ds = nullptr;   // per-call split of one vector group of C: [M][<=8] float2 or [M][<=4] float4
    void *g_ds = nullptr;   // g_so split into (hi, lo) floats
    void *fref_ds = nullptr;  // fref split into (hi, lo) floats
    int64_t tab_elems = 0;

    // determinants
    int have_dets = 0;
    int64_t M = 0;
    int na = 0, nb = 0, N = 0;
    uint64_t ref = 0;       // the reference (lowest orbitals), bits 0..63
    uint64_t ref_hi = 0;    // its bits 64..127 (two- and three-word lists)
    uint64_t ref_w2 = 0;    // its bits 128..191 (three- and four-word lists)
    uint64_t ref_w3 = 0;    // its bits 192..255 (four-word lists)
    int nwords = 1;         // 64-bit words per key: 1, 2 past 64 spin-orbitals, 3 past 128, 4 past 192
    uint64_t *keys = nullptr;  // [M][nwords], word 0 holding orbitals 0..63
    double *hdiag = nullptr;
    void *fref = nullptr;   // [norb][norb]

    int64_t e2 = 0, nb2 = 0;
    uint32_t *e2_idx = nullptr;
    uint32_t *e2_code = nullptr;
    uint32_t *e2_pos = nullptr;
    int64_t e1 = 0, nb1 = 0;
    uint32_t *e1_idx = nullptr;
    uint64_t *e1_S = nullptr;   // [e1][nwords]: the bucket key S of each entry
    uint32_t *e1_meta = nullptr;
    int maxb2 = 0, maxb1 = 0;
    int64_t pairs = 0, pairs2 = 0, pairs1 = 0;

    // (N-2) buckets of more than tile_b members (min(tile_b, kTileBucketWide) for wide
    // launches, unless the caller set the threshold) are walked by the tiled kernel, their
    // members staged in shared memory a tile at a time, instead of the window kernels:
    // split2 for the full tables, rsplit2 for the range tables
    int tile_b = sci::kTileBucket;
    int tile_user = 0;   // the threshold was set by sci_set_tile_threshold: one for all launches
    sci::TileSplit split2, rsplit2;

    // row range of sci_sigma() (sci_set_row_range): when `ranged`, sigma computes rows
    // [row_b, row_e) only, walking range tables r2_* / r1_* that keep (whole, in table
    // order) the buckets with a member in the range; range_pairs counts the connected
    // pairs (I, J) with I in the range
    int ranged = 0;
    int64_t row_b = 0, row_e = 0;
    int64_t r2 = 0, r1 = 0, range_pairs = 0, range_pairs2 = 0, range_pairs1 = 0;
    uint32_t *r2_idx = nullptr, *r2_code = nullptr, *r2_pos = nullptr;
    uint32_t *r1_idx = nullptr;
    uint64_t *r1_S = nullptr;
    uint32_t *r1_meta = nullptr;
    size_t range_bytes = 0;

    // deterministic accumulation (sci_set_deterministic): when det_nvec > 0, sigma stores
    // each (bucket, member) row sum at slot det_inv[entry] of det_part2 / det_part1
    // ([entries][det_nvec] scalars), the entry's position among the entries sorted by row
    // (stable, so ascending table position within a row), and a second kernel adds each
    // row's contiguous segment [det_ptr[I], det_ptr[I + 1]) in a fixed order
    int det_nvec = 0;
    uint32_t *det_ptr2 = nullptr, *det_inv2 = nullptr, *det_ptr1 = nullptr, *det_inv1 = nullptr;
    void *det_part2 = nullptr, *det_part1 = nullptr;
    size_t det_bytes = 0;

    // host-buffer sigma staging
    void *stage_c = nullptr, *stage_s = nullptr;
    size_t stage_bytes = 0;

    // block-vector kernels: per-CTA partials of P = A^T B, grown on demand
    void *bv_part = nullptr;
    size_t bv_bytes = 0;

    // density matrices: per-call scratch (grown on demand) and the device copy of the weights
    void *rdm_scratch = nullptr;
    size_t rdm_bytes = 0;
    void *rdm_w = nullptr;
    size_t rdm_wbytes = 0;

    // kernel timing
    int profile = 0;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

    int *status = nullptr;  // device status word (sci::DevErr bits)
    size_t bytes_held = 0;
};

// the context's reference string over all words
inline sci::RefW ref_words(const sci_ctx *ctx) { return sci::RefW{{ctx->ref, ctx->ref_hi, ctx->ref_w2, ctx->ref_w3}}; }

// helpers shared by the translation units of the library
int sci_fail(sci_ctx *ctx, int code, const std::string &msg);
int sci_cuda_check(sci_ctx *ctx, cudaError_t e, const char *what);

// Commits the fixed scratch array of sci_connections_noalloc() on `device` (which must be
// current) and caches its address; sci_noalloc.cu.
cudaError_t sci_noalloc_prepare(int device);

// row ranges (sci_rows.cu): frees the range tables and clears the range
void sci_free_range(sci_ctx *ctx);
// deterministic accumulation (sci_rows.cu): frees its index and buffers, back to atomics
void sci_free_det(sci_ctx *ctx);

// the tiled prefixes of the full (ranged = false) or range tables for the context's
// thresholds: split2 / rsplit2 (sci_setup.cu); synchronous
int sci_table_split(sci_ctx *ctx, bool ranged);
void sci_free_split(sci_ctx *ctx, bool ranged);

// launchers (sci_sigma.cu)
bool sci_sigma_window_fits(const sci_ctx *ctx);
// whole_list: every row over the full tables whatever the context's row range (internal
// callers such as ENPT2); otherwise the rows of the range, if one is set
int sci_launch_sigma(sci_ctx *ctx, const void *C, void *S, int nvec, int prec, bool whole_list = false);
int sci_count_pairs_device(sci_ctx *ctx, int64_t *pairs2, int64_t *pairs1);
int sci_connections_device(sci_ctx *ctx, int64_t row_begin, int64_t row_end, int64_t *count,
                           int64_t *rows, int64_t *J, int8_t *degree, int8_t *phase,
                           int64_t cap);
