// Epstein-Nesbet second-order energies (Sec. 2.4, constraint-based ENPT2) on the GPU.
//
// For the roots (E0_k, c_k) of the variational space P (here P_m = P):
//   E2_k[Q] = E2_k[W] - E2_k[P]                                      (Eq. PT2final)
//   E2_k[W] = sum_{I in W} (sum_{J in P, J != I} H_IJ c_Jk)^2 / (E0_k - H_II)     (Eq. EW1)
//   E2_k[P] = sum_{I in P} (<I|H|c_k> - c_Ik H_II)^2 / (E0_k - H_II)              (Eq. EP1)
// where W is every determinant a single or double excitation away from some J in P.
// The W - P form avoids testing membership of each generated determinant in P.
//
// E2[W] is accumulated in batches W_b, disjoint by a constraint on the determinant I, so
// that the numerators of one batch fit a hash table in device memory (the memory-bounded
// pipeline of the paper's constraint-based algorithm).  The constraint here is a linear
// code over GF(2) of I's beta string, f(I_beta) = XOR of g(o) over its occupied orbitals,
// with g a random t-bit code per orbital: the batch of an excitation of J follows from
// f(J_beta) and the codes of the moved beta orbitals alone, so a warp that owns J reaches
// exactly the excitations of the current batch --
//   alpha singles and alpha-alpha doubles: all of them when f(J_beta) = b;
//   beta singles j -> v (and the alpha-beta doubles built on them): g(j) ^ g(v) = b ^ f(J_beta);
//   beta-beta doubles j1 j2 -> b1 < b2: g(b2) = b ^ f(J_beta) ^ g(j1) ^ g(j2) ^ g(b1),
// with the orbitals grouped by code so that each lookup is a short list.
// Each generated (I, H_IJ c_J) is added to the table entry of I (open addressing, linear
// probing bounded by kMaxProbe, key and values in one slot, FP64 atomic adds); then every
// entry is evaluated with
//   H_II = E_ref - sum_{i in holes} F_ii + sum_{a in particles} F_aa
//          + sum_{pairs in holes} G + sum_{pairs in particles} G - sum_{holes x particles} G,
// F the Fock diagonal of the reference and G_pq = (pp|qq) - (pq|qp): O(level^2) per I.
// Element formulas and phases are those of the sigma kernels (bra I, ket J).
//
// Screening (eps > 0): a contribution with |H_IJ| max_k |c_Jk| < eps is left out.  Before
// any element of a double-excitation class is evaluated, the class is tested against an
// upper bound of its elements over the table, the GPU form of the paper's screening by the
// upper bounds of Table 1 (Sec. 2.3): for determinants the double element is one entry of
// the pair table, independent of the spectators, so
//   same spin:   B[P(i,j)][a] = max_{b > a} |W(ij -> ab)|,  and its max over a;
//   alpha-beta:  B[i, j] = max_{a,b} |(ai|bj)|;
//   spinors:     B[P(i,j)][a] = max_{b > a} |W(ij -> ab)|.
// A class whose bound times max_k |c_Jk| is below eps is skipped whole; since the bound is
// at least every element of the class, the sum equals that of the per-element test.
//
// Spinor mode (complex Hermitian integrals, no spin conservation; the 4C workloads of
// Sec. 4): every single i -> a and double i < j -> a < b over the n <= 64 spinors.  The
// batch code runs over the whole string, f(I) = XOR of g(o) over I's occupied spinors, so
// the warp that owns J finds the excitations of batch b by lookups in the spinors grouped
// by code:
//   singles:  g(a) = b ^ f(J) ^ g(i)                         for each occupied i;
//   doubles:  g(b') = b ^ f(J) ^ g(i) ^ g(j) ^ g(a), b' > a    for each occupied pair and
//             first virtual a.
// Numerators are complex (2 words per root in a slot) and a slot adds |num|^2 / (E0 - H_II);
// E2[P] takes |<I|H|c> - c_I H_II|^2.
#include <algorithm>
#include <cstring>
#include <random>
#include <type_traits>
#include <vector>

#include "sci_bits.cuh"
#include "sci_ds.cuh"
#include "sci_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint64_t kEmpty = 0;   // no determinant with electrons has key 0
constexpr int kMaxProbe = 1 << 12;
constexpr int kMaxBits = 10;   // at most 1024 batches

struct Pt2 {
    int n, norb, na, nb;
    uint64_t ref, ref_hi, ref_w2;   // the reference string: orbitals 0..63, 64..127, 128..191
    const double *tab, *fref, *g_so;
    const double *fdiag, *G;  // [norb], [norb][norb]
    const double *Eref;
    uint32_t gcode[192];      // codes of the beta orbitals (spin-orbital mode) or spinors
    uint8_t obc[192];         // those orbitals sorted by code
    uint8_t cstart[(1 << kMaxBits) + 1];  // first index in obc of each code
    uint64_t *tab2;           // slots of (key words, value words), key 0 = empty
    uint64_t mask;            // capacity - 1
    unsigned long long *count;
    unsigned long long limit;
    int *flag;
    double eps;
    // screening bounds (NULL when eps = 0): see the header
    const double *bss3;   // [NP][n] same-spin (real) or spinor: max over b > a, per (pair, a)
    const double *bss;    // [NP] same-spin (real): max over a of bss3
    const double *bab;    // [n][n] alpha-beta (real): [j_beta * n + i_alpha]
};

using sci::below;
using sci::kMaxPairs;
using sci::sflip;

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Occupation strings of one word (K = uint64_t, up to 64 orbitals) or two (K = W2, up to
// 128 orbitals; word 0 = orbitals 0..63).  W2 is a pair of words with the bit operations
// the excitations need, written out per word, so that the masks and shifts of the
// generation code read the same for both.  (An earlier form held two-word strings as
// unsigned __int128; in the generation kernel built for sm_103a the mask that clears an
// orbital p >= 64 also cleared orbital p - 64 in some excitations, which dropped an
// electron.  W2 has no 128-bit shifts.)
struct W2 {
    uint64_t lo, hi;
    __host__ __device__ constexpr W2(uint64_t l = 0, uint64_t h = 0) : lo(l), hi(h) {}
    __device__ explicit operator bool() const { return (lo | hi) != 0; }
    __device__ explicit operator uint64_t() const { return lo; }
};
__device__ __forceinline__ W2 operator&(W2 a, W2 b) { return W2(a.lo & b.lo, a.hi & b.hi); }
__device__ __forceinline__ W2 operator|(W2 a, W2 b) { return W2(a.lo | b.lo, a.hi | b.hi); }
__device__ __forceinline__ W2 operator~(W2 a) { return W2(~a.lo, ~a.hi); }
__device__ __forceinline__ W2 &operator&=(W2 &a, W2 b) { a.lo &= b.lo, a.hi &= b.hi; return a; }
// a - 1 (borrow into the high word)
__device__ __forceinline__ W2 operator-(W2 a, int one) { return W2(a.lo - (uint64_t)one, a.hi - (a.lo < (uint64_t)one ? 1ull : 0ull)); }
// logical right shift by 0 <= s < 128
__device__ __forceinline__ W2 operator>>(W2 a, int s)
{
    if (s == 0) return a;
    if (s < 64) return W2((a.lo >> s) | (a.hi << (64 - s)), a.hi >> s);
    return W2(a.hi >> (s - 64), 0);
}

// three words (up to 192 spinors), written out the same way
struct W3 {
    uint64_t w0, w1, w2;
    __host__ __device__ constexpr W3(uint64_t a = 0, uint64_t b = 0, uint64_t c = 0) : w0(a), w1(b), w2(c) {}
    __device__ explicit operator bool() const { return (w0 | w1 | w2) != 0; }
};
__device__ __forceinline__ W3 operator&(W3 a, W3 b) { return W3(a.w0 & b.w0, a.w1 & b.w1, a.w2 & b.w2); }
__device__ __forceinline__ W3 operator|(W3 a, W3 b) { return W3(a.w0 | b.w0, a.w1 | b.w1, a.w2 | b.w2); }
__device__ __forceinline__ W3 operator~(W3 a) { return W3(~a.w0, ~a.w1, ~a.w2); }
__device__ __forceinline__ W3 &operator&=(W3 &a, W3 b) { a.w0 &= b.w0, a.w1 &= b.w1, a.w2 &= b.w2; return a; }
// a - 1 (borrows through the words)
__device__ __forceinline__ W3 operator-(W3 a, int one)
{
    const uint64_t u = (uint64_t)one;
    const uint64_t b0 = a.w0 < u ? 1ull : 0ull, b1 = a.w1 < b0 ? 1ull : 0ull;
    return W3(a.w0 - u, a.w1 - b0, a.w2 - b1);
}

template <int KW> struct KeyOf;
template <> struct KeyOf<1> { using T = uint64_t; };
template <> struct KeyOf<2> { using T = W2; };
template <> struct KeyOf<3> { using T = W3; };

__device__ __forceinline__ int popck(uint64_t x) { return __popcll(x); }
__device__ __forceinline__ int popck(W2 x) { return __popcll(x.lo) + __popcll(x.hi); }
__device__ __forceinline__ int popck(W3 x) { return __popcll(x.w0) + __popcll(x.w1) + __popcll(x.w2); }
// lowest set bit (x != 0)
__device__ __forceinline__ int lowbit(uint64_t x) { return __ffsll((long long)x) - 1; }
__device__ __forceinline__ int lowbit(W2 x)
{
    return x.lo ? __ffsll((long long)x.lo) - 1 : 64 + __ffsll((long long)x.hi) - 1;
}
__device__ __forceinline__ int lowbit(W3 x)
{
    return x.w0 ? __ffsll((long long)x.w0) - 1
                : x.w1 ? 64 + __ffsll((long long)x.w1) - 1 : 128 + __ffsll((long long)x.w2) - 1;
}
template <typename K> __device__ __forceinline__ K bitk(int p);
template <> __device__ __forceinline__ uint64_t bitk<uint64_t>(int p) { return 1ull << p; }
template <> __device__ __forceinline__ W2 bitk<W2>(int p) { return p < 64 ? W2(1ull << p, 0) : W2(0, 1ull << (p - 64)); }
template <> __device__ __forceinline__ W3 bitk<W3>(int p)
{
    const uint64_t b = 1ull << (p & 63);
    return W3(p < 64 ? b : 0ull, p >= 64 && p < 128 ? b : 0ull, p >= 128 ? b : 0ull);
}
__device__ __forceinline__ bool has(uint64_t k, int p) { return (k >> p) & 1; }
__device__ __forceinline__ bool has(W2 k, int p) { return p < 64 ? (k.lo >> p) & 1 : (k.hi >> (p - 64)) & 1; }
__device__ __forceinline__ bool has(W3 k, int p) { return ((p < 64 ? k.w0 : p < 128 ? k.w1 : k.w2) >> (p & 63)) & 1; }
// occupied orbitals of k below orbital x
template <typename K> __device__ __forceinline__ int belowk(K k, int x) { return popck(k & (bitk<K>(x) - 1)); }
template <int KW> __device__ __forceinline__ typename KeyOf<KW>::T load_key(const uint64_t *keys, int64_t J)
{
    if constexpr (KW == 1) return keys[J];
    else if constexpr (KW == 2) return W2(keys[2 * J], keys[2 * J + 1]);
    else return W3(keys[3 * J], keys[3 * J + 1], keys[3 * J + 2]);
}
template <typename K> __device__ __forceinline__ K ref_of(const Pt2 &p)
{
    if constexpr (sizeof(K) == 8) return p.ref;
    else if constexpr (sizeof(K) == 16) return W2(p.ref, p.ref_hi);
    else return W3(p.ref, p.ref_hi, p.ref_w2);
}
__device__ __forceinline__ uint64_t key_lo(W2 x) { return x.lo; }
__device__ __forceinline__ uint64_t key_hi(W2 x) { return x.hi; }
__device__ __forceinline__ uint64_t key_lo(W3 x) { return x.w0; }
__device__ __forceinline__ uint64_t key_hi(W3 x) { return x.w1; }
__device__ __forceinline__ uint64_t hash_key(uint64_t x) { return mix64(x); }
__device__ __forceinline__ uint64_t hash_key(W2 x) { return mix64(x.lo ^ mix64(x.hi + 0x9e3779b97f4a7c15ull)); }
__device__ __forceinline__ uint64_t hash_key(W3 x)
{
    return mix64(x.w0 ^ mix64(x.w1 + 0x9e3779b97f4a7c15ull) ^ mix64(x.w2 + 0x632be59bd9b4e019ull));
}

// H_IJ for I = J - {i, j} + {a, b} (i < j, a < b, spin-orbital indices)
template <typename K>
__device__ __forceinline__ double h_double(const Pt2 &p, K J, int i, int j, int a, int b)
{
    const K Kh = J & ~bitk<K>(i) & ~bitk<K>(j);
    uint32_t rowoff, colbase, r2, c2;
    const sci::TabRule tr{0, p.n};
    sci::pair_offsets(tr, a, b, rowoff, r2);      // bra (I) extras
    sci::pair_offsets(tr, i, j, c2, colbase);     // ket (J) extras
    const bool ph = (belowk(Kh, a) + belowk(Kh, b) + belowk(Kh, i) + belowk(Kh, j)) & 1;
    return sflip(ph, __ldg(p.tab + rowoff + colbase));
}

// H_IJ for I = J - {i} + {a}
template <typename K>
__device__ __forceinline__ double h_single(const Pt2 &p, K J, int i, int a)
{
    const K S = J & ~bitk<K>(i), ref = ref_of<K>(p);
    const int norb = p.norb;
    double f = __ldg(p.fref + i * norb + a);
    const K part = S & ~ref, holes = ref & ~S;
    for (K m = part; m; m &= m - 1) f += __ldg(p.g_so + ((int64_t)lowbit(m) * norb + i) * norb + a);
    for (K m = holes; m; m &= m - 1) f -= __ldg(p.g_so + ((int64_t)lowbit(m) * norb + i) * norb + a);
    const bool ph = (belowk(S, a) + belowk(S, i)) & 1;
    return sflip(ph, f);
}

// The slot of key I in a table of (key, NW value words) slots, claimed if I is new (nc
// counts the thread's claims: the kernel adds them to the distinct count once per warp at
// its end, and the host compares that count with the load limit, instead of one add to a
// single counter per claim); NULL after kMaxProbe probes (the table is too full: flag bit 2).
//
// Slots: KW key words, then NW value words; with two or three key words the slot is padded
// to an even number of words, so that every slot is 16-byte aligned for the 128-bit CAS.
// With three key words the third is stored complemented, so that 0 still marks a slot
// whose third word is not yet set (a determinant of fewer than 64 electrons never has all
// of orbitals 128..191 occupied).
template <int KW, int NW> __host__ __device__ constexpr int slot_words() { return KW == 1 ? 1 + NW : (KW + NW + 1) & ~1; }

// 128-bit compare-and-swap (sm_90 and later): [a] = n if [a] == e; returns the old value
__device__ __forceinline__ void cas128(uint64_t *a, uint64_t e0, uint64_t e1, uint64_t n0, uint64_t n1, uint64_t &r0,
                                       uint64_t &r1)
{
    unsigned long long o0, o1;
    asm volatile("{\n\t.reg .b128 d, b, c;\n\tmov.b128 b, {%2, %3};\n\tmov.b128 c, {%4, %5};\n\t"
                 "atom.global.cas.b128 d, [%6], b, c;\n\tmov.b128 {%0, %1}, d;\n\t}"
                 : "=l"(o0), "=l"(o1)
                 : "l"((unsigned long long)e0), "l"((unsigned long long)e1), "l"((unsigned long long)n0),
                   "l"((unsigned long long)n1), "l"((unsigned long long)__cvta_generic_to_global(a))
                 : "memory");
    r0 = o0, r1 = o1;
}

template <int KW, int NW, typename K>
__device__ __forceinline__ uint64_t *claim(const Pt2 &p, K I, uint32_t &nc)
{
    constexpr int SW = slot_words<KW, NW>();
    uint64_t s = hash_key(I) & p.mask;
    for (int probe = 0; probe < kMaxProbe; probe++) {
        uint64_t *slot = p.tab2 + s * SW;
        if constexpr (KW == 1) {
            uint64_t k = *slot;
            if (k == kEmpty) {
                k = atomicCAS(reinterpret_cast<unsigned long long *>(slot), (unsigned long long)kEmpty,
                              (unsigned long long)I);
                if (k == kEmpty) {
                    nc++;
                    k = I;
                }
            }
            if (k == I) return slot;   // the value words share the key's sector
        } else {
            // one atomic per probe: a plain 16-byte read of a key being written could be torn
            const uint64_t lo = key_lo(I), hi = key_hi(I);
            uint64_t r0, r1;
            cas128(slot, 0, 0, lo, hi, r0, r1);
            const bool first = (r0 | r1) == 0;
            if constexpr (KW == 2) {
                if (first) {
                    nc++;
                    return slot;
                }
                if (r0 == lo && r1 == hi) return slot;
            } else {
                // three words: the first two are claimed together; the slot's third word is
                // then set by a 64-bit CAS from 0 by whichever thread with those two words
                // gets there first (its claimer or another), and that key owns the slot.
                // No thread waits on another: one whose third word lost probes on.
                if (first || (r0 == lo && r1 == hi)) {
                    const unsigned long long w2 = ~I.w2;
                    const unsigned long long o =
                        atomicCAS(reinterpret_cast<unsigned long long *>(slot + 2), 0ull, w2);
                    if (o == 0ull) {
                        nc++;
                        return slot;
                    }
                    if (o == w2) return slot;
                }
            }
        }
        s = (s + 1) & p.mask;
    }
    atomicOr(p.flag, 2);  // probe limit: the table is too full
    return nullptr;
}

template <int R, int KW, typename K>
__device__ __forceinline__ void insert(const Pt2 &p, K I, double hij, const double *cJ, double cmax, uint32_t &nc)
{
    if (p.eps > 0.0 && fabs(hij) * cmax < p.eps) return;
    uint64_t *slot = claim<KW, R>(p, I, nc);
    if (!slot) return;
#pragma unroll
    for (int v = 0; v < R; v++) atomicAdd(reinterpret_cast<double *>(slot + KW + v), hij * cJ[v]);
}

// The alpha (bits 0..n-1) and beta (bits n..2n-1) strings of a spin-orbital key.  One-
// and two-word keys give 32- or 64-bit strings (n <= 64); three-word keys (n <= 96) give
// two-word strings.
template <typename S, typename K> __device__ __forceinline__ void split_ab(K key, int n, S full, S &oa, S &ob)
{
    if constexpr (sizeof(K) == 24) {
        // key >> n, its low 128 bits (0 < n <= 96: word 2 reaches at most bit 191 - n)
        const int q = n >> 6, r = n & 63;
        const uint64_t w[4] = {key.w0, key.w1, key.w2, 0ull};
        const uint64_t lo = r ? (w[q] >> r) | (w[q + 1] << (64 - r)) : w[q];
        const uint64_t hi = r ? (w[q + 1] >> r) | (w[q + 2] << (64 - r)) : w[q + 1];
        oa = W2(key.w0, key.w1) & full;
        ob = W2(lo, hi) & full;
    } else {
        oa = (S)(uint64_t)key & full;
        ob = (S)(uint64_t)(key >> n) & full;
    }
}

// orbital o of a string of the spin-orbital generator (32- or 64-bit, or two words)
__device__ __forceinline__ bool bit_of(uint32_t s, int o) { return (s >> o) & 1u; }
__device__ __forceinline__ bool bit_of(uint64_t s, int o) { return (s >> o) & 1ull; }
__device__ __forceinline__ bool bit_of(W2 s, int o) { return has(s, o); }

// the batch code of a string: XOR of the codes of its occupied orbitals
__device__ __forceinline__ uint32_t code_of64(const uint32_t *g, uint64_t s)
{
    uint32_t c = 0;
    for (; s; s &= s - 1) c ^= g[__ffsll((long long)s) - 1];
    return c;
}
__device__ __forceinline__ uint32_t code_ofk(const uint32_t *g, uint64_t s) { return code_of64(g, s); }
__device__ __forceinline__ uint32_t code_ofk(const uint32_t *g, W2 s) { return code_of64(g, s.lo) ^ code_of64(g + 64, s.hi); }
__device__ __forceinline__ uint32_t code_ofk(const uint32_t *g, W3 s)
{
    return code_of64(g, s.w0) ^ code_of64(g + 64, s.w1) ^ code_of64(g + 128, s.w2);
}

// the claims of a warp's threads, added to the distinct count once
__device__ __forceinline__ void add_claims(const Pt2 &p, uint32_t nc, int lane)
{
    unsigned long long t = nc;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0 && t) atomicAdd(p.count, t);
}

// A warp's queue of found excitations (packed orbital quadruples), in shared memory, 64
// entries.  The code lookups find 0, 1 or a few second virtuals per (pair, first virtual)
// class, so a lane that inserted its own finds would leave most of the warp idle; the
// finds of a step are appended by ballot instead, and each time 32 are queued every lane
// inserts one.  `cnt` is the same in every lane.  Spinor mode, 120k-determinant 64-spinor
// space, 1 GB table: 10 -> 27 active lanes per instruction, 8.9 -> 3.3 ms per generation
// launch (ncu), 1.09 -> 0.88 s for the whole sum.
template <typename F>
__device__ __forceinline__ void wq_push(uint32_t *q, int &cnt, bool hit, uint32_t e, int lane, F &&proc)
{
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) q[cnt + __popc(m & ((1u << lane) - 1u))] = e;
    cnt += __popc(m);
    __syncwarp();
    if (cnt >= 32) {
        proc(q[lane]);
        __syncwarp();
        cnt -= 32;
        if (lane < cnt) q[lane] = q[32 + lane];
        __syncwarp();
    }
}

template <typename F>
__device__ __forceinline__ void wq_flush(uint32_t *q, int &cnt, int lane, F &&proc)
{
    if (lane < cnt) proc(q[lane]);
    __syncwarp();
    cnt = 0;
}

// warp per determinant J of P: the excitations of J that fall in batch `batch`.  KW = 1:
// n <= 32 orbitals per spin (one-word keys); KW = 2: n <= 64; KW = 3: n <= 96.
template <int R, int KW>
// (one-word keys, one or two roots: held to 40 registers, 6 CTAs per SM, as the kernel
// was before the two-word form; at 48 registers the 2M-space sum took 8.6 s, at 40 8.05 s)
// KW = 3: n <= 96 orbitals per spin; the pair table is then decoded arithmetically and
// the beta-singles list holds (n/2)^2 entries, so that the static shared memory stays
// under 48 KB.
__global__ void __launch_bounds__(kThreads, KW == 1 && R <= 2 ? 6 : 1)
k_pt2_gen(const uint64_t *__restrict__ Pkeys, int64_t M, const double *__restrict__ C, Pt2 p, uint32_t batch, int tbits)
{
    using K = typename KeyOf<KW>::T;
    constexpr int NO = 32 * KW;                   // orbitals per spin at most
    constexpr int kMP = NO * (NO - 1) / 2;        // their unordered pairs
    constexpr int kNL = (NO / 2) * (NO / 2);      // beta singles at most (nb (n - nb))
    __shared__ uint8_t s_orb[kWarps][4 * NO];     // occ alpha | vir alpha | occ beta | vir beta
    __shared__ uint16_t s_list[kWarps][kNL];      // beta singles of this batch (j | v << 8)
    __shared__ uint16_t s_pair[KW == 3 ? 1 : kMP];   // P -> (a, b)
    __shared__ uint8_t s_cstart[(1 << kMaxBits) + 1];
    __shared__ uint8_t s_obc[NO];                 // beta orbitals sorted by code
    __shared__ uint32_t s_g[NO];                  // beta-orbital codes
    __shared__ int s_nl[kWarps];
    if constexpr (KW != 3)
        for (int P = threadIdx.x; P < kMP; P += blockDim.x) {
            int y = 1;
            while ((y + 1) * y / 2 <= P) y++;
            s_pair[P] = (uint16_t)((P - y * (y - 1) / 2) | (y << 8));
        }
    // pair P = y(y-1)/2 + x, x < y -> x | y << 8
    auto pair_of = [&](int P) -> uint16_t {
        if constexpr (KW != 3) {
            return s_pair[P];
        } else {
            int y = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)P)) * 0.5f);
            while (y * (y - 1) / 2 > P) y--;
            while ((y + 1) * y / 2 <= P) y++;
            return (uint16_t)((P - y * (y - 1) / 2) | (y << 8));
        }
    };
    for (int c = threadIdx.x; c <= (1 << tbits); c += blockDim.x) s_cstart[c] = p.cstart[c];
    if (threadIdx.x < NO) s_obc[threadIdx.x] = p.obc[threadIdx.x], s_g[threadIdx.x] = p.gcode[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint8_t *orb = s_orb[w];
    // alpha and beta strings: 32-bit words for one-word keys (fewer registers), 64-bit
    // for two, two words for three
    using S = std::conditional_t<KW == 1, uint32_t, std::conditional_t<KW == 2, uint64_t, W2>>;
    const int n = p.n, na = p.na, nb = p.nb, ua = n - na, ub = n - nb;
    S full;
    if constexpr (KW == 3) full = bitk<W2>(n) - 1;
    else full = n == 8 * (int)sizeof(S) ? ~(S)0 : (S)((1ull << n) - 1);
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    uint32_t nclaim = 0;
    for (int64_t J = (int64_t)blockIdx.x * kWarps + w; J < M; J += warps_total) {
        const K key = load_key<KW>(Pkeys, J);
        S oa, ob;
        split_ab<S>(key, n, full, oa, ob);
        const S va = full & ~oa, vb = full & ~ob;
        double cJ[R], cmax = 0.0;
#pragma unroll
        for (int v = 0; v < R; v++) cJ[v] = C[J * R + v], cmax = fmax(cmax, fabs(cJ[v]));
        __syncwarp();
        for (int o = lane; o < n; o += 32) {
            if constexpr (KW == 3) {
                const W2 lm = bitk<W2>(o) - 1;
                if (has(oa, o)) orb[popck(oa & lm)] = (uint8_t)o;
                else orb[NO + popck(va & lm)] = (uint8_t)o;
                if (has(ob, o)) orb[2 * NO + popck(ob & lm)] = (uint8_t)o;
                else orb[3 * NO + popck(vb & lm)] = (uint8_t)o;
            } else {
                const S lm = (S)((1ull << o) - 1);
                if ((oa >> o) & 1) orb[__popcll(oa & lm)] = (uint8_t)o;
                else orb[NO + __popcll(va & lm)] = (uint8_t)o;
                if ((ob >> o) & 1) orb[2 * NO + __popcll(ob & lm)] = (uint8_t)o;
                else orb[3 * NO + __popcll(vb & lm)] = (uint8_t)o;
            }
        }
        __syncwarp();
        uint32_t target;
        if constexpr (KW == 3) target = batch ^ code_ofk(s_g, ob);
        else target = batch ^ code_of64(s_g, ob);

        // alpha singles and alpha-alpha doubles: the beta string is unchanged
        if (target == 0) {
            const int c0 = na * ua, qa = ua * (ua - 1) / 2, c2 = na * (na - 1) / 2 * qa;
            for (int t = lane; t < c0 + c2; t += 32) {
                if (t < c0) {
                    const int i = orb[t / ua], a = orb[NO + t % ua];
                    insert<R, KW>(p, (key & ~bitk<K>(i)) | bitk<K>(a), h_single(p, key, i, a), cJ, cmax, nclaim);
                } else {
                    const int s = t - c0;
                    const uint16_t po = pair_of(s / qa), pv = pair_of(s % qa);
                    const int i = orb[po & 0xFF], j = orb[po >> 8], a = orb[NO + (pv & 0xFF)], b = orb[NO + (pv >> 8)];
                    if (p.bss && p.bss[j * (j - 1) / 2 + i] * cmax < p.eps) continue;   // the class's bound
                    const K I = (key & ~bitk<K>(i) & ~bitk<K>(j)) | bitk<K>(a) | bitk<K>(b);
                    insert<R, KW>(p, I, h_double(p, key, i, j, a, b), cJ, cmax, nclaim);
                }
            }
        }

        // beta singles j -> v of this batch (g(v) = target ^ g(j)), and the alpha-beta
        // doubles built on them
        if (lane == 0) s_nl[w] = 0;
        __syncwarp();
        for (int x = lane; x < nb; x += 32) {
            const int j = orb[2 * NO + x];
            const uint32_t c = target ^ s_g[j];
            for (int q = s_cstart[c]; q < s_cstart[c + 1]; q++) {
                const int v = s_obc[q];
                if (bit_of(ob, v)) continue;
                const int slot = atomicAdd(&s_nl[w], 1);
                s_list[w][slot] = (uint16_t)(j | (v << 8));
            }
        }
        __syncwarp();
        const int nl = s_nl[w], c0 = na * ua;
        for (int t = lane; t < nl * (1 + c0); t += 32) {
            const uint16_t e = s_list[w][t / (1 + c0)];
            const int jb = n + (e & 0xFF), vb_ = n + (e >> 8);
            const int s = t % (1 + c0);
            if (s == 0) {
                insert<R, KW>(p, (key & ~bitk<K>(jb)) | bitk<K>(vb_), h_single(p, key, jb, vb_), cJ, cmax, nclaim);
            } else {
                const int i = orb[(s - 1) / ua], a = orb[NO + (s - 1) % ua];
                if (p.bab && p.bab[(e & 0xFF) * n + i] * cmax < p.eps) continue;   // the class's bound
                const K I = (key & ~bitk<K>(i) & ~bitk<K>(jb)) | bitk<K>(a) | bitk<K>(vb_);
                insert<R, KW>(p, I, h_double(p, key, i, jb, a, vb_), cJ, cmax, nclaim);
            }
        }

        // beta-beta doubles j1 < j2 -> b1 < b2: for each occupied pair and first virtual
        // b1, the second virtual has code target ^ g(j1) ^ g(j2) ^ g(b1).  (A warp queue
        // as in spinor mode made the 2M-space sum slower here: 7.9 -> 9.4 s.)
        const int pb = nb * (nb - 1) / 2;
        for (int t = lane; t < pb * ub; t += 32) {
            const uint16_t po = pair_of(t / ub);
            const int j1 = orb[2 * NO + (po & 0xFF)], j2 = orb[2 * NO + (po >> 8)], b1 = orb[3 * NO + t % ub];
            if (p.bss3 && p.bss3[(j2 * (j2 - 1) / 2 + j1) * n + b1] * cmax < p.eps) continue;   // the class's bound
            const uint32_t c = target ^ s_g[j1] ^ s_g[j2] ^ s_g[b1];
            for (int q = s_cstart[c]; q < s_cstart[c + 1]; q++) {
                const int b2 = s_obc[q];
                if (b2 <= b1 || bit_of(ob, b2)) continue;
                const K I = (key & ~bitk<K>(n + j1) & ~bitk<K>(n + j2)) | bitk<K>(n + b1) | bitk<K>(n + b2);
                insert<R, KW>(p, I, h_double(p, key, n + j1, n + j2, n + b1, n + b2), cJ, cmax, nclaim);
            }
        }
        __syncwarp();
    }
    add_claims(p, nclaim, lane);
}


// ------------------------------------------------------------------ spinor mode
using sci::zdbl;

__device__ __forceinline__ zdbl ldz(const zdbl *p)
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return zdbl{v.x, v.y};
}

// H_IJ (spinors) for I = J - {i, j} + {a, b}: the antisymmetrised table entry of the bra
// pair (a, b) and the ket pair (i, j), with the phase of the sigma kernels
template <typename K>
__device__ __forceinline__ zdbl hz_double(const Pt2 &p, K J, int i, int j, int a, int b)
{
    const K Kh = J & ~bitk<K>(i) & ~bitk<K>(j);
    uint32_t rowoff, colbase, r2, c2;
    const sci::TabRule tr{1, p.n};
    sci::pair_offsets(tr, a, b, rowoff, r2);
    sci::pair_offsets(tr, i, j, c2, colbase);
    const bool ph = (belowk(Kh, a) + belowk(Kh, b) + belowk(Kh, i) + belowk(Kh, j)) & 1;
    return sflip(ph, ldz(reinterpret_cast<const zdbl *>(p.tab) + rowoff + colbase));
}

// H_IJ (spinors) for I = J - {i} + {a}: F^ref_ai plus the terms of the spinors where
// S = J - {i} and the reference differ
template <typename K>
__device__ __forceinline__ zdbl hz_single(const Pt2 &p, K J, int i, int a)
{
    const K S = J & ~bitk<K>(i), ref = ref_of<K>(p);
    const int norb = p.norb;
    const zdbl *fref = reinterpret_cast<const zdbl *>(p.fref), *g = reinterpret_cast<const zdbl *>(p.g_so);
    zdbl f = ldz(fref + i * norb + a);
    const K part = S & ~ref, holes = ref & ~S;
    for (K m = part; m; m &= m - 1) {
        const zdbl t = ldz(g + ((int64_t)lowbit(m) * norb + i) * norb + a);
        f.x += t.x, f.y += t.y;
    }
    for (K m = holes; m; m &= m - 1) {
        const zdbl t = ldz(g + ((int64_t)lowbit(m) * norb + i) * norb + a);
        f.x -= t.x, f.y -= t.y;
    }
    const bool ph = (belowk(S, a) + belowk(S, i)) & 1;
    return sflip(ph, f);
}

template <int R, int KW, typename K>
__device__ __forceinline__ void insert_z(const Pt2 &p, K I, zdbl h, const zdbl *cJ, double cmax, uint32_t &nc)
{
    if (p.eps > 0.0 && sqrt(h.x * h.x + h.y * h.y) * cmax < p.eps) return;
    uint64_t *slot = claim<KW, 2 * R>(p, I, nc);
    if (!slot) return;
    double *val = reinterpret_cast<double *>(slot + KW);
#pragma unroll
    for (int v = 0; v < R; v++) {
        atomicAdd(val + 2 * v, h.x * cJ[v].x - h.y * cJ[v].y);
        atomicAdd(val + 2 * v + 1, h.x * cJ[v].y + h.y * cJ[v].x);
    }
}

// warp per determinant J of P: the excitations of J (spinors) that fall in batch `batch`.
// KW = 1: n <= 64 spinors (one-word keys); KW = 2: n <= 128; KW = 3: n <= 192.
template <int R, int KW>
__global__ void __launch_bounds__(kThreads)
k_pt2_gen_z(const uint64_t *__restrict__ Pkeys, int64_t M, const zdbl *__restrict__ C, Pt2 p, uint32_t batch, int tbits)
{
    using K = typename KeyOf<KW>::T;
    constexpr int NZ = 64 * KW;                  // spinors at most
    constexpr int kMP = NZ * (NZ - 1) / 2;       // pairs x < y, P = y(y-1)/2 + x -> x | y << 8
    __shared__ uint8_t s_orb[kWarps][2 * NZ];    // occupied spinors | virtual spinors (+ NZ)
    __shared__ uint16_t s_pair[kMP];
    __shared__ uint8_t s_cstart[(1 << kMaxBits) + 1];
    __shared__ uint8_t s_obc[NZ];                // spinors sorted by code
    __shared__ uint32_t s_g[NZ];                 // spinor codes
    __shared__ uint32_t s_q[kWarps][64];         // the warp's queue of double finds
    for (int P = threadIdx.x; P < kMP; P += blockDim.x) {
        int y = 1;
        while ((y + 1) * y / 2 <= P) y++;
        s_pair[P] = (uint16_t)((P - y * (y - 1) / 2) | (y << 8));
    }
    for (int c = threadIdx.x; c <= (1 << tbits); c += blockDim.x) s_cstart[c] = p.cstart[c];
    if (threadIdx.x < NZ) s_obc[threadIdx.x] = p.obc[threadIdx.x], s_g[threadIdx.x] = p.gcode[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint8_t *orb = s_orb[w];
    const int n = p.n, N = p.na, nv = n - N;
    const K full = n == 8 * (int)sizeof(K) ? ~(K)0 : bitk<K>(n) - 1;
    const int npairs = N * (N - 1) / 2;
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    uint32_t nclaim = 0;
    for (int64_t J = (int64_t)blockIdx.x * kWarps + w; J < M; J += warps_total) {
        const K key = load_key<KW>(Pkeys, J);
        const K vir = full & ~key;
        zdbl cJ[R];
        double cmax = 0.0;
#pragma unroll
        for (int v = 0; v < R; v++) {
            cJ[v] = C[J * R + v];
            cmax = fmax(cmax, sqrt(cJ[v].x * cJ[v].x + cJ[v].y * cJ[v].y));
        }
        __syncwarp();
        for (int o = lane; o < n; o += 32) {
            const K lm = bitk<K>(o) - 1;
            if (has(key, o)) orb[popck(key & lm)] = (uint8_t)o;
            else orb[NZ + popck(vir & lm)] = (uint8_t)o;
        }
        __syncwarp();
        const uint32_t target = batch ^ code_ofk(s_g, key);
        // singles i -> a of this batch: g(a) = target ^ g(i)
        for (int x = lane; x < N; x += 32) {
            const int i = orb[x];
            const uint32_t c = target ^ s_g[i];
            for (int q = s_cstart[c]; q < s_cstart[c + 1]; q++) {
                const int a = s_obc[q];
                if (has(key, a)) continue;
                insert_z<R, KW>(p, (key & ~bitk<K>(i)) | bitk<K>(a), hz_single(p, key, i, a), cJ, cmax, nclaim);
            }
        }
        // doubles i < j -> a < b: for each occupied pair and first virtual a, the second
        // virtual has code target ^ g(i) ^ g(j) ^ g(a); the finds go through the warp's queue
        auto ins = [&](uint32_t e) {
            const int i = e & 0xFF, j = (e >> 8) & 0xFF, a = (e >> 16) & 0xFF, b = e >> 24;
            const K I = (key & ~bitk<K>(i) & ~bitk<K>(j)) | bitk<K>(a) | bitk<K>(b);
            insert_z<R, KW>(p, I, hz_double(p, key, i, j, a, b), cJ, cmax, nclaim);
        };
        int cnt = 0;
        for (int base = 0; base < npairs * nv; base += 32) {
            const int t = base + lane;
            int q = 0, qe = 0, i = 0, j = 0, a = 0;
            if (t < npairs * nv) {
                const uint16_t po = s_pair[t / nv];
                i = orb[po & 0xFF], j = orb[po >> 8], a = orb[NZ + t % nv];
                if (!(p.bss3 && p.bss3[(j * (j - 1) / 2 + i) * n + a] * cmax < p.eps)) {   // the class's bound
                    const uint32_t c = target ^ s_g[i] ^ s_g[j] ^ s_g[a];
                    q = s_cstart[c], qe = s_cstart[c + 1];
                }
            }
            for (; __any_sync(0xffffffffu, q < qe); q++) {
                bool hit = false;
                int b = 0;
                if (q < qe) {
                    b = s_obc[q];
                    hit = b > a && !has(key, b);
                }
                wq_push(s_q[w], cnt, hit, (uint32_t)i | (uint32_t)j << 8 | (uint32_t)a << 16 | (uint32_t)b << 24, lane,
                        ins);
            }
        }
        wq_flush(s_q[w], cnt, lane, ins);
    }
    add_claims(p, nclaim, lane);
}

// sum over the table entries of num^2 / (E0 - H_II).  Each warp packs the occupied slots
// it scans into a buffer of 32 and evaluates full buffers, so every lane works; H_II
// (E_ref plus O(level^2) table terms) is summed in paired FP32 from split copies of F and
// G in shared memory, and added to E_ref in FP64.
// GS: G in shared memory (up to 168 orbitals); else read from global memory and split on
// the fly.
template <int R, bool CPLX, int KW, bool GS = true>
__global__ void __launch_bounds__(kThreads)
k_pt2_eval(Pt2 p, uint64_t cap, const double *__restrict__ E0, double *__restrict__ out)
{
    using K = typename KeyOf<KW>::T;
    constexpr int NW = CPLX ? 2 * R : R;   // value words per slot
    constexpr int SW = slot_words<KW, NW>();
    extern __shared__ float2 s_gf[];       // F [norb], then G [norb][norb] (dynamic)
    __shared__ uint64_t sbuf[kWarps][64];
    __shared__ double red[kWarps][R];
    const int norb = p.norb;
    float2 *sF = s_gf, *sGs = s_gf + norb;
    for (int t = threadIdx.x; t < norb; t += blockDim.x) sF[t] = sci::ds_split_int(p.fdiag[t]);
    if constexpr (GS)
        for (int t = threadIdx.x; t < norb * norb; t += blockDim.x) sGs[t] = sci::ds_split_int(p.G[t]);
    __syncthreads();
    auto gget = [&](int t) -> float2 {
        if constexpr (GS) return sGs[t];
        else return sci::ds_split_int(__ldg(p.G + t));
    };
    const double Eref = *p.Eref;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double acc[R], e0[R];
#pragma unroll
    for (int v = 0; v < R; v++) acc[v] = 0.0, e0[v] = E0[v];
    const K ref = ref_of<K>(p);
    auto evaluate = [&](uint64_t s) {
        const uint64_t *slot = p.tab2 + s * SW;
        K I;
        if constexpr (KW == 1) I = slot[0];
        else if constexpr (KW == 2) I = W2(slot[0], slot[1]);
        else I = W3(slot[0], slot[1], ~slot[2]);
        const K H = ref & ~I, Pm = I & ~ref;
        sci::Ds e;
        sci::ds_zero(e);
        for (K m = H; m; m &= m - 1) {
            const int i = lowbit(m);
            const float2 f = sF[i];
            sci::ds_add(e, make_float2(-f.x, -f.y));
            for (K m2 = m & (m - 1); m2; m2 &= m2 - 1) sci::ds_add(e, gget(i * norb + lowbit(m2)));
            for (K m2 = Pm; m2; m2 &= m2 - 1) {
                const float2 g = gget(i * norb + lowbit(m2));
                sci::ds_add(e, make_float2(-g.x, -g.y));
            }
        }
        for (K m = Pm; m; m &= m - 1) {
            const int a = lowbit(m);
            sci::ds_add(e, sF[a]);
            for (K m2 = m & (m - 1); m2; m2 &= m2 - 1) sci::ds_add(e, gget(a * norb + lowbit(m2)));
        }
        const double hii = Eref + sci::ds_value(e);
#pragma unroll
        for (int v = 0; v < R; v++) {
            double num2;
            if constexpr (CPLX) {
                const double re = __longlong_as_double((long long)slot[KW + 2 * v]);
                const double im = __longlong_as_double((long long)slot[KW + 1 + 2 * v]);
                num2 = re * re + im * im;
            } else {
                const double num = __longlong_as_double((long long)slot[KW + v]);
                num2 = num * num;
            }
            acc[v] += num2 / (e0[v] - hii);
        }
    };
    int nbuf = 0;  // occupied slots waiting in this warp's buffer (warp-uniform)
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t s0 = (uint64_t)blockIdx.x * kThreads + (uint64_t)w * 32; s0 < cap; s0 += stride) {
        const uint64_t s = s0 + lane;
        bool occ = false;
        if (s < cap) {
            const uint64_t *slot = p.tab2 + s * SW;
            occ = KW == 1 ? slot[0] != kEmpty : KW == 2 ? (slot[0] | slot[1]) != kEmpty : slot[2] != 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, occ);
        if (occ) sbuf[w][nbuf + __popc(m & ((1u << lane) - 1))] = s;
        nbuf += __popc(m);
        __syncwarp();
        if (nbuf >= 32) {
            evaluate(sbuf[w][lane]);
            __syncwarp();
            if (lane < nbuf - 32) sbuf[w][lane] = sbuf[w][32 + lane];
            nbuf -= 32;
            __syncwarp();
        }
    }
    if (lane < nbuf) evaluate(sbuf[w][lane]);
#pragma unroll
    for (int v = 0; v < R; v++) {
        double x = acc[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < R) {
        double x = 0.0;
        for (int i = 0; i < kWarps; i++) x += red[i][threadIdx.x];
        atomicAdd(out + threadIdx.x, x);
    }
}

// E2[P] of Eq. EP1 from sigma = H c and the diagonal
__device__ __forceinline__ double abs2_minus(double s, double c, double d) { const double x = s - c * d; return x * x; }
__device__ __forceinline__ double abs2_minus(zdbl s, zdbl c, double d)
{
    const double x = s.x - c.x * d, y = s.y - c.y * d;
    return x * x + y * y;
}

template <int R, typename T>
__global__ void __launch_bounds__(kThreads)
k_pt2_p(int64_t M, const T *__restrict__ C, const T *__restrict__ S, const double *__restrict__ hdiag,
        const double *__restrict__ E0, double *__restrict__ out)
{
    __shared__ double red[kWarps][R];
    double acc[R];
#pragma unroll
    for (int v = 0; v < R; v++) acc[v] = 0.0;
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < M; I += (int64_t)gridDim.x * blockDim.x) {
        const double d = hdiag[I];
#pragma unroll
        for (int v = 0; v < R; v++) acc[v] += abs2_minus(S[I * R + v], C[I * R + v], d) / (E0[v] - d);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < R; v++) {
        double x = acc[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < R) {
        double x = 0.0;
        for (int i = 0; i < kWarps; i++) x += red[i][threadIdx.x];
        atomicAdd(out + threadIdx.x, x);
    }
}

// G = (pp|qq) - (pq|qp) without the diagonal, the reference Fock diagonal and E_ref (real:
// for Hermitian integrals (pp|qq), (pq|qp) and h_pp are real, the imaginary parts zero)
__device__ __forceinline__ double re_of(double a) { return a; }
__device__ __forceinline__ double re_of(zdbl a) { return a.x; }

template <typename T>
__global__ void k_pt2_setup(int norb, uint64_t ref_lo, uint64_t ref_hi, uint64_t ref_w2, const T *__restrict__ h_so,
                            const T *__restrict__ jd, const T *__restrict__ kd, double *__restrict__ G,
                            double *__restrict__ fdiag, double *__restrict__ Eref)
{
    const W3 ref(ref_lo, ref_hi, ref_w2);
    for (int t = threadIdx.x; t < norb * norb; t += blockDim.x) {
        const int a = t / norb, b = t % norb;
        G[t] = a == b ? 0.0 : re_of(jd[t]) - re_of(kd[t]);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < norb; a += blockDim.x) {
        double f = re_of(h_so[a * norb + a]);
        for (W3 m = ref; m; m &= m - 1) f += G[a * norb + lowbit(m)];
        fdiag[a] = f;
    }
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (W3 m = ref; m; m &= m - 1) {
            const int i = lowbit(m);
            e += re_of(h_so[i * norb + i]);
            for (W3 m2 = m & (m - 1); m2; m2 &= m2 - 1) e += G[i * norb + lowbit(m2)];
        }
        *Eref = e;
    }
}


// Screening bounds of the double-excitation classes (see the header).  Real mode: the
// same-spin region W[P(i,j)][P(a,b)] (after the n^4 alpha-beta block T) and the alpha-beta
// block T[u_ket][u_bra] with u = j_beta * n + i_alpha; spinor mode: the complex W.
__device__ __forceinline__ double mag(double a) { return fabs(a); }
__device__ __forceinline__ double mag(zdbl a) { return sqrt(a.x * a.x + a.y * a.y); }

template <typename T>
__global__ void k_pt2_bounds3(int n, const T *__restrict__ W, double *__restrict__ b3)
{
    const int64_t NP = (int64_t)n * (n - 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NP * n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t Pij = t / n;
        const int a = (int)(t % n);
        double m = 0.0;
        for (int b = a + 1; b < n; b++) m = fmax(m, mag(W[Pij * NP + (int64_t)b * (b - 1) / 2 + a]));
        b3[t] = m;
    }
}

__global__ void k_pt2_bounds_pair(int n, const double *__restrict__ b3, double *__restrict__ b2)
{
    const int64_t NP = (int64_t)n * (n - 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NP; t += (int64_t)gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int a = 0; a < n; a++) m = fmax(m, b3[t * n + a]);
        b2[t] = m;
    }
}

__global__ void k_pt2_bounds_ab(int n, const double *__restrict__ T, double *__restrict__ bab)
{
    const int64_t n2 = (int64_t)n * n;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n2; u += (int64_t)gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int64_t r = 0; r < n2; r++) m = fmax(m, fabs(T[u * n2 + r]));
        bab[u] = m;
    }
}

int grid_for(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8));
}

// SPIN: complex spinor mode (C is [M][R] complex128); otherwise real spin-orbital mode.
// KW: key words (1, 2 or 3) of the determinant list.
template <int R, bool SPIN, int KW>
int pt2_run(sci_ctx *ctx, const double *C, const double *E0h, double eps, size_t table_bytes, double *E2, int64_t *stats)
{
    constexpr int NW = SPIN ? 2 * R : R;   // value words per table slot
    constexpr int SW = slot_words<KW, NW>();
    constexpr int SC = SPIN ? 2 : 1;       // doubles per coefficient
    const int64_t M = ctx->M;
    const int n = ctx->n, norb = ctx->norb, na = ctx->na, nb = ctx->nb;
    cudaStream_t st = ctx->stream;
    // scratch: sigma [M][R], E0 [R], results W/P [2R], G, fdiag, Eref, count, flag
    double *S = nullptr, *small = nullptr;
    uint64_t *tab2 = nullptr;
    int rc = SCI_OK;
    double *bnd_free = nullptr;   // the screening bounds, once allocated
    auto cleanup = [&]() {
        if (S) cudaFree(S);
        if (small) cudaFree(small);
        if (tab2) cudaFree(tab2);
        if (bnd_free) cudaFree(bnd_free);
    };
    const size_t nsmall = (size_t)R * 3 + (size_t)norb * norb + norb + 1 + 2;
    if (cudaMalloc(&S, sizeof(double) * SC * std::max<int64_t>(1, M) * R) != cudaSuccess ||
        cudaMalloc(&small, sizeof(double) * nsmall) != cudaSuccess) {
        cleanup();
        return sci_fail(ctx, SCI_ERR_NOMEM, "enpt2: scratch");
    }
    double *dE0 = small, *outW = small + R, *outP = small + 2 * R, *G = small + 3 * R, *fdiag = G + norb * norb,
           *Eref = fdiag + norb;
    unsigned long long *count = reinterpret_cast<unsigned long long *>(Eref + 1);
    int *flag = reinterpret_cast<int *>(count + 1);
    if (sci_cuda_check(ctx, cudaMemsetAsync(small, 0, sizeof(double) * nsmall, st), "enpt2 memset") ||
        sci_cuda_check(ctx, cudaMemcpyAsync(dE0, E0h, sizeof(double) * R, cudaMemcpyHostToDevice, st), "enpt2 E0")) {
        cleanup();
        return SCI_ERR_CUDA;
    }
    // E2[P]: one FP64 sigma
    if (M > 0) {
        rc = sci_launch_sigma(ctx, C, S, R, SCI_PREC_F64, true);   // every row, whatever the row range
        if (rc) {
            cleanup();
            return rc;
        }
        if constexpr (SPIN)
            k_pt2_p<R, zdbl><<<grid_for(M), kThreads, 0, st>>>(M, reinterpret_cast<const zdbl *>(C),
                                                               reinterpret_cast<const zdbl *>(S), ctx->hdiag, dE0, outP);
        else
            k_pt2_p<R, double><<<grid_for(M), kThreads, 0, st>>>(M, C, S, ctx->hdiag, dE0, outP);
    }
    if constexpr (SPIN)
        k_pt2_setup<zdbl><<<1, 256, 0, st>>>(norb, ctx->ref, ctx->ref_hi, ctx->ref_w2, (const zdbl *)ctx->h_so,
                                             (const zdbl *)ctx->jd, (const zdbl *)ctx->kd, G, fdiag, Eref);
    else
        k_pt2_setup<double><<<1, 256, 0, st>>>(norb, ctx->ref, ctx->ref_hi, ctx->ref_w2, (const double *)ctx->h_so,
                                               (const double *)ctx->jd, (const double *)ctx->kd, G, fdiag, Eref);
    // the table: capacity a power of two within the budget
    const size_t slot = sizeof(uint64_t) * SW;
    uint64_t cap = 1ull << 8;  // at least 256 entries
    while ((cap << 1) * slot <= table_bytes) cap <<= 1;
    if (cudaMalloc(&tab2, cap * slot) != cudaSuccess) {
        cleanup();
        return sci_fail(ctx, SCI_ERR_NOMEM, "enpt2: hash table");
    }
    // batches: the generated excitations (an upper bound on the distinct determinants)
    // split so that one batch fills at most 60% of the table
    int64_t per;  // excitations generated per determinant
    if constexpr (SPIN) {
        const int64_t N = na, u = n - na;
        per = N * u + N * (N - 1) / 2 * (u * (u - 1) / 2);
    } else {
        const int64_t ua = n - na, ub = n - nb;
        per = na * ua + nb * ub + (int64_t)na * (na - 1) / 2 * (ua * (ua - 1) / 2) +
              (int64_t)nb * (nb - 1) / 2 * (ub * (ub - 1) / 2) + (int64_t)na * ua * nb * ub;
    }
    const double total = (double)M * (double)per;
    // (at most 1024 batches: when even that bound does not fit, the distinct count decides,
    // and a batch that overflows the table ends with SCI_ERR_OVERFLOW)
    int tbits = 0;
    while (tbits < kMaxBits && total / (double)(1ull << tbits) > 0.6 * (double)cap) tbits++;
    Pt2 p{};
    // screening bounds of the double-excitation classes (eps > 0 only)
    double *bnd = nullptr;
    if (eps > 0.0) {
        const int64_t NP = (int64_t)n * (n - 1) / 2, nb3 = NP * n, nb2 = NP, nab = SPIN ? 0 : (int64_t)n * n;
        if (cudaMalloc(&bnd, sizeof(double) * std::max<int64_t>(1, nb3 + nb2 + nab)) != cudaSuccess) {
            cleanup();
            return sci_fail(ctx, SCI_ERR_NOMEM, "enpt2: screening bounds");
        }
        bnd_free = bnd;
        double *b3 = bnd, *b2 = bnd + nb3, *bab = b2 + nb2;
        if constexpr (SPIN) {
            k_pt2_bounds3<zdbl><<<grid_for(nb3), kThreads, 0, st>>>(n, (const zdbl *)ctx->tab, b3);
        } else {
            const double *T = (const double *)ctx->tab;
            k_pt2_bounds3<double><<<grid_for(nb3), kThreads, 0, st>>>(n, T + (int64_t)n * n * n * n, b3);
            k_pt2_bounds_pair<<<grid_for(nb2), kThreads, 0, st>>>(n, b3, b2);
            k_pt2_bounds_ab<<<grid_for(nab), kThreads, 0, st>>>(n, T, bab);
            p.bss = b2, p.bab = bab;
        }
        p.bss3 = b3;
    }
    p.n = n, p.norb = norb, p.na = na, p.nb = nb, p.ref = ctx->ref, p.ref_hi = ctx->ref_hi, p.ref_w2 = ctx->ref_w2;
    p.tab = (const double *)ctx->tab, p.fref = (const double *)ctx->fref, p.g_so = (const double *)ctx->g_so;
    p.fdiag = fdiag, p.G = G, p.Eref = Eref;
    p.tab2 = tab2, p.mask = cap - 1, p.count = count, p.flag = flag;
    p.limit = (unsigned long long)(0.85 * (double)cap);
    p.eps = eps;
    int64_t passes = 0, distinct = 0, sample = -1;
    float t_clear = 0.f, t_gen = 0.f, t_eval = 0.f;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cleanup();
            return sci_fail(ctx, SCI_ERR_CUDA, "enpt2: events");
        }
    auto done = [&](int code) {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        cleanup();
        return code;
    };
    // the batch code: t random bits per beta orbital (spinor mode: per spinor), and the
    // orbitals grouped by code
    auto set_codes = [&](int t) {
        std::mt19937 rng(20250130u + (unsigned)t);
        for (int o = 0; o < 192; o++) p.gcode[o] = t ? (uint32_t)(rng() & ((1u << t) - 1)) : 0u;
        std::vector<int> cnt((1 << t) + 1, 0);
        for (int o = 0; o < n; o++) cnt[p.gcode[o] + 1]++;
        for (int c = 1; c <= (1 << t); c++) cnt[c] += cnt[c - 1];
        for (int c = 0; c <= (1 << t); c++) p.cstart[c] = (uint8_t)cnt[c];
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int o = 0; o < n; o++) p.obc[fill[p.gcode[o]]++] = (uint8_t)o;
    };
    // the evaluation kernel's F and G (paired floats) in dynamic shared memory; past 165
    // orbitals (three-word keys only) G is read from global memory
    size_t eval_smem = sizeof(float2) * ((size_t)norb * norb + norb);
    const bool eval_gs = KW < 3 || eval_smem <= 216 * 1024;
    auto keval = k_pt2_eval<R, SPIN, KW, true>;
    if constexpr (KW == 3)
        if (!eval_gs) keval = k_pt2_eval<R, SPIN, KW, false>, eval_smem = sizeof(float2) * norb;
    if (sci_cuda_check(ctx, cudaFuncSetAttribute(keval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eval_smem),
                       "enpt2 eval attr"))
        return done(SCI_ERR_CUDA);
    // one batch: clear the table, generate, evaluate (optional); returns the distinct
    // count and the overflow flag
    auto pass = [&](uint32_t b, int t, bool eval, int64_t &cnt_out, int &flag_out) -> int {
        if (sci_cuda_check(ctx, cudaEventRecord(ev[0], st), "enpt2 event") ||
            sci_cuda_check(ctx, cudaMemsetAsync(tab2, 0, cap * slot, st), "enpt2 table") ||
            sci_cuda_check(ctx, cudaMemsetAsync(count, 0, sizeof(unsigned long long) + sizeof(int) * 2, st), "enpt2 count") ||
            sci_cuda_check(ctx, cudaEventRecord(ev[1], st), "enpt2 event"))
            return SCI_ERR_CUDA;
        if (M > 0) {
            const unsigned blocks = (unsigned)std::min<int64_t>((M + kWarps - 1) / kWarps, 152 * 16);
            if constexpr (SPIN)
                k_pt2_gen_z<R, KW><<<blocks, kThreads, 0, st>>>(ctx->keys, M, reinterpret_cast<const zdbl *>(C), p, b,
                                                               t);
            else
                k_pt2_gen<R, KW><<<blocks, kThreads, 0, st>>>(ctx->keys, M, C, p, b, t);
        }
        if (sci_cuda_check(ctx, cudaEventRecord(ev[2], st), "enpt2 event")) return SCI_ERR_CUDA;
        if (eval)
            keval<<<grid_for((int64_t)std::min<uint64_t>(cap, 1ull << 40)), kThreads, eval_smem, st>>>(p, cap, dE0, outW);
        unsigned long long hc[2] = {0, 0};
        if (sci_cuda_check(ctx, cudaEventRecord(ev[3], st), "enpt2 event") ||
            sci_cuda_check(ctx, cudaMemcpyAsync(hc, count, sizeof(hc), cudaMemcpyDeviceToHost, st), "enpt2 flag") ||
            sci_cuda_check(ctx, cudaStreamSynchronize(st), "enpt2 pass"))
            return SCI_ERR_CUDA;
        float a = 0.f, g = 0.f, e = 0.f;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&g, ev[1], ev[2]);
        cudaEventElapsedTime(&e, ev[2], ev[3]);
        t_clear += a, t_gen += g, t_eval += e;
        cnt_out = (int64_t)hc[0];
        // bit 1: the distinct count reached the load limit; bit 2: a probe limit was hit
        flag_out = (int)(hc[1] & 0xFFFFFFFFull) | (hc[0] >= p.limit ? 1 : 0);
        return SCI_OK;
    };
    // sampling: one batch of a four-times finer split estimates the distinct determinants
    // of W (duplicates make them far fewer than the generated excitations); the batch
    // count is chosen from that estimate with a 25% margin, never above the upper bound
    if (tbits > 0 && M > 0) {
        const int ts = std::min(kMaxBits, tbits + 2);
        set_codes(ts);
        int64_t c0 = 0;
        int f0 = 0;
        if (int rc2 = pass(0, ts, false, c0, f0)) return done(rc2);
        if (f0 == 0) {
            sample = c0;
            const double D = 1.25 * (double)c0 * (double)(1ull << ts);
            int t = 0;
            while (t < tbits && D / (double)(1ull << t) > 0.6 * (double)cap) t++;
            tbits = t;
        }
    }
    for (;;) {
        set_codes(tbits);
        bool overflow = false;
        distinct = 0;
        if (sci_cuda_check(ctx, cudaMemsetAsync(outW, 0, sizeof(double) * R, st), "enpt2 memset")) return done(SCI_ERR_CUDA);
        for (uint32_t b = 0; b < (1u << tbits) && !overflow; b++) {
            int64_t c = 0;
            int f = 0;
            if (int rc2 = pass(b, tbits, true, c, f)) return done(rc2);
            distinct += c;
            passes++;
            overflow = f != 0;
        }
        if (!overflow) break;
        if (++tbits > kMaxBits) return done(sci_fail(ctx, SCI_ERR_OVERFLOW, "enpt2: a batch overflowed the hash table at 1024 batches"));
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    double hw[R], hp[R];
    if (sci_cuda_check(ctx, cudaMemcpyAsync(hw, outW, sizeof(hw), cudaMemcpyDeviceToHost, st), "enpt2 W") ||
        sci_cuda_check(ctx, cudaMemcpyAsync(hp, outP, sizeof(hp), cudaMemcpyDeviceToHost, st), "enpt2 P") ||
        sci_cuda_check(ctx, cudaStreamSynchronize(st), "enpt2 result")) {
        cleanup();
        return SCI_ERR_CUDA;
    }
    for (int v = 0; v < R; v++) E2[v] = hw[v], E2[R + v] = hp[v], E2[2 * R + v] = hw[v] - hp[v];
    if (stats) {
        stats[0] = 1ll << tbits;
        stats[1] = distinct;
        stats[2] = passes;
        stats[3] = (int64_t)cap;
        stats[4] = (int64_t)(1e3f * t_clear);
        stats[5] = (int64_t)(1e3f * t_gen);
        stats[6] = (int64_t)(1e3f * t_eval);
        stats[7] = sample;
    }
    cleanup();
    return SCI_OK;
}

template <int KW>
int enpt2_dispatch(sci_ctx *ctx, const double *C, int nroots, const double *E0, double eps, size_t table_bytes,
                   double *E2, int64_t *stats)
{
    if (ctx->spinors) {
        switch (nroots) {
            case 1: return pt2_run<1, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
            case 2: return pt2_run<2, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
            case 3: return pt2_run<3, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
            case 4: return pt2_run<4, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
            case 5: return pt2_run<5, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
            case 6: return pt2_run<6, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
            case 7: return pt2_run<7, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
            default: return pt2_run<8, true, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        }
    }
    switch (nroots) {
        case 1: return pt2_run<1, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        case 2: return pt2_run<2, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        case 3: return pt2_run<3, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        case 4: return pt2_run<4, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        case 5: return pt2_run<5, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        case 6: return pt2_run<6, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        case 7: return pt2_run<7, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
        default: return pt2_run<8, false, KW>(ctx, C, E0, eps, table_bytes, E2, stats);
    }
}

}  // namespace

extern "C" int sci_enpt2(sci_ctx *ctx, const double *C, int nroots, const double *E0, double eps, size_t table_bytes,
                         double *E2, int64_t *stats)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_ints || !ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "enpt2: integrals and determinants first");
    if (ctx->spinors != ctx->cplx)
        return sci_fail(ctx, SCI_ERR_ARG, "enpt2: real spin-orbital mode or complex spinor mode");
    if (ctx->nwords > 3 || ctx->norb > 64 * ctx->nwords)
        return sci_fail(ctx, SCI_ERR_ARG, "enpt2: at most three key words (192 spin-orbitals or spinors)");
    if (ctx->nwords == 3 && ctx->norb == 192 && ctx->na + (ctx->spinors ? 0 : ctx->nb) >= 64)
        return sci_fail(ctx, SCI_ERR_ARG, "enpt2: 64 or more electrons in 192 spin-orbitals or spinors");
    if (nroots < 1 || nroots > 8 || !E0 || !E2 || (ctx->M > 0 && !C))
        return sci_fail(ctx, SCI_ERR_ARG, "enpt2: need 1 <= nroots <= 8, C, E0 and E2");
    if (eps < 0.0) return sci_fail(ctx, SCI_ERR_ARG, "enpt2: eps < 0");
    if (sci_cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) return SCI_ERR_CUDA;
    return ctx->nwords == 3   ? enpt2_dispatch<3>(ctx, C, nroots, E0, eps, table_bytes, E2, stats)
           : ctx->nwords == 2 ? enpt2_dispatch<2>(ctx, C, nroots, E0, eps, table_bytes, E2, stats)
                              : enpt2_dispatch<1>(ctx, C, nroots, E0, eps, table_bytes, E2, stats);
}
