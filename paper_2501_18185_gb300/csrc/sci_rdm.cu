// Reduced density matrices (Sec. 3.4) by the same bucket walks as sigma.
//
//   g1[p][q]       = sum_k w_k <c_k| a+_p a_q |c_k>
//   g2[p][q][r][s] = sum_k w_k <c_k| a+_p a+_r a_s a_q |c_k>
// over spin-orbitals (bit order of the keys) or spinors, unnormalised, so that for a
// normalised c the energy of Eq. Hamiltonian is sum h g1 + 1/2 sum (pq|rs) g2.
//
// The connections are recomputed from the setup tables, never stored.  The pairs of the
// three Slater-Condon classes (Sec. 2.3: zero, one and two differences) touch disjoint
// sets of g2 elements, so each class is accumulated into its own compact table and
// expanded once at the end:
//   diagonal (I = J): g1[p][p] and g2[p][p][r][r] = -g2[p][r][r][p] = sum_I w_I n_p n_r.
//     With n(I) = n(ref) + Delta(I) (Delta nonzero on the <= 2 x level orbitals where I
//     and the reference differ) the pair occupation is
//       O[p][r] = Wt n_p n_r + n_p D_r + D_p n_r + DD[p][r],
//     Wt = sum w_I, D = sum w_I Delta(I), DD = sum w_I Delta Delta^T,
//     accumulated per CTA in shared memory.
//   singles (members X = S + x, Y = S + y of one (N-1) bucket): w = conj(c_X) c_Y ph,
//     g1[x][y] += w, and for every spectator k in S
//       g2[x][y][k][k] = g2[k][k][x][y] = -g2[x][k][k][y] = -g2[k][y][x][k] += w.
//     The spectator sum b[x][y][k] = sum w n_k(S) is kept as A[x][y] n_k(ref) + Bc[x][y][k]
//     with Bc taking only the orbitals of S that differ from the reference (the same
//     reference decomposition as the sigma singles).
//   doubles (members I = K + {a,b}, J = K + {i,j} of one (N-2) bucket, disjoint): one
//     atomic add of w = conj(c_I) c_J ph into a table laid out like the pair-integral
//     table (with separate alpha-alpha and beta-beta regions), for the pairs with the
//     bra before the ket in the bucket; the other orientation is its conjugate.  Then
//       g2[a][i][b][j] = g2[b][j][a][i] = -g2[a][j][b][i] = -g2[b][i][a][j]
//         = dT[bra, ket] + conj(dT[ket, bra]).
// Signs: <I| a+_a a+_b a_j a_i |J> is the phase (-1)^(pi_I + pi_J) of the sigma kernels.
#include <algorithm>
#include <vector>

#include "sci_bits.cuh"
#include "sci_bucket.cuh"
#include "sci_internal.cuh"

using sci::zdbl;

namespace {

constexpr int kThreads = 256;
constexpr int kMaxVec = 8;  // vectors per walk; wider blocks take several walks

using sci::sflip;
__device__ __forceinline__ double conjv(double a) { return a; }
__device__ __forceinline__ zdbl conjv(zdbl a) { return zdbl{a.x, -a.y}; }
__device__ __forceinline__ double sqnorm(double a) { return a * a; }
__device__ __forceinline__ double sqnorm(zdbl a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double scale(double a, double s) { return a * s; }
__device__ __forceinline__ zdbl scale(zdbl a, double s) { return zdbl{a.x * s, a.y * s}; }
__device__ __forceinline__ void zero(double &a) { a = 0.0; }
__device__ __forceinline__ void zero(zdbl &a) { a = zdbl{0.0, 0.0}; }
// a += x * y
__device__ __forceinline__ void mac(double &a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void mac(zdbl &a, zdbl x, zdbl y)
{
    a.x = fma(x.x, y.x, fma(-x.y, y.y, a.x));
    a.y = fma(x.x, y.y, fma(x.y, y.x, a.y));
}
__device__ __forceinline__ void red(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void red(zdbl *p, zdbl v)
{
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ zdbl neg(zdbl a) { return zdbl{-a.x, -a.y}; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
template <typename TC> __device__ __forceinline__ TC from_real(double v);
template <> __device__ __forceinline__ double from_real<double>(double v) { return v; }
template <> __device__ __forceinline__ zdbl from_real<zdbl>(double v) { return zdbl{v, 0.0}; }
__device__ __forceinline__ zdbl add(zdbl a, zdbl b) { return zdbl{a.x + b.x, a.y + b.y}; }

// gradient-table offsets: the pair-table offsets, with beta-beta pairs moved to a region
// of their own after the alpha-alpha one (real spin-orbital mode)
__device__ __forceinline__ void grad_offsets(sci::TabRule tr, int x, int y, uint32_t bb_off, uint32_t &rowoff,
                                             uint32_t &colbase)
{
    sci::pair_offsets(tr, x, y, rowoff, colbase);
    if (!tr.spinors && x >= tr.n) colbase += bb_off;
}

// ------------------------------------------------------------------ diagonal
// occupation strings of KW 64-bit words: word w holds orbitals 64 w .. 64 w + 63
template <int KW> struct Str {
    uint64_t w[KW];
};
template <int KW> __device__ __forceinline__ Str<KW> load_str(const uint64_t *keys, int64_t I)
{
    Str<KW> s;
#pragma unroll
    for (int k = 0; k < KW; k++) s.w[k] = keys[I * KW + k];
    return s;
}
template <int KW> __device__ __forceinline__ bool occ(const Str<KW> &s, int p)
{
    return (s.w[p >> 6] >> (p & 63)) & 1;
}
using sci::RefW;   // the reference string over all words

// Diagonal class: O[p][r] = sum_I w_I n_p n_r in the reference decomposition n = n_ref + d
// (d = key ^ ref has a few bits), accumulated per CTA in shared memory ([norb]^2 doubles,
// dynamic: up to 226 KB, 168 spin-orbitals) when SM, else straight into DD and D in
// global memory (more orbitals).
template <typename TC, int KW, bool SM = true>
__global__ void __launch_bounds__(kThreads)
k_rdm_diag(const uint64_t *__restrict__ keys, int64_t M, int norb, RefW ref,
           const TC *__restrict__ C, int nvec, int v0, int nv, const double *__restrict__ wk, double *__restrict__ Wt,
           double *__restrict__ D, double *__restrict__ DD)
{
    extern __shared__ double s_dyn[];
    __shared__ double s_wsum[kThreads / 32];
    double *sDD = SM ? s_dyn : DD, *sD = SM ? s_dyn + norb * norb : D, *sW = s_wsum;
    if constexpr (SM) {
        for (int i = threadIdx.x; i < norb * norb; i += blockDim.x) sDD[i] = 0.0;
        for (int i = threadIdx.x; i < norb; i += blockDim.x) sD[i] = 0.0;
        __syncthreads();
    }
    Str<KW> rs;
#pragma unroll
    for (int k = 0; k < KW; k++) rs.w[k] = ref.w[k];
    double wsum = 0.0;
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < M; I += (int64_t)gridDim.x * blockDim.x) {
        double w = 0.0;
        for (int v = 0; v < nv; v++) w = fma(wk[v0 + v], sqnorm(C[I * nvec + v0 + v]), w);
        wsum += w;
        const Str<KW> key = load_str<KW>(keys, I);
#pragma unroll
        for (int k1 = 0; k1 < KW; k1++)
            for (uint64_t m = key.w[k1] ^ rs.w[k1]; m; m &= m - 1) {
                const int p = 64 * k1 + __ffsll((long long)m) - 1;
                const double wp = occ(key, p) ? w : -w;
                atomicAdd(&sD[p], wp);
#pragma unroll
                for (int k2 = 0; k2 < KW; k2++)
                    for (uint64_t m2 = key.w[k2] ^ rs.w[k2]; m2; m2 &= m2 - 1) {
                        const int r = 64 * k2 + __ffsll((long long)m2) - 1;
                        atomicAdd(&sDD[p * norb + r], occ(key, r) ? wp : -wp);
                    }
            }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
    if ((threadIdx.x & 31) == 0) sW[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kThreads / 32; i++) t += sW[i];
        atomicAdd(Wt, t);
    }
    if constexpr (SM) {
        for (int i = threadIdx.x; i < norb * norb; i += blockDim.x)
            if (sDD[i] != 0.0) atomicAdd(DD + i, sDD[i]);
        for (int i = threadIdx.x; i < norb; i += blockDim.x)
            if (sD[i] != 0.0) atomicAdd(D + i, sD[i]);
    }
}

// ------------------------------------------------------------------ singles
template <typename TC, int NV, int KW>
__global__ void __launch_bounds__(kThreads)
k_rdm_singles(const uint32_t *__restrict__ e_idx, const uint64_t *__restrict__ e_S, const uint32_t *__restrict__ e_meta,
              int64_t E, int norb, RefW ref, const TC *__restrict__ C, int nvec, int v0,
              const double *__restrict__ wk, TC *__restrict__ A, TC *__restrict__ Bc)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t meta = e_meta[p];
        const int x = sci::meta_x(meta);
        const bool par = sci::meta_par(meta);
        const int64_t bs = p - (int64_t)sci::meta_off(meta);
        const int64_t be = bs + (int64_t)sci::meta_size(meta);
        // the spectator string's orbitals outside (part) and missing from (holes) the
        // reference, per word
        uint64_t part[KW], holes[KW];
#pragma unroll
        for (int k = 0; k < KW; k++) {
            const uint64_t Sk = e_S[p * KW + k], rk = ref.w[k];
            part[k] = Sk & ~rk, holes[k] = rk & ~Sk;
        }
        const int64_t idx = e_idx[p];
        TC rowc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) rowc[v] = scale(conjv(sflip(par, C[idx * nvec + v0 + v])), wk[v0 + v]);
        for (int64_t q = bs; q < be; q++) {
            if (q == p) continue;
            const uint32_t mq = e_meta[q];
            const int y = sci::meta_x(mq);
            const bool parq = sci::meta_par(mq);
            const int64_t idxq = e_idx[q];
            TC w;
            zero(w);
#pragma unroll
            for (int v = 0; v < NV; v++) mac(w, rowc[v], sflip(parq, C[idxq * nvec + v0 + v]));
            const int64_t xy = (int64_t)x * norb + y;
            red(A + xy, w);
            const TC nw = neg(w);
#pragma unroll
            for (int k = 0; k < KW; k++) {
                for (uint64_t m = part[k]; m; m &= m - 1) red(Bc + xy * norb + 64 * k + (__ffsll((long long)m) - 1), w);
                for (uint64_t m = holes[k]; m; m &= m - 1) red(Bc + xy * norb + 64 * k + (__ffsll((long long)m) - 1), nw);
            }
        }
    }
}

// ------------------------------------------------------------------ doubles
// Each unordered pair of a bucket of size s is walked once, with balanced work per lane:
// the member at position q takes the members at q + d (mod s) for d = 1 .. (s-1)/2, and
// for even s the member at distance s/2 is taken by the first half of the bucket.  The
// orientation of a pair does not matter: the expansion adds both orientations.
template <typename TC, int NV>
__global__ void __launch_bounds__(kThreads)
k_rdm_doubles(const uint32_t *__restrict__ e_idx, const uint32_t *__restrict__ e_code, const uint32_t *__restrict__ e_pos,
              int64_t E, int CH, sci::TabRule tr, uint32_t bb_off, const TC *__restrict__ C, int nvec, int v0,
              const double *__restrict__ wk, TC *__restrict__ dT)
{
    constexpr int nv = NV;
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t r0, r1;
    sci::window(e_pos, E, CH, r0, r1);
    if (r0 >= r1) return;
    const int W = (int)(r1 - r0);
    TC *s_c = reinterpret_cast<TC *>(smem);  // [W][nv]: c of each member times (-1)^pi
    const size_t cbytes = ((size_t)W * nv * sizeof(TC) + 15) & ~(size_t)15;
    uint2 *s_kc = reinterpret_cast<uint2 *>(smem + cbytes);
    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        const int64_t g = r0 + q;
        const uint32_t code = e_code[g];
        const int64_t idx = e_idx[g];
        uint32_t rowoff, colbase;
        grad_offsets(tr, sci::code_x(code), sci::code_y(code), bb_off, rowoff, colbase);
        s_kc[q] = make_uint2(sci::col_code(code), colbase);
        const bool par = sci::code_par(code);
        for (int v = 0; v < nv; v++) s_c[q * nv + v] = sflip(par, C[idx * nvec + v0 + v]);
    }
    __syncthreads();
    for (int q0 = threadIdx.x; q0 < W; q0 += blockDim.x) {
        const uint32_t code = e_code[r0 + q0], pos = e_pos[r0 + q0];
        uint32_t rowoff, colbase;
        grad_offsets(tr, sci::code_x(code), sci::code_y(code), bb_off, rowoff, colbase);
        const int qp = sci::pos_off(pos), sz = sci::pos_size(pos), bs = q0 - qp;
        const int dmax = (sz - 1) / 2 + ((sz & 1) == 0 && qp < sz / 2 ? 1 : 0);
        const uint32_t rc = sci::row_code(code);
        TC rowc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) rowc[v] = scale(conjv(s_c[q0 * nv + v]), wk[v0 + v]);
        TC *trow = dT + rowoff;
        int j = qp;
        for (int d = 1; d <= dmax; d++) {
            j = j + 1 == sz ? 0 : j + 1;
            const uint2 kc = s_kc[bs + j];
            if (!sci::disjoint(rc, kc.x)) continue;
            TC w;
            zero(w);
#pragma unroll
            for (int v = 0; v < NV; v++) mac(w, rowc[v], s_c[(bs + j) * nv + v]);
            red(trow + kc.y, w);
        }
    }
}

// ------------------------------------------------------------------ expansion
// g1 and the g2 elements of the diagonal and single-excitation classes; one thread per
// (x, y)
// occupation of orbital k in the reference
__device__ __forceinline__ double ref_occ(const RefW &ref, int k) { return (double)((ref.w[k >> 6] >> (k & 63)) & 1); }

template <typename TC>
__global__ void k_rdm_expand1(int norb, RefW ref, const double *__restrict__ Wt,
                              const double *__restrict__ D, const double *__restrict__ DD, const TC *__restrict__ A,
                              const TC *__restrict__ Bc, TC *__restrict__ g1, TC *__restrict__ g2)
{
    const int64_t n2 = (int64_t)norb * norb, n3 = n2 * norb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n2; t += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(t / norb), y = (int)(t % norb);
        const double nx = ref_occ(ref, x), ny = ref_occ(ref, y);
        const double O = *Wt * nx * ny + nx * D[y] + D[x] * ny + DD[t];
        const TC o = from_real<TC>(O);
        if (x == y) {
            g1[t] = o;
            continue;
        }
        const TC a = A[t];
        g1[t] = a;
        if (!g2) continue;
        g2[(int64_t)x * n3 + (int64_t)x * n2 + (int64_t)y * norb + y] = o;         // (x x | y y)
        g2[(int64_t)x * n3 + (int64_t)y * n2 + (int64_t)y * norb + x] = neg(o);    // (x y | y x)
        for (int k = 0; k < norb; k++) {
            if (k == x || k == y) continue;
            const TC b = add(scale(a, ref_occ(ref, k)), Bc[t * norb + k]);
            const TC nb = neg(b);
            g2[(int64_t)x * n3 + (int64_t)y * n2 + (int64_t)k * norb + k] = b;     // (x y | k k)
            g2[(int64_t)k * n3 + (int64_t)k * n2 + (int64_t)x * norb + y] = b;     // (k k | x y)
            g2[(int64_t)x * n3 + (int64_t)k * n2 + (int64_t)k * norb + y] = nb;    // (x k | k y)
            g2[(int64_t)k * n3 + (int64_t)y * n2 + (int64_t)x * norb + k] = nb;    // (k y | x k)
        }
    }
}

// unordered pair index P(a, b) = b(b-1)/2 + a, a < b -> (a, b)
__device__ __forceinline__ void unpair(int P, int &a, int &b)
{
    int bb = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)P)) * 0.5f);
    while (bb * (bb - 1) / 2 > P) bb--;
    while ((bb + 1) * bb / 2 <= P) bb++;
    b = bb;
    a = P - bb * (bb - 1) / 2;
}

// g2 elements of the double-excitation class from the gradient table; one thread per
// table entry (bra, ket), writing the four elements of that orientation
template <typename TC>
__global__ void k_rdm_expand2(sci::TabRule tr, int norb, int64_t nT, const TC *__restrict__ dT, TC *__restrict__ g2)
{
    const int n = tr.n;
    const int64_t n2 = (int64_t)norb * norb, n3 = n2 * norb;
    const int64_t NP = (int64_t)n * (n - 1) / 2;
    const int64_t nab = tr.spinors ? 0 : (int64_t)n * n * n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nT; e += (int64_t)gridDim.x * blockDim.x) {
        int a, b, i, j;
        int64_t et;
        if (e < nab) {  // alpha-beta: e = u_ket * n^2 + u_bra, u = (y - n) * n + x
            const int64_t ub = e % ((int64_t)n * n), uk = e / ((int64_t)n * n);
            a = (int)(ub % n), b = n + (int)(ub / n);
            i = (int)(uk % n), j = n + (int)(uk / n);
            et = ub * ((int64_t)n * n) + uk;
        } else {        // same spin (spinor mode: all): e = p_ket * NP + p_bra
            const int64_t e2 = e - nab;
            const int64_t reg = e2 / (NP * NP), r = e2 % (NP * NP);
            const int pb = (int)(r % NP), pk = (int)(r / NP);
            unpair(pb, a, b);
            unpair(pk, i, j);
            if (reg) a += n, b += n, i += n, j += n;  // beta-beta region
            et = nab + reg * (NP * NP) + (int64_t)pb * NP + pk;
        }
        if (a == i || a == j || b == i || b == j) continue;  // not a double: other classes own these
        const TC u = add(dT[e], conjv(dT[et]));
        const TC nu = neg(u);
        g2[(int64_t)a * n3 + (int64_t)i * n2 + (int64_t)b * norb + j] = u;
        g2[(int64_t)b * n3 + (int64_t)j * n2 + (int64_t)a * norb + i] = u;
        g2[(int64_t)a * n3 + (int64_t)j * n2 + (int64_t)b * norb + i] = nu;
        g2[(int64_t)b * n3 + (int64_t)i * n2 + (int64_t)a * norb + j] = nu;
    }
}

int grid_for(int64_t n)
{
    const int64_t b = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

template <typename TC> struct Walk {
    const TC *C;
    int nvec, v0;
    const double *wk;
    TC *A, *Bc, *dT;  // dT == nullptr: no double-excitation walk
    int CH;
    size_t smem;
    sci::TabRule tr;
    uint32_t bb_off;
};

// the single- and double-excitation walks for one group of NV vectors
template <typename TC, int NV>
int launch_walks(sci_ctx *ctx, const Walk<TC> &w)
{
    if (ctx->e1 > 0) {
        auto ks = ctx->nwords == 4   ? k_rdm_singles<TC, NV, 4>
                  : ctx->nwords == 3 ? k_rdm_singles<TC, NV, 3>
                  : ctx->nwords == 2 ? k_rdm_singles<TC, NV, 2>
                                     : k_rdm_singles<TC, NV, 1>;
        ks<<<grid_for(ctx->e1), kThreads, 0, ctx->stream>>>(ctx->e1_idx, ctx->e1_S, ctx->e1_meta, ctx->e1, ctx->norb,
                                                            ref_words(ctx), w.C, w.nvec, w.v0, w.wk, w.A, w.Bc);
    }
    if (w.dT) {
        auto kern = k_rdm_doubles<TC, NV>;
        if (w.smem > 48 * 1024 &&
            sci_cuda_check(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w.smem),
                           "rdm12 attr"))
            return SCI_ERR_CUDA;
        const int64_t blocks = (ctx->e2 + w.CH - 1) / w.CH;
        kern<<<(unsigned)blocks, kThreads, w.smem, ctx->stream>>>(ctx->e2_idx, ctx->e2_code, ctx->e2_pos, ctx->e2, w.CH,
                                                                 w.tr, w.bb_off, w.C, w.nvec, w.v0, w.wk, w.dT);
    }
    return SCI_OK;
}

template <typename TC>
int rdm_run(sci_ctx *ctx, const TC *C, int nvec, const double *wk_dev, TC *g1, TC *g2)
{
    const int norb = ctx->norb, n = ctx->n;
    const int64_t n2 = (int64_t)norb * norb;
    const int64_t NP = (int64_t)n * (n - 1) / 2;
    const int64_t nT = ctx->spinors ? NP * NP : (int64_t)n * n * n * n + 2 * NP * NP;
    const uint32_t bb_off = ctx->spinors ? 0u : (uint32_t)(NP * NP);
    // scratch: Wt, D[norb], DD[norb^2] (double); A[norb^2], Bc[norb^3], dT[nT] (TC)
    const size_t dbytes = sizeof(double) * (1 + norb + n2);
    const size_t tbytes = sizeof(TC) * (n2 + n2 * norb + (g2 ? nT : 0));
    const size_t need = ((dbytes + 255) & ~(size_t)255) + tbytes;
    if (need > ctx->rdm_bytes) {
        if (ctx->rdm_scratch) cudaFree(ctx->rdm_scratch);
        ctx->rdm_scratch = nullptr, ctx->rdm_bytes = 0;
        if (cudaMalloc(&ctx->rdm_scratch, need) != cudaSuccess) return sci_fail(ctx, SCI_ERR_NOMEM, "rdm12: scratch");
        ctx->rdm_bytes = need;
    }
    unsigned char *base = static_cast<unsigned char *>(ctx->rdm_scratch);
    double *Wt = reinterpret_cast<double *>(base), *D = Wt + 1, *DD = D + norb;
    TC *A = reinterpret_cast<TC *>(base + ((dbytes + 255) & ~(size_t)255));
    TC *Bc = A + n2;
    TC *dT = Bc + n2 * norb;
    if (sci_cuda_check(ctx, cudaMemsetAsync(ctx->rdm_scratch, 0, need, ctx->stream), "rdm12 memset") ||
        (g2 && sci_cuda_check(ctx, cudaMemsetAsync(g2, 0, sizeof(TC) * n2 * n2, ctx->stream), "rdm12 memset g2")))
        return SCI_ERR_CUDA;
    const sci::TabRule tr{ctx->spinors, n};
    const int CH = 768;
    auto stage_bytes = [&](int nv) {
        return (((size_t)(CH + ctx->maxb2) * nv * sizeof(TC) + 15) & ~(size_t)15) + (size_t)(CH + ctx->maxb2) * sizeof(uint2);
    };
    // vectors per walk: at most kMaxVec, fewer when the staged window would not fit
    int kv = kMaxVec;
    while (kv > 1 && stage_bytes(kv) > 200 * 1024) kv >>= 1;
    if (g2 && ctx->e2 > 0 && stage_bytes(kv) > 200 * 1024)
        return sci_fail(ctx, SCI_ERR_OVERFLOW, "rdm12: largest bucket too large for shared memory");
    // the diagonal kernel: DD [norb]^2 and D [norb] in shared memory while they fit (up to
    // 168 orbitals), else accumulated in global memory
    size_t diag_smem = sizeof(double) * ((size_t)norb * norb + norb);
    const bool diag_sm = diag_smem + 1024 <= 227 * 1024;
    auto kd = ctx->nwords == 4   ? (diag_sm ? k_rdm_diag<TC, 4, true> : k_rdm_diag<TC, 4, false>)
              : ctx->nwords == 3 ? (diag_sm ? k_rdm_diag<TC, 3, true> : k_rdm_diag<TC, 3, false>)
              : ctx->nwords == 2 ? k_rdm_diag<TC, 2, true>
                                 : k_rdm_diag<TC, 1, true>;
    if (!diag_sm) diag_smem = 0;
    if (diag_sm && sci_cuda_check(ctx, cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                            (int)diag_smem), "rdm12 diag attr"))
        return SCI_ERR_CUDA;
    for (int v0 = 0; v0 < nvec; v0 += kv) {
        const int nv = std::min(kv, nvec - v0);
        kd<<<grid_for(ctx->M), kThreads, diag_smem, ctx->stream>>>(ctx->keys, ctx->M, norb, ref_words(ctx), C, nvec, v0,
                                                                   nv, wk_dev, Wt, D, DD);
        const Walk<TC> wlk{C, nvec, v0, wk_dev, A, Bc, g2 && ctx->e2 > 0 ? dT : nullptr, CH, stage_bytes(nv), tr, bb_off};
        int rc = SCI_OK;
        switch (nv) {
            case 1: rc = launch_walks<TC, 1>(ctx, wlk); break;
            case 2: rc = launch_walks<TC, 2>(ctx, wlk); break;
            case 3: rc = launch_walks<TC, 3>(ctx, wlk); break;
            case 4: rc = launch_walks<TC, 4>(ctx, wlk); break;
            case 5: rc = launch_walks<TC, 5>(ctx, wlk); break;
            case 6: rc = launch_walks<TC, 6>(ctx, wlk); break;
            case 7: rc = launch_walks<TC, 7>(ctx, wlk); break;
            default: rc = launch_walks<TC, 8>(ctx, wlk); break;
        }
        if (rc) return rc;
    }
    k_rdm_expand1<TC><<<grid_for(n2), kThreads, 0, ctx->stream>>>(norb, ref_words(ctx), Wt, D, DD, A, Bc, g1, g2);
    if (g2) k_rdm_expand2<TC><<<grid_for(nT), kThreads, 0, ctx->stream>>>(tr, norb, nT, dT, g2);
    return sci_cuda_check(ctx, cudaGetLastError(), "rdm12 launch") ? SCI_ERR_CUDA : SCI_OK;
}

// ------------------------------------------------------------------ gradients of E
// Spin sums of the spin-orbital density matrices (bit p < n alpha p, bit n + p beta p):
//   gamma[p][q]        = sum_s g1[ps][qs]
//   Gamma[p][q][r][s]  = sum_{s1,s2} g2[p s1][q s1][r s2][s s2]
__global__ void k_spin_sum1(int n, const double *__restrict__ g1, double *__restrict__ gamma)
{
    const int norb = 2 * n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
        const int p = t / n, q = t % n;
        gamma[t] = g1[p * norb + q] + g1[(n + p) * norb + n + q];
    }
}

__global__ void k_spin_sum2(int n, const double *__restrict__ g2, double *__restrict__ Gamma)
{
    const int64_t norb = 2 * n, n4 = (int64_t)n * n * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t % n, r = (t / n) % n, q = (t / n / n) % n, p = t / n / n / n;
        double v = 0.0;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                v += g2[(((p + a * n) * norb + q + a * n) * norb + r + b * n) * norb + s + b * n];
        Gamma[t] = v;
    }
}

// gL[P][i] = sum_k Gamma[i][k] L[P][k] for i, k < n^2 (the chain rule of
// (pq|rs) = sum_P L^P_pq L^P_rs through the free entries of L^P, with Gamma symmetric in
// its two index pairs): a 64 x 32 output tile per CTA, k in steps of 16 staged in shared
// memory, 8 outputs per thread, FP64 FMA
constexpr int kGI = 64, kGP = 32, kGK = 16;
__global__ void __launch_bounds__(256) k_gamma_chol(int nn, int naux, const double *__restrict__ Gamma,
                                                     const double *__restrict__ L, double *__restrict__ gL)
{
    __shared__ double sG[kGK][kGI + 1];
    __shared__ double sL[kGK][kGP + 1];
    const int i0 = blockIdx.x * kGI, P0 = blockIdx.y * kGP;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // P = P0 + tx, i = i0 + ty + 8 u
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k0 = 0; k0 < nn; k0 += kGK) {
        for (int t = threadIdx.x; t < kGK * kGI; t += blockDim.x) {
            const int kk = t % kGK, ii = t / kGK;
            const int i = i0 + ii, k = k0 + kk;
            sG[kk][ii] = (i < nn && k < nn) ? Gamma[(int64_t)i * nn + k] : 0.0;
        }
        for (int t = threadIdx.x; t < kGK * kGP; t += blockDim.x) {
            const int kk = t % kGK, pp = t / kGK;
            const int P = P0 + pp, k = k0 + kk;
            sL[kk][pp] = (P < naux && k < nn) ? L[(int64_t)P * nn + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; kk++) {
            const double l = sL[kk][tx];
#pragma unroll
            for (int u = 0; u < 8; u++) acc[u] = fma(sG[kk][ty + 8 * u], l, acc[u]);
        }
        __syncthreads();
    }
    const int P = P0 + tx;
    if (P < naux)
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int i = i0 + ty + 8 * u;
            if (i < nn) gL[(int64_t)P * nn + i] = acc[u];
        }
}

}  // namespace

extern "C" int sci_rdm_grads(sci_ctx *ctx, const double *C, int nvec, const double *weights, double *gamma,
                             double *Gamma, int naux, const double *chol, double *gchol)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_ints || !ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "rdm_grads: integrals and determinants first");
    if (ctx->cplx || ctx->spinors) return sci_fail(ctx, SCI_ERR_ARG, "rdm_grads: real spin-orbital mode only");
    if (nvec < 1 || (ctx->M > 0 && !C)) return sci_fail(ctx, SCI_ERR_ARG, "rdm_grads: need nvec >= 1 and C");
    if ((chol == nullptr) != (gchol == nullptr) || (chol && naux < 1))
        return sci_fail(ctx, SCI_ERR_ARG, "rdm_grads: chol and gchol go together, naux >= 1");
    if (sci_cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) return SCI_ERR_CUDA;
    const int n = ctx->n, norb = ctx->norb;
    const int64_t nn = (int64_t)n * n, n4 = nn * nn, o2 = (int64_t)norb * norb, o4 = o2 * o2;
    const bool two = Gamma || chol;
    // spin-orbital g1, g2 and (when the caller passes no Gamma but needs the contraction)
    // the spin-summed Gamma, in a buffer of their own
    double *buf = nullptr;
    const size_t need = sizeof(double) * (o2 + (two ? o4 : 0) + (two && !Gamma ? n4 : 0));
    if (cudaMalloc(&buf, need) != cudaSuccess) return sci_fail(ctx, SCI_ERR_NOMEM, "rdm_grads: scratch");
    double *g1 = buf, *g2 = two ? buf + o2 : nullptr, *G = Gamma ? Gamma : (two ? buf + o2 + o4 : nullptr);
    int rc = sci_rdm12(ctx, C, nvec, weights, g1, g2);
    cudaStream_t st = ctx->stream;
    if (rc == SCI_OK && gamma) k_spin_sum1<<<grid_for(nn), kThreads, 0, st>>>(n, g1, gamma);
    if (rc == SCI_OK && two) k_spin_sum2<<<grid_for(n4), kThreads, 0, st>>>(n, g2, G);
    if (rc == SCI_OK && chol) {
        const dim3 grid((unsigned)((nn + kGI - 1) / kGI), (unsigned)((naux + kGP - 1) / kGP));
        k_gamma_chol<<<grid, 256, 0, st>>>((int)nn, naux, G, chol, gchol);
    }
    if (rc == SCI_OK) rc = sci_cuda_check(ctx, cudaGetLastError(), "rdm_grads launch");
    // the buffer is freed after the queued work has read it
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (rc == SCI_OK) rc = sci_cuda_check(ctx, e, "rdm_grads");
    return rc;
}

extern "C" int sci_rdm12(sci_ctx *ctx, const void *C, int nvec, const double *weights, void *rdm1, void *rdm2)
{
    if (!ctx) return SCI_ERR_ARG;
    if (!ctx->have_ints || !ctx->have_dets) return sci_fail(ctx, SCI_ERR_STATE, "rdm12: integrals and determinants first");
    if (nvec < 1 || !rdm1 || (ctx->M > 0 && !C)) return sci_fail(ctx, SCI_ERR_ARG, "rdm12: need nvec >= 1, C and rdm1");
    if (ctx->norb > 256 || ctx->nwords > sci::kMaxWords) return sci_fail(ctx, SCI_ERR_ARG, "rdm12: at most 256 orbitals");
    if (sci_cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) return SCI_ERR_CUDA;
    // weights to the device (a host array of nvec doubles, NULL = all ones)
    const size_t wbytes = sizeof(double) * nvec;
    if (wbytes > ctx->rdm_wbytes) {
        if (ctx->rdm_w) cudaFree(ctx->rdm_w);
        ctx->rdm_w = nullptr, ctx->rdm_wbytes = 0;
        if (cudaMalloc(&ctx->rdm_w, wbytes) != cudaSuccess) return sci_fail(ctx, SCI_ERR_NOMEM, "rdm12: weights");
        ctx->rdm_wbytes = wbytes;
    }
    std::vector<double> w(nvec, 1.0);
    if (weights) std::copy(weights, weights + nvec, w.begin());
    if (sci_cuda_check(ctx, cudaMemcpyAsync(ctx->rdm_w, w.data(), wbytes, cudaMemcpyHostToDevice, ctx->stream), "rdm12 weights") ||
        sci_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "rdm12 weights sync"))
        return SCI_ERR_CUDA;
    const double *wk = static_cast<const double *>(ctx->rdm_w);
    if (ctx->cplx)
        return rdm_run<zdbl>(ctx, static_cast<const zdbl *>(C), nvec, wk, static_cast<zdbl *>(rdm1), static_cast<zdbl *>(rdm2));
    return rdm_run<double>(ctx, static_cast<const double *>(C), nvec, wk, static_cast<double *>(rdm1), static_cast<double *>(rdm2));
}
