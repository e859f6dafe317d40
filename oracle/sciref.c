/*
 * sciref.c -- plain CPU oracle for sigma = H c over a sorted determinant list.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load this library.  It shares no code, header, table or helper with the
 * CUDA path; it is slow on purpose and written to be checked against the paper by eye.
 *
 * What it computes (paper, Sec. 2.1, Eq. Hamiltonian and Eq. sym_op):
 *   H = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs (pq|rs) a+_p a+_r a_s a_q      (Mulliken)
 *   sigma_I = sum_J <D_I|H|D_J> c_J                                          (Sec. 2.4,
 *             the diagonalisation paragraph: H is applied through matrix-vector
 *             products with elements recomputed when needed, never stored)
 *
 * Determinants and phases.  A determinant is a 64-bit occupation string; bit p is
 * spin-orbital (or spinor) p.  |D> = a+_{p1} a+_{p2} ... |0> with p1 < p2 < ... in bit
 * order.  Spin-orbital mode with n spatial orbitals: bit p < n is alpha orbital p, bit
 * n + p is beta orbital p, and the spatial integrals are expanded to spin-orbital ones
 * with (pq|rs) nonzero only for spin(p) = spin(q) and spin(r) = spin(s).
 *
 * Matrix elements (Slater-Condon rules, derived from the operator form above):
 *   diagonal:  H_II = sum_{i in occ} h_ii + 1/2 sum_{i,j in occ} [(ii|jj) - (ij|ji)]
 *   single I = a+_a a_i J:
 *              H_IJ = s [ h_ai + sum_{k in occ(J), k != i} ((ai|kk) - (ak|ki)) ]
 *   double I = a+_b a+_a a_i a_j J (i<j, a<b; a_j applied first):
 *              H_IJ = s [ (ai|bj) - (aj|bi) ]
 *   s is the sign picked up while applying the operators one at a time to the ket
 *   string: each a_p or a+_p passes over the occupied orbitals below p, counted with an
 *   explicit loop over bits.
 *
 * Connections of row I are found by generating every single and double excitation of
 * D_I (spin-orbital mode: only those conserving the numbers of alpha and beta
 * electrons) and looking each up in the sorted list (binary search).  An independent
 * all-pairs route (sciref_sigma_brute_rows) tests every J of the list instead.
 * Rows are independent and are run in parallel with OpenMP.
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SCIREF_OK 0
#define SCIREF_ERR_ARG (-1)
#define SCIREF_ERR_UNSORTED (-2)
#define SCIREF_ERR_CAP (-8)

typedef double complex zd;

/* An occupation string of up to 256 spin-orbitals or spinors: orbital p is bit p % 64 of
 * word p / 64 (determinants of up to 64 orbitals use word 0 only).  Strings compare as
 * unsigned 256-bit integers, word 3 most significant. */
#define SCIREF_WORDS 4
#define SCIREF_MAXORB (64 * SCIREF_WORDS)
typedef struct { uint64_t w[SCIREF_WORDS]; } bits_t;

typedef struct sciref_ctx {
    int is_complex;   /* 0: real FP64 scalars, 1: complex128 scalars */
    int spinors;      /* 0: spin-orbital mode, 1: spinor mode */
    int n;            /* spatial orbitals or spinors */
    int norb;         /* bits in use: 2n (spin-orbital) or n (spinor) */
    zd *h;            /* norb x norb */
    zd *eri;          /* norb^4, [p][q][r][s] = (pq|rs) */
    bits_t *keys;
    int64_t M;
} sciref_ctx;

static int spin_of(const sciref_ctx *c, int p) { return c->spinors ? 0 : (p >= c->n); }
static int spatial_of(const sciref_ctx *c, int p) { return c->spinors ? p : (p % c->n); }

static zd H1(const sciref_ctx *c, int p, int q) { return c->h[(size_t)p * c->norb + q]; }
/* (pq|rs) over spin-orbitals or spinors: in spin-orbital mode zero unless p, q share a spin
 * and r, s share a spin, else the spatial integral of their orbitals (Eq. Hamiltonian with
 * a spin-free two-electron operator); the n^4 input values are kept as given. */
static zd ERI(const sciref_ctx *c, int p, int q, int r, int s)
{
    if (spin_of(c, p) != spin_of(c, q) || spin_of(c, r) != spin_of(c, s)) return 0.0;
    const size_t n = (size_t)c->n;
    const size_t P = spatial_of(c, p), Q = spatial_of(c, q), R = spatial_of(c, r), S = spatial_of(c, s);
    return c->eri[((P * n + Q) * n + R) * n + S];
}

/* ------------------------------------------------------------------ creation */
/* h: n*n, eri: n^4 (row-major, [p][q][r][s] = (pq|rs)); complex data interleaved re,im.
 * Spin-orbital mode expands h to the 2n spin-orbitals; ERI() maps spin-orbital indices to
 * the n^4 values. */
int sciref_create(sciref_ctx **out, int is_complex, int spinors, int n,
                  const double *h, const double *eri)
{
    if (!out || !h || !eri || n <= 0) return SCIREF_ERR_ARG;
    if (spinors ? n > SCIREF_MAXORB : 2 * n > SCIREF_MAXORB) return SCIREF_ERR_ARG;
    sciref_ctx *c = (sciref_ctx *)calloc(1, sizeof(sciref_ctx));
    c->is_complex = is_complex;
    c->spinors = spinors;
    c->n = n;
    c->norb = spinors ? n : 2 * n;
    size_t m = (size_t)c->norb, n4 = (size_t)n * n * n * n;
    c->h = (zd *)calloc(m * m, sizeof(zd));
    c->eri = (zd *)calloc(n4, sizeof(zd));
    if (!c->h || !c->eri) { free(c->h); free(c->eri); free(c); return SCIREF_ERR_ARG; }
    for (int p = 0; p < c->norb; p++)
        for (int q = 0; q < c->norb; q++) {
            if (spin_of(c, p) != spin_of(c, q)) continue;
            size_t s = (size_t)spatial_of(c, p) * n + spatial_of(c, q);
            c->h[p * m + q] = is_complex ? CMPLX(h[2 * s], h[2 * s + 1]) : CMPLX(h[s], 0.0);
        }
    for (size_t t = 0; t < n4; t++) c->eri[t] = is_complex ? CMPLX(eri[2 * t], eri[2 * t + 1]) : CMPLX(eri[t], 0.0);
    *out = c;
    return SCIREF_OK;
}

void sciref_destroy(sciref_ctx *c)
{
    if (!c) return;
    free(c->h);
    free(c->eri);
    free(c->keys);
    free(c);
}

static int key_cmp(bits_t a, bits_t b);

/* keys: M strings of nwords (1 to 4) 64-bit words each, word 0 holding orbitals 0..63;
 * the list must be strictly ascending as unsigned (64 x nwords)-bit integers. */
int sciref_set_determinants_w(sciref_ctx *c, const uint64_t *keys, int nwords, int64_t M)
{
    if (!c || (M > 0 && !keys) || M < 0 || nwords < 1 || nwords > SCIREF_WORDS) return SCIREF_ERR_ARG;
    bits_t *k = (bits_t *)calloc((size_t)(M > 0 ? M : 1), sizeof(bits_t));
    for (int64_t i = 0; i < M; i++) {
        for (int t = 0; t < nwords; t++) k[i].w[t] = keys[i * nwords + t];
        if (i > 0 && key_cmp(k[i - 1], k[i]) >= 0) { free(k); return SCIREF_ERR_UNSORTED; }
    }
    free(c->keys);
    c->keys = k;
    c->M = M;
    return SCIREF_OK;
}

/* One-word strings: strictly ascending as unsigned 64-bit integers. */
int sciref_set_determinants(sciref_ctx *c, const uint64_t *keys, int64_t M)
{
    return sciref_set_determinants_w(c, keys, 1, M);
}

/* OpenMP threads of the parallel loops below (n <= 0 restores the default); returns the
 * number that later loops will use.  Timing only: the results do not depend on it. */
static int sciref_default_threads = 0;
int sciref_set_threads(int n)
{
    if (sciref_default_threads == 0) sciref_default_threads = omp_get_max_threads();
    omp_set_num_threads(n > 0 ? n : sciref_default_threads);
    return omp_get_max_threads();
}

/* ------------------------------------------------------------------ helpers */
static int occupied(bits_t d, int p) { return (int)((d.w[p >> 6] >> (p & 63)) & 1u); }
static bits_t with_bit(bits_t d, int p) { d.w[p >> 6] |= 1ull << (p & 63); return d; }
static bits_t without_bit(bits_t d, int p) { d.w[p >> 6] &= ~(1ull << (p & 63)); return d; }
/* -1, 0, +1 as unsigned 256-bit integers */
static int key_cmp(bits_t a, bits_t b)
{
    for (int t = SCIREF_WORDS - 1; t >= 0; t--)
        if (a.w[t] != b.w[t]) return a.w[t] < b.w[t] ? -1 : 1;
    return 0;
}
static int key_eq(bits_t a, bits_t b) { return key_cmp(a, b) == 0; }

/* number of occupied orbitals strictly below p, counted one bit at a time */
static int count_below(bits_t d, int p)
{
    int cnt = 0;
    for (int q = 0; q < p; q++) cnt += occupied(d, q);
    return cnt;
}

/* apply a_p to *d: returns +1/-1, or 0 if p is empty */
static int annihilate(bits_t *d, int p)
{
    if (!occupied(*d, p)) return 0;
    int s = (count_below(*d, p) & 1) ? -1 : 1;
    *d = without_bit(*d, p);
    return s;
}

/* apply a+_p to *d: returns +1/-1, or 0 if p is occupied */
static int create(bits_t *d, int p)
{
    if (occupied(*d, p)) return 0;
    int s = (count_below(*d, p) & 1) ? -1 : 1;
    *d = with_bit(*d, p);
    return s;
}

static int n_diff(bits_t a, bits_t b)
{
    int cnt = 0;
    for (int p = 0; p < SCIREF_MAXORB; p++) cnt += occupied(a, p) != occupied(b, p);
    return cnt;
}

static int64_t find_key(const sciref_ctx *c, bits_t k)
{
    int64_t lo = 0, hi = c->M;          /* first index with keys[idx] >= k */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (key_cmp(c->keys[mid], k) < 0) lo = mid + 1; else hi = mid;
    }
    return (lo < c->M && key_eq(c->keys[lo], k)) ? lo : -1;
}

/* <D_I|H|D_I> */
static zd diag_element(const sciref_ctx *c, bits_t d)
{
    zd e = 0;
    for (int i = 0; i < c->norb; i++) {
        if (!occupied(d, i)) continue;
        e += H1(c, i, i);
        for (int j = 0; j < c->norb; j++) {
            if (!occupied(d, j)) continue;
            e += 0.5 * (ERI(c, i, i, j, j) - ERI(c, i, j, j, i));
        }
    }
    return e;
}

/* <D_I|H|D_J> for I != J; *degree receives the excitation degree and *sign the phase.
 * Returns 0 with *degree > 2 when the pair is not connected. */
static zd offdiag_element(const sciref_ctx *c, bits_t bra, bits_t ket, int *degree, int *sign)
{
    int nd = n_diff(bra, ket);
    *degree = nd / 2;
    *sign = 0;
    if (nd != 2 && nd != 4) return 0;
    int from[2], to[2], nf = 0, nt = 0;        /* from: in ket only; to: in bra only */
    for (int p = 0; p < SCIREF_MAXORB; p++) {
        if (occupied(ket, p) && !occupied(bra, p)) from[nf++] = p;
        if (occupied(bra, p) && !occupied(ket, p)) to[nt++] = p;
    }
    bits_t d = ket;
    if (nd == 2) {
        int i = from[0], a = to[0];
        int s = annihilate(&d, i);
        s *= create(&d, a);
        zd v = H1(c, a, i);
        for (int k = 0; k < c->norb; k++) {
            if (!occupied(ket, k) || k == i) continue;
            v += ERI(c, a, i, k, k) - ERI(c, a, k, k, i);
        }
        *sign = s;
        return s * v;
    }
    int i = from[0], j = from[1], a = to[0], b = to[1];   /* i<j, a<b */
    int s = annihilate(&d, j);
    s *= annihilate(&d, i);
    s *= create(&d, a);
    s *= create(&d, b);
    *sign = s;
    return s * (ERI(c, a, i, b, j) - ERI(c, a, j, b, i));
}

/* connections of row I by generation + lookup, sorted ascending by J */
typedef struct { int64_t j; int8_t degree; int8_t sign; zd h; } conn_t;

static int cmp_conn(const void *x, const void *y)
{
    int64_t a = ((const conn_t *)x)->j, b = ((const conn_t *)y)->j;
    return (a > b) - (a < b);
}

static int64_t row_connections(const sciref_ctx *c, int64_t row, conn_t **out)
{
    bits_t d = c->keys[row];
    int occ[SCIREF_MAXORB], vir[SCIREF_MAXORB], no = 0, nv = 0;
    for (int p = 0; p < c->norb; p++) {
        if (occupied(d, p)) occ[no++] = p; else vir[nv++] = p;
    }
    size_t cap = 64, cnt = 0;
    conn_t *list = (conn_t *)malloc(cap * sizeof(conn_t));
    /* singles: i -> a */
    for (int x = 0; x < no; x++)
        for (int y = 0; y < nv; y++) {
            int i = occ[x], a = vir[y];
            if (spin_of(c, i) != spin_of(c, a)) continue;
            bits_t e = with_bit(without_bit(d, i), a);
            int64_t J = find_key(c, e);
            if (J < 0) continue;
            if (cnt == cap) { cap *= 2; list = (conn_t *)realloc(list, cap * sizeof(conn_t)); }
            int deg, sg;
            list[cnt].h = offdiag_element(c, d, e, &deg, &sg);
            list[cnt].j = J; list[cnt].degree = (int8_t)deg; list[cnt].sign = (int8_t)sg;
            cnt++;
        }
    /* doubles: i<j -> a<b */
    for (int x1 = 0; x1 < no; x1++)
        for (int x2 = x1 + 1; x2 < no; x2++)
            for (int y1 = 0; y1 < nv; y1++)
                for (int y2 = y1 + 1; y2 < nv; y2++) {
                    int i = occ[x1], j = occ[x2], a = vir[y1], b = vir[y2];
                    if (spin_of(c, i) + spin_of(c, j) != spin_of(c, a) + spin_of(c, b)) continue;
                    bits_t e = with_bit(with_bit(without_bit(without_bit(d, i), j), a), b);
                    int64_t J = find_key(c, e);
                    if (J < 0) continue;
                    if (cnt == cap) { cap *= 2; list = (conn_t *)realloc(list, cap * sizeof(conn_t)); }
                    int deg, sg;
                    list[cnt].h = offdiag_element(c, d, e, &deg, &sg);
                    list[cnt].j = J; list[cnt].degree = (int8_t)deg; list[cnt].sign = (int8_t)sg;
                    cnt++;
                }
    qsort(list, cnt, sizeof(conn_t), cmp_conn);
    *out = list;
    return (int64_t)cnt;
}

/* ------------------------------------------------------------------ exports */
/* H_II for all rows; out has M scalars (complex: interleaved). */
int sciref_diagonal(const sciref_ctx *c, double *out)
{
    if (!c || !out) return SCIREF_ERR_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < c->M; row++) {
        zd e = diag_element(c, c->keys[row]);
        if (c->is_complex) { out[2 * row] = creal(e); out[2 * row + 1] = cimag(e); }
        else out[row] = creal(e);
    }
    return SCIREF_OK;
}

/* One matrix element <bra|H|ket> of two occupation strings (need not be in the list). */
int sciref_hij(const sciref_ctx *c, uint64_t bra, uint64_t ket, double *out)
{
    if (!c || !out) return SCIREF_ERR_ARG;
    bits_t b = {{bra, 0, 0}}, k = {{ket, 0, 0}};
    zd v;
    if (bra == ket) v = diag_element(c, b);
    else { int deg, sg; v = offdiag_element(c, b, k, &deg, &sg); }
    out[0] = creal(v);
    if (c->is_complex) out[1] = cimag(v);
    return SCIREF_OK;
}

/* Connection list of one row: J ascending, excitation degree, phase (+1/-1).
 * Returns SCIREF_ERR_CAP (with *count set) when cap is too small. */
int sciref_connections(const sciref_ctx *c, int64_t row, int64_t *count, int64_t *J,
                       int8_t *degree, int8_t *phase, int64_t cap)
{
    if (!c || !count || row < 0 || row >= c->M) return SCIREF_ERR_ARG;
    conn_t *list;
    int64_t n = row_connections(c, row, &list);
    *count = n;
    if (n > cap) { free(list); return SCIREF_ERR_CAP; }
    for (int64_t t = 0; t < n; t++) {
        if (J) J[t] = list[t].j;
        if (degree) degree[t] = list[t].degree;
        if (phase) phase[t] = list[t].sign;
    }
    free(list);
    return SCIREF_OK;
}

/* Connections of one row together with their matrix elements <D_row|H|D_J>
 * (complex: interleaved).  Returns SCIREF_ERR_CAP (with *count set) when cap is too small. */
int sciref_row_elements(const sciref_ctx *c, int64_t row, int64_t *count, int64_t *J,
                        double *hvals, int64_t cap)
{
    if (!c || !count || row < 0 || row >= c->M) return SCIREF_ERR_ARG;
    conn_t *list;
    int64_t n = row_connections(c, row, &list);
    *count = n;
    if (n > cap) { free(list); return SCIREF_ERR_CAP; }
    for (int64_t t = 0; t < n; t++) {
        if (J) J[t] = list[t].j;
        if (hvals) {
            if (c->is_complex) { hvals[2 * t] = creal(list[t].h); hvals[2 * t + 1] = cimag(list[t].h); }
            else hvals[t] = creal(list[t].h);
        }
    }
    free(list);
    return SCIREF_OK;
}

/* Number of connected ordered pairs (I, J), I != J, over rows [row_begin, row_end). */
int sciref_count_pairs(const sciref_ctx *c, int64_t row_begin, int64_t row_end, int64_t *count)
{
    if (!c || !count || row_begin < 0 || row_end > c->M || row_begin > row_end) return SCIREF_ERR_ARG;
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t row = row_begin; row < row_end; row++) {
        conn_t *list;
        total += row_connections(c, row, &list);
        free(list);
    }
    *count = total;
    return SCIREF_OK;
}

/* sigma for the listed rows: S[r][v] = sum_J <D_rows[r]|H|D_J> C[J][v].
 * C is [M][nvec] row-major (complex interleaved); S is [nrows][nvec].
 * The diagonal term comes first, then connections in ascending J. */
int sciref_sigma_rows(const sciref_ctx *c, const int64_t *rows, int64_t nrows,
                      const double *C, int nvec, double *S)
{
    if (!c || !rows || !C || !S || nvec <= 0) return SCIREF_ERR_ARG;
    for (int64_t r = 0; r < nrows; r++)
        if (rows[r] < 0 || rows[r] >= c->M) return SCIREF_ERR_ARG;
    const int z = c->is_complex;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t row = rows[r];
        zd *acc = (zd *)malloc((size_t)nvec * sizeof(zd));
        zd hd = diag_element(c, c->keys[row]);
        for (int v = 0; v < nvec; v++) {
            size_t t = (size_t)row * nvec + v;
            zd cv = z ? CMPLX(C[2 * t], C[2 * t + 1]) : CMPLX(C[t], 0.0);
            acc[v] = hd * cv;
        }
        conn_t *list;
        int64_t n = row_connections(c, row, &list);
        for (int64_t k = 0; k < n; k++)
            for (int v = 0; v < nvec; v++) {
                size_t t = (size_t)list[k].j * nvec + v;
                zd cv = z ? CMPLX(C[2 * t], C[2 * t + 1]) : CMPLX(C[t], 0.0);
                acc[v] += list[k].h * cv;
            }
        free(list);
        for (int v = 0; v < nvec; v++) {
            size_t t = (size_t)r * nvec + v;
            if (z) { S[2 * t] = creal(acc[v]); S[2 * t + 1] = cimag(acc[v]); }
            else S[t] = creal(acc[v]);
        }
        free(acc);
    }
    return SCIREF_OK;
}

/* Row sums of magnitudes, the scale that rounding errors of sigma are measured against:
 *   A[r][v] = |H_II| |C_Iv| + sum_J |H_IJ| |C_Jv|,   I = rows[r],
 * over the same connections and elements as sciref_sigma_rows (|.| the modulus in complex
 * mode; A is real, [nrows][nvec]).  sigma_I is a sum of these terms, so |sigma_I| <= A_I,
 * and an error of relative size u in every term moves sigma_I by at most u A_I. */
int sciref_sigma_abs_rows(const sciref_ctx *c, const int64_t *rows, int64_t nrows,
                          const double *C, int nvec, double *A)
{
    if (!c || !rows || !C || !A || nvec <= 0) return SCIREF_ERR_ARG;
    for (int64_t r = 0; r < nrows; r++)
        if (rows[r] < 0 || rows[r] >= c->M) return SCIREF_ERR_ARG;
    const int z = c->is_complex;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t row = rows[r];
        const double hd = cabs(diag_element(c, c->keys[row]));
        for (int v = 0; v < nvec; v++) {
            size_t t = (size_t)row * nvec + v;
            A[(size_t)r * nvec + v] = hd * (z ? cabs(CMPLX(C[2 * t], C[2 * t + 1])) : fabs(C[t]));
        }
        conn_t *list;
        int64_t n = row_connections(c, row, &list);
        for (int64_t k = 0; k < n; k++) {
            const double hk = cabs(list[k].h);
            for (int v = 0; v < nvec; v++) {
                size_t t = (size_t)list[k].j * nvec + v;
                A[(size_t)r * nvec + v] += hk * (z ? cabs(CMPLX(C[2 * t], C[2 * t + 1])) : fabs(C[t]));
            }
        }
        free(list);
    }
    return SCIREF_OK;
}

/* The same sigma rows by the all-pairs route: every J of the list is tested, the
 * excitation degree taken by counting differing bits; no excitation is generated. */
int sciref_sigma_brute_rows(const sciref_ctx *c, const int64_t *rows, int64_t nrows,
                            const double *C, int nvec, double *S)
{
    if (!c || !rows || !C || !S || nvec <= 0) return SCIREF_ERR_ARG;
    for (int64_t r = 0; r < nrows; r++)
        if (rows[r] < 0 || rows[r] >= c->M) return SCIREF_ERR_ARG;
    const int z = c->is_complex;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t row = rows[r];
        bits_t bra = c->keys[row];
        zd *acc = (zd *)calloc((size_t)nvec, sizeof(zd));
        for (int64_t col = 0; col < c->M; col++) {
            bits_t ket = c->keys[col];
            int nd = n_diff(bra, ket);
            if (nd > 4) continue;
            zd hv;
            if (col == row) hv = diag_element(c, bra);
            else { int deg, sg; hv = offdiag_element(c, bra, ket, &deg, &sg); }
            for (int v = 0; v < nvec; v++) {
                size_t t = (size_t)col * nvec + v;
                zd cv = z ? CMPLX(C[2 * t], C[2 * t + 1]) : CMPLX(C[t], 0.0);
                acc[v] += hv * cv;
            }
        }
        for (int v = 0; v < nvec; v++) {
            size_t t = (size_t)r * nvec + v;
            if (z) { S[2 * t] = creal(acc[v]); S[2 * t + 1] = cimag(acc[v]); }
            else S[t] = creal(acc[v]);
        }
        free(acc);
    }
    return SCIREF_OK;
}

/* ------------------------------------------------------------------ density matrices */
/* <bra| a+_p a+_r a_s a_q |ket>: the operators applied one at a time to the ket, right
 * to left (a_q first); 0 when the result is not bra. */
static int two_body_sign(bits_t bra, bits_t ket, int p, int q, int r, int s)
{
    bits_t d = ket;
    int sg = annihilate(&d, q);
    if (!sg) return 0;
    sg *= annihilate(&d, s);
    if (!sg) return 0;
    sg *= create(&d, r);
    if (!sg) return 0;
    sg *= create(&d, p);
    if (!sg || !key_eq(d, bra)) return 0;
    return sg;
}

static int one_body_sign(bits_t bra, bits_t ket, int p, int q)
{
    bits_t d = ket;
    int sg = annihilate(&d, q);
    if (!sg) return 0;
    sg *= create(&d, p);
    if (!sg || !key_eq(d, bra)) return 0;
    return sg;
}

static void add_z(double *a, size_t idx, int is_complex, zd v)
{
    if (is_complex) {
#pragma omp atomic
        a[2 * idx] += creal(v);
#pragma omp atomic
        a[2 * idx + 1] += cimag(v);
    } else {
#pragma omp atomic
        a[idx] += creal(v);
    }
}

/* One- and two-particle density matrices of one vector C (paper Sec. 3.4, density
 * matrices), over spin-orbitals (spin-orbital mode) or spinors:
 *   g1[p][q]       = sum_IJ C_I^* C_J <D_I| a+_p a_q |D_J>
 *   g2[p][q][r][s] = sum_IJ C_I^* C_J <D_I| a+_p a+_r a_s a_q |D_J>
 * so that sum_pq h_pq g1_pq + 1/2 sum_pqrs (pq|rs) g2_pqrs = C^+ H C (Eq. Hamiltonian).
 * Unnormalised (divide by C^+C).  Every candidate operator string for a connected pair
 * (I, J) (the diagonal, singles and doubles of generation + lookup) is applied to D_J
 * explicitly.  g1: norb^2 scalars, g2: norb^4 scalars, zeroed here (complex interleaved). */
int sciref_rdm12(const sciref_ctx *c, const double *C, double *g1, double *g2)
{
    if (!c || !C || !g1 || !g2) return SCIREF_ERR_ARG;
    const int z = c->is_complex;
    const size_t m = (size_t)c->norb;
    memset(g1, 0, m * m * (z ? 2 : 1) * sizeof(double));
    memset(g2, 0, m * m * m * m * (z ? 2 : 1) * sizeof(double));
#pragma omp parallel
    {
        const int maxc = 2 * SCIREF_MAXORB * SCIREF_MAXORB;  /* candidate operator strings per pair */
        int *cq = (int *)malloc(4 * sizeof(int) * maxc);
        int *cs = cq + maxc, *cp = cs + maxc, *cr = cp + maxc;
#pragma omp for schedule(dynamic, 8)
        for (int64_t row = 0; row < c->M; row++) {
            const bits_t bra = c->keys[row];
            const zd cI = conj(z ? CMPLX(C[2 * row], C[2 * row + 1]) : CMPLX(C[row], 0.0));
            conn_t *list;
            int64_t n = row_connections(c, row, &list);
            for (int64_t t = -1; t < n; t++) {   /* t = -1: the diagonal */
                const int64_t col = t < 0 ? row : list[t].j;
                const bits_t ket = c->keys[col];
                const zd w = cI * (z ? CMPLX(C[2 * col], C[2 * col + 1]) : CMPLX(C[col], 0.0));
                int occ[SCIREF_MAXORB], no = 0, from[2], to[2], nf = 0, nt = 0;
                for (int p = 0; p < c->norb; p++) {
                    if (occupied(ket, p)) occ[no++] = p;
                    if (occupied(ket, p) && !occupied(bra, p)) from[nf++] = p;
                    if (occupied(bra, p) && !occupied(ket, p)) to[nt++] = p;
                }
                /* candidate annihilated (q, s) and created (p, r) orbitals */
                int nc = 0;
                if (nf == 0) {
                    for (int x = 0; x < no; x++) {
                        add_z(g1, (size_t)occ[x] * m + occ[x], z, one_body_sign(bra, ket, occ[x], occ[x]) * w);
                        for (int y = 0; y < no; y++) {
                            if (x == y) continue;
                            cq[nc] = occ[x]; cs[nc] = occ[y]; cp[nc] = occ[x]; cr[nc] = occ[y]; nc++;
                            cq[nc] = occ[x]; cs[nc] = occ[y]; cp[nc] = occ[y]; cr[nc] = occ[x]; nc++;
                        }
                    }
                } else if (nf == 1) {
                    const int i = from[0], a = to[0];
                    add_z(g1, (size_t)a * m + i, z, one_body_sign(bra, ket, a, i) * w);
                    for (int x = 0; x < no; x++) {
                        const int k = occ[x];
                        if (k == i) continue;
                        const int qs[2][2] = {{i, k}, {k, i}}, pr[2][2] = {{a, k}, {k, a}};
                        for (int u = 0; u < 2; u++)
                            for (int v = 0; v < 2; v++) {
                                cq[nc] = qs[u][0]; cs[nc] = qs[u][1]; cp[nc] = pr[v][0]; cr[nc] = pr[v][1]; nc++;
                            }
                    }
                } else {
                    const int qs[2][2] = {{from[0], from[1]}, {from[1], from[0]}};
                    const int pr[2][2] = {{to[0], to[1]}, {to[1], to[0]}};
                    for (int u = 0; u < 2; u++)
                        for (int v = 0; v < 2; v++) {
                            cq[nc] = qs[u][0]; cs[nc] = qs[u][1]; cp[nc] = pr[v][0]; cr[nc] = pr[v][1]; nc++;
                        }
                }
                for (int e = 0; e < nc; e++) {
                    const int sg = two_body_sign(bra, ket, cp[e], cq[e], cr[e], cs[e]);
                    if (!sg) continue;
                    const size_t idx = (((size_t)cp[e] * m + cq[e]) * m + cr[e]) * m + cs[e];
                    add_z(g2, idx, z, sg * w);
                }
            }
            free(list);
        }
        free(cq);
    }
    return SCIREF_OK;
}

/* ------------------------------------------------------------------ ENPT2 */
/* Epstein-Nesbet second-order energies of the columns of C (paper Sec. 2.4, Eq. ENPT2E):
 *   E2_k = sum_{I in Q} |sum_{J in P} H_IJ C_Jk|^2 / (E0_k - H_II)
 * with P the determinant list of the context and Q every determinant outside P.  A
 * determinant of Q adds a nonzero term only if some J in P is a single or double
 * excitation away from it (otherwise every H_IJ vanishes), so Q is replaced by the set of
 * single and double excitations of the members of P that are not members of P; nothing
 * else is left out.
 *
 * Steps, each plain:
 *   1. for every J in P, generate each single i -> a and double i<j -> a<b (spin-orbital
 *      mode: alpha and beta counts conserved), in the loops of row_connections, and keep
 *      the pair (I, J) when I is not in the list (binary search);
 *   2. put the pairs into 256 bins by a multiplicative hash of I (equal I, equal bin) and
 *      sort each bin by (I, J), so the J of one I are contiguous and ascending;
 *   3. for each distinct I: numerator_k = sum over its J (ascending) of H_IJ C_Jk, with H_IJ
 *      from offdiag_element (operator application, bra I, ket J), H_II from diag_element,
 *      and add |numerator_k|^2 / (E0_k - H_II) to the bin's partial sum;
 *   4. E2_k = the bins' partial sums added in bin order (the result does not depend on the
 *      number of threads).
 * over_w = 1 sums over W instead of Q: every single and double excitation of the list,
 * members of the list included (their numerators run over the other members J, since an
 * excitation of J is never J): the E2[W] of Eq. EW1, with E2[Q] = E2[W] - E2[P] (Eq.
 * PT2final).
 * Screening (eps > 0): a contribution H_IJ C_J is left out of every numerator of I when
 * |H_IJ| max_k |C_Jk| < eps, the per-element form of the paper's screening of ENPT2
 * contributions by the size of their matrix elements (Sec. 2.3, Table 1's bounds; Sec. 2.4);
 * an I none of whose contributions is kept adds no term.  eps = 0 is the exact sum.
 * C: [M][nroots] row-major (complex interleaved); E0, E2: nroots doubles.  *n_external
 * (if not NULL) receives the number of distinct determinants summed (|Q| restricted as
 * above).  Memory: 16 bytes per generated external pair. */
typedef struct { bits_t key; uint64_t j; } ext_pair;

static int cmp_ext(const void *x, const void *y)
{
    const ext_pair *a = (const ext_pair *)x, *b = (const ext_pair *)y;
    const int k = key_cmp(a->key, b->key);
    if (k) return k;
    return (a->j > b->j) - (a->j < b->j);
}

/* single and double excitations of row j that are not in the list (all of them when
 * keep_members), written to out (if not NULL) in generation order; returns their number */
static int64_t external_excitations(const sciref_ctx *c, int64_t j, ext_pair *out, int keep_members)
{
    bits_t d = c->keys[j];
    int occ[SCIREF_MAXORB], vir[SCIREF_MAXORB], no = 0, nv = 0;
    for (int p = 0; p < c->norb; p++) {
        if (occupied(d, p)) occ[no++] = p; else vir[nv++] = p;
    }
    int64_t cnt = 0;
    for (int x = 0; x < no; x++)
        for (int y = 0; y < nv; y++) {
            int i = occ[x], a = vir[y];
            if (spin_of(c, i) != spin_of(c, a)) continue;
            bits_t e = with_bit(without_bit(d, i), a);
            if (!keep_members && find_key(c, e) >= 0) continue;
            if (out) { out[cnt].key = e; out[cnt].j = (uint64_t)j; }
            cnt++;
        }
    for (int x1 = 0; x1 < no; x1++)
        for (int x2 = x1 + 1; x2 < no; x2++)
            for (int y1 = 0; y1 < nv; y1++)
                for (int y2 = y1 + 1; y2 < nv; y2++) {
                    int i = occ[x1], jj = occ[x2], a = vir[y1], b = vir[y2];
                    if (spin_of(c, i) + spin_of(c, jj) != spin_of(c, a) + spin_of(c, b)) continue;
                    bits_t e = with_bit(with_bit(without_bit(without_bit(d, i), jj), a), b);
                    if (!keep_members && find_key(c, e) >= 0) continue;
                    if (out) { out[cnt].key = e; out[cnt].j = (uint64_t)j; }
                    cnt++;
                }
    return cnt;
}

#define ENPT2_BINS 256
static unsigned enpt2_bin(bits_t key)
{
    const uint64_t folded = key.w[0] ^ key.w[1] * 0xC2B2AE3D27D4EB4Full ^ key.w[2] * 0x165667B19E3779F9ull;
    return (unsigned)((folded * 0x9E3779B97F4A7C15ull) >> 56);
}

int sciref_enpt2(const sciref_ctx *c, const double *C, int nroots, const double *E0, double eps, int over_w,
                 double *E2, int64_t *n_external)
{
    if (!c || !E0 || !E2 || nroots <= 0 || (c->M > 0 && !C) || eps < 0) return SCIREF_ERR_ARG;
    const int z = c->is_complex;
    const int64_t M = c->M;
    /* 1. count, then write, the external pairs of each J */
    int64_t *off = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    if (!off) return SCIREF_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < M; j++) off[j + 1] = external_excitations(c, j, NULL, over_w);
    for (int64_t j = 0; j < M; j++) off[j + 1] += off[j];
    const int64_t np = off[M];
    ext_pair *pairs = (ext_pair *)malloc((size_t)(np > 0 ? np : 1) * sizeof(ext_pair));
    ext_pair *binned = (ext_pair *)malloc((size_t)(np > 0 ? np : 1) * sizeof(ext_pair));
    if (!pairs || !binned) { free(off); free(pairs); free(binned); return SCIREF_ERR_ARG; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < M; j++) external_excitations(c, j, pairs + off[j], over_w);
    free(off);
    /* 2. bins by hash of I (a counting sort), then each bin sorted by (I, J) */
    int64_t bstart[ENPT2_BINS + 1], bfill[ENPT2_BINS];
    memset(bstart, 0, sizeof(bstart));
    for (int64_t t = 0; t < np; t++) bstart[enpt2_bin(pairs[t].key) + 1]++;
    for (int b = 0; b < ENPT2_BINS; b++) bstart[b + 1] += bstart[b];
    for (int b = 0; b < ENPT2_BINS; b++) bfill[b] = bstart[b];
    for (int64_t t = 0; t < np; t++) binned[bfill[enpt2_bin(pairs[t].key)]++] = pairs[t];
    free(pairs);
    double *part = (double *)calloc((size_t)ENPT2_BINS * nroots, sizeof(double));
    int64_t ndist[ENPT2_BINS];
    memset(ndist, 0, sizeof(ndist));
    /* 3. one term per distinct I */
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < ENPT2_BINS; b++) {
        ext_pair *v = binned + bstart[b];
        const int64_t nb = bstart[b + 1] - bstart[b];
        qsort(v, (size_t)nb, sizeof(ext_pair), cmp_ext);
        zd *num = (zd *)malloc((size_t)nroots * sizeof(zd));
        for (int64_t s = 0; s < nb;) {
            int64_t e = s;
            while (e < nb && key_eq(v[e].key, v[s].key)) e++;
            const bits_t ext = v[s].key;
            for (int k = 0; k < nroots; k++) num[k] = 0;
            int kept = 0;
            for (int64_t t = s; t < e; t++) {
                int deg, sg;
                const zd hIJ = offdiag_element(c, ext, c->keys[v[t].j], &deg, &sg);
                double cmax = 0.0;
                for (int k = 0; k < nroots; k++) {
                    const size_t q = (size_t)v[t].j * nroots + k;
                    const double m = z ? cabs(CMPLX(C[2 * q], C[2 * q + 1])) : fabs(C[q]);
                    if (m > cmax) cmax = m;
                }
                if (eps > 0 && cabs(hIJ) * cmax < eps) continue;
                kept = 1;
                for (int k = 0; k < nroots; k++) {
                    const size_t q = (size_t)v[t].j * nroots + k;
                    num[k] += hIJ * (z ? CMPLX(C[2 * q], C[2 * q + 1]) : CMPLX(C[q], 0.0));
                }
            }
            if (!kept) {
                s = e;
                continue;
            }
            const double hII = creal(diag_element(c, ext));
            for (int k = 0; k < nroots; k++) {
                const double m2 = creal(num[k]) * creal(num[k]) + cimag(num[k]) * cimag(num[k]);
                part[(size_t)b * nroots + k] += m2 / (E0[k] - hII);
            }
            ndist[b]++;
            s = e;
        }
        free(num);
    }
    /* 4. bins in order */
    int64_t total = 0;
    for (int k = 0; k < nroots; k++) E2[k] = 0.0;
    for (int b = 0; b < ENPT2_BINS; b++) {
        for (int k = 0; k < nroots; k++) E2[k] += part[(size_t)b * nroots + k];
        total += ndist[b];
    }
    if (n_external) *n_external = total;
    free(part);
    free(binned);
    return SCIREF_OK;
}
