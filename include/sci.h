/*
 * sci.h -- C ABI of libsci: sigma = H c for selected configuration interaction on one
 * GB300 (sm_103a).
 *
 * The operation (MetaWave, arXiv 2501.18185):
 *   H = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs (pq|rs) a+_p a+_r a_s a_q   (Sec. 2.1,
 *       Eq. Hamiltonian / Eq. sym_op, Mulliken notation, H = H^+)
 *   sigma_I = sum_J <D_I|H|D_J> C_J over a sorted determinant list   (Sec. 2.4, the
 *       diagonalisation paragraph: H is applied through matrix-vector products whose
 *       nonzero elements are recomputed whenever needed and never stored)
 * The library stores integrals (Sec. 3.2, IntegralManager) and a sorted basis
 * (Sec. 3.2, BasisManager) in device memory and evaluates every Slater-Condon element
 * on the fly.
 *
 * Determinant keys.  One uint64 per determinant.
 *   Spin-orbital mode (n spatial orbitals, n <= 32): bit p (p < n) is alpha orbital p,
 *   bit n+p is beta orbital p; bits >= 2n are zero.
 *   Spinor mode (n spinors, n <= 64): bit p is spinor p.
 * Phase convention: |D> = a+_{p1} a+_{p2} ... |0> with p1 < p2 < ... in bit order (so
 * every alpha creator precedes every beta creator).  Energies do not depend on this
 * convention; the signs of sigma and of off-diagonal elements do.
 * The list must be strictly ascending as unsigned 64-bit integers; a list that is not
 * is rejected (no resorting).
 *
 * Vectors.  C and S are [M][nvec] row-major: the nvec coefficients of one determinant
 * are contiguous.  Real mode: double (or float input, see SCI_PREC_*).  Complex mode:
 * interleaved (re, im) double pairs.  There is no conjugation of C: S = H C.
 *
 * Errors.  Every call returns SCI_OK (0) or a negative code; no C++ exception crosses
 * the ABI.  Argument errors are detected before any work is queued.  Conditions found
 * on the device set a sticky status word that sci_sync_status() returns.  After an
 * error the context stays valid; calls that need missing state return SCI_ERR_STATE.
 * sci_last_error() gives a readable message for the last failure of a context.
 *
 * Ownership.  The caller owns every pointer it passes.  The library copies integrals
 * and keys into device memory owned by the context and freed by sci_destroy().  C and S
 * of sci_sigma() are borrowed device pointers (e.g. torch tensor data_ptr()).
 *
 * Streams.  Work is queued on the stream given at creation (or by sci_set_stream); a
 * NULL stream is the legacy default stream.  sci_sigma() allocates nothing, takes no
 * host synchronisation and only queues kernels.
 */
#ifndef SCI_H
#define SCI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sci_ctx sci_ctx;

enum {
    SCI_OK = 0,
    SCI_ERR_ARG = -1,        /* invalid argument (null pointer, bad size, bad enum, ...) */
    SCI_ERR_UNSORTED = -2,   /* determinant list not ascending */
    SCI_ERR_DUPLICATE = -3,  /* determinant list holds a key twice */
    SCI_ERR_POPCOUNT = -4,   /* a key has the wrong electron count or stray bits */
    SCI_ERR_NOMEM = -5,      /* device allocation failed */
    SCI_ERR_CUDA = -6,       /* a CUDA runtime call failed */
    SCI_ERR_STATE = -7,      /* call needs state that is missing (e.g. no integrals) */
    SCI_ERR_OVERFLOW = -8,   /* a size exceeds an internal limit or an output capacity */
    SCI_ERR_TIMEOUT = -9     /* reserved: a bounded device wait gave up */
};

enum { SCI_REAL64 = 1, SCI_COMPLEX128 = 2 };                 /* Hamiltonian scalar type */
enum { SCI_SPIN_ORBITALS = 1, SCI_SPINORS = 2 };             /* orbital mode */
enum {
    SCI_PREC_F64 = 1,                /* C double (complex: double pairs), S double */
    SCI_PREC_F32_STORE_F64_ACC = 2,  /* real mode only.  C float, S double.  The double-
                                        excitation table ((ai|bj) - (aj|bi) and (ai|bj))
                                        is rounded to float once; each product of two
                                        floats is formed exactly (FMA error term), the
                                        per-bucket sums are compensated (paired FP32) and
                                        accumulated into S in FP64.  Singles use the
                                        paired-FP32 Fock sums of SCI_PREC_F64_DS.  The
                                        result carries the FP32 rounding of the integrals
                                        and of C (~1e-7 relative). */
    SCI_PREC_F64_DS = 3              /* C and S as for SCI_PREC_F64; the double-excitation
                                        products and per-bucket sums run in paired FP32
                                        ("double-single") arithmetic on the FP32 pipes:
                                        each FP64 operand is split into hi + lo floats,
                                        products keep ~47 bits, sums are compensated, and
                                        the bucket sums are added to S in FP64.  Agrees with
                                        SCI_PREC_F64 to ~1e-13 relative. */
};

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t (may be
 * NULL).  Allocates a 4-byte status word; the first context on a device also commits the
 * fixed scratch array of sci_connections_noalloc() there.  Returns SCI_ERR_ARG for a bad
 * device, SCI_ERR_CUDA if the device or that scratch cannot be set up. */
int sci_create(sci_ctx **out, int device, void *cuda_stream);

/* Free every device buffer of the context and the context itself.  NULL is allowed. */
int sci_destroy(sci_ctx *ctx);

/* Change the stream used by later calls. */
int sci_set_stream(sci_ctx *ctx, void *cuda_stream);

/* Load the Hamiltonian (Sec. 2.1, Eq. Hamiltonian; Sec. 3.2, IntegralManager).
 *   scalar: SCI_REAL64 or SCI_COMPLEX128.  mode: SCI_SPIN_ORBITALS (n <= 128 spatial
 *   orbitals, real only) or SCI_SPINORS (n <= 256 spinors); above 32 spatial orbitals or
 *   64 spinors the determinant list needs two-word keys, above 64 or 128 three-word keys,
 *   above 96 or 192 four-word keys (sci_set_determinants_w).
 *   h:    host, n*n row-major, h[p*n+q] = h_pq, Hermitian (complex: interleaved re,im).
 *   eri:  host, n^4 row-major, eri[((p*n+q)*n+r)*n+s] = (pq|rs), or NULL.
 *   chol: host, naux*n*n, (pq|rs) = sum_P chol[P][p][q] chol[P][r][s], or NULL.
 * Exactly one of eri / chol must be given.  The permutation symmetries
 * (pq|rs) = (rs|pq) = (qp|sr)^* and h = h^+ (Sec. 3.2, IntegralManager; the symmetry of
 * Eq. sym_op) are checked to 1e-10 relative and violations return SCI_ERR_ARG.
 * Synchronous: returns after the device tables are built.  A later call with the same
 * mode and n keeps the determinant list; a different mode or n drops it. */
int sci_set_integrals(sci_ctx *ctx, int scalar, int mode, int n, const void *h,
                      const void *eri, int naux, const void *chol);

/* The same with the integrals' location given: on_device = 0 reads h, eri and chol from
 * host memory (as sci_set_integrals); on_device = 1 reads them from memory of the
 * context's device (or managed memory), in place, with the same layouts, and runs the
 * symmetry checks on the device (max |a - b| over symmetric pairs against 1e-10 of the
 * largest magnitude; a value that is not finite is rejected).  Pointers that are not
 * memory of the context's device return SCI_ERR_ARG.  The caller keeps ownership; the
 * buffers are not read after the call returns.  Synchronous. */
int sci_set_integrals_ex(sci_ctx *ctx, int scalar, int mode, int n, const void *h,
                         const void *eri, int naux, const void *chol, int on_device);

/* Load a strictly ascending determinant list (Sec. 3.2, BasisManager) and build the
 * connection tables: keys are validated on the device (order, duplicates, electron
 * counts), the (N-2)- and (N-1)-hole bucket tables are sorted out, and the diagonal
 * H_II is computed.  Needs integrals (SCI_ERR_STATE otherwise).
 *   keys: host or device pointer (keys_on_device 0/1), M entries, M >= 0.
 *   n_alpha, n_beta: electrons per spin (spin-orbital mode); spinor mode: n_alpha = N
 *   electrons and n_beta = -1.
 * Errors: SCI_ERR_UNSORTED, SCI_ERR_DUPLICATE, SCI_ERR_POPCOUNT for bad lists,
 * SCI_ERR_NOMEM when the tables do not fit, SCI_ERR_OVERFLOW for M >= 2^31.
 * Synchronous. */
int sci_set_determinants(sci_ctx *ctx, const uint64_t *keys, int64_t M, int n_alpha,
                         int n_beta, int keys_on_device);

/* The same for occupation strings of more than 64 spin-orbitals or spinors (up to 256):
 * keys are M strings of nwords (1 to 4) 64-bit words, word w holding orbitals
 * 64w..64w+63 (the paper keeps an orbital configuration as an array of 64-bit integers,
 * Sec. 3.2), strictly ascending as unsigned (64 x nwords)-bit integers; nwords must cover
 * the orbitals (64 nwords >= 2n, or >= n spinors; SCI_ERR_ARG otherwise).  The bucket keys
 * are then (64 x nwords)-bit, sorted by nwords stable radix passes.  Sigma (every precision
 * mode, deterministic mode included), the diagonal, pair counts, row costs, the connection
 * exports, row ranges (sci_set_row_range) and the density matrices (sci_rdm12,
 * sci_rdm_grads) work on two- to four-word lists as on one word; ENPT2 (sci_enpt2) on
 * up to three words (SCI_ERR_ARG for four); batches need one-word keys (SCI_ERR_ARG).  sci_set_determinants (one word) returns
 * SCI_ERR_ARG when the orbitals do not fit one word.  Errors as sci_set_determinants. */
int sci_set_determinants_w(sci_ctx *ctx, const uint64_t *keys, int nwords, int64_t M, int n_alpha,
                           int n_beta, int keys_on_device);

/* Copy the diagonal H_II (real, FP64) into the device array hdiag[M].  Queued on the
 * context stream. */
int sci_diagonal(sci_ctx *ctx, double *hdiag);

/* S = H C (Sec. 2.4, the diagonalisation paragraph) for nvec >= 1 vectors.
 *   C: device, [M][nvec]; S: device, [M][nvec], overwritten (see SCI_PREC_* for types).
 *   C and S must not overlap.  Queued on the context stream; allocates nothing.
 * Accumulation into S uses FP64 atomic adds, so the summation order (and the last bits
 * of S) can differ between calls. */
int sci_sigma(sci_ctx *ctx, const void *C, void *S, int nvec, int prec);

/* Row range of later sci_sigma() and sci_sigma_host() calls on this context: the data
 * path of a row-partitioned sigma over several processes.  The paper keeps the static
 * data on every process and distributes the results, which are merged at the end
 * (Sec. 3.1, the MPI dynamic scheduler); here every process holds the integrals and the
 * whole determinant list, computes the rows [row_begin, row_end) of S, and the rows of
 * all processes are merged by one all-gather (the caller's collective).
 * After this call sci_sigma() writes S rows [row_begin, row_end) only and leaves every
 * other row of S as it was (sci_sigma_host() copies back only those rows), and
 * sci_count_pairs() counts the pairs (I, J) with I in the range.  The call builds range
 * tables: the (N-2)- and (N-1)-hole buckets that hold a member in the range, whole and in
 * the order of the full tables, so a range costs device memory in proportion to the
 * buckets it touches.  row_begin = 0 and row_end = M return to the whole list and free
 * them; a new determinant list clears the range.  Density matrices, ENPT2, the
 * connection exports and batches always use the whole list.
 * Synchronous (waits for the context stream first).  Errors: SCI_ERR_STATE without
 * determinants, SCI_ERR_ARG for a range outside [0, M], SCI_ERR_NOMEM. */
int sci_set_row_range(sci_ctx *ctx, int64_t row_begin, int64_t row_end);

/* Buckets walked in tiles.  The double excitations of sigma (Sec. 2.4) are summed per
 * (N-2)-hole bucket of the connection tables (the determinants that share N-2
 * electrons), each bucket staged in shared memory beside a window of rows.  Buckets of
 * more than `members` members are instead walked by a tiled kernel that takes 256 of a
 * bucket's members as rows per CTA and streams all its members through shared memory in
 * column tiles.  By default (members = 0) the threshold is 512 members, and 384 for
 * launches that stage 64 bytes or more per window row (8 real vectors); a threshold set
 * here applies to every launch.  So no bucket is too large for sigma
 * (up to the table format's 65,535 members), and a few large buckets no longer widen
 * every window.  Results are the same sums in another order: equal within rounding, and
 * the deterministic mode stays bit for bit reproducible at a fixed threshold.  Density
 * matrices (sci_rdm12) keep whole-bucket staging and return SCI_ERR_OVERFLOW for a bucket
 * that does not fit.  A threshold above what the window kernels can stage returns
 * SCI_ERR_OVERFLOW and keeps the previous one.  Synchronous (waits for the context
 * stream; rebuilds the tile lists of the list and of a row range).  Errors: SCI_ERR_ARG
 * for members outside [0, 65535]. */
int sci_set_tile_threshold(sci_ctx *ctx, int members);

/* Deterministic accumulation for later sci_sigma() calls on this context.  By default
 * sigma adds each (bucket, member) row sum into S with an FP64 atomic add, so the order of
 * the additions, and the last bits of S, vary between calls.  With max_nvec > 0 the
 * context holds, for up to max_nvec vectors, one slot per bucket entry and per vector for
 * those row sums, in row order (each table's entries sorted by row with a stable sort, so
 * ascending table position within a row; built once here); sigma then stores each row sum
 * in its slot and a second kernel forms S_I = H_II C_I + the sum of row I's contiguous
 * slots, one warp per row: lane l takes the row's slots l, l + 32, ... and the lanes are
 * combined by a fixed butterfly of warp shuffles.  Repeated calls on the same inputs give
 * bitwise equal S.  Costs
 * device memory: (entries of both tables) x max_nvec scalars plus 4 bytes per entry and
 * per row; sigma with nvec > max_nvec returns SCI_ERR_ARG.  Every precision mode is
 * served; a row range (sci_set_row_range) cannot be combined with it (SCI_ERR_STATE).
 * max_nvec = 0 returns to atomics and frees the buffers; a new determinant list clears it.
 * Synchronous.  Errors: SCI_ERR_STATE without determinants or with a row range set,
 * SCI_ERR_ARG for max_nvec < 0, SCI_ERR_NOMEM. */
int sci_set_deterministic(sci_ctx *ctx, int max_nvec);

/* Cost of each row of sigma, for balancing row ranges: cost[I] = the number of
 * determinants J != I of the list within a single or double excitation of I (the
 * off-diagonal elements of row I of H), exact.  cost: device, M int64, overwritten.
 * Queued on the context stream; uses the whole list whatever the row range. */
int sci_row_costs(sci_ctx *ctx, int64_t *cost);

/* Connection list of rows [row_begin, row_end) for tests and debugging: every ordered
 * pair (I, J), I != J, with excitation degree 1 or 2 and both in the list, sorted by
 * (I, J), with the degree and the phase (+1/-1) of <D_I| relative to the excitation
 * operator applied to |D_J> (a+_a a_i for singles; a+_b a+_a a_i a_j, i<j, a<b, for
 * doubles).  rows, J, degree, phase are host arrays of capacity cap (any may be NULL).
 * *count receives the number of pairs; SCI_ERR_OVERFLOW if it exceeds cap.
 * Synchronous; allocates temporary device memory. */
int sci_connections(sci_ctx *ctx, int64_t row_begin, int64_t row_end, int64_t *count,
                    int64_t *rows, int64_t *J, int8_t *degree, int8_t *phase, int64_t cap);

/* The paper has no counterpart to this call: it is a service for callers that cannot
 * allocate device memory.  Such callers include processes whose device memory belongs to
 * a pooling allocator (a framework's caching allocator, or an arena sized to the whole
 * card), where a late cudaMalloc fails or fragments the pool, and programs that keep
 * several streams busy and cannot afford cudaFree, which synchronises the whole device.
 *
 * Same results as sci_connections() (same arguments, same sorted output), but it calls
 * no cudaMalloc, cudaFree or other allocating routine, on the device or on the host.
 * Its device scratch (a slot counter and the unsorted pairs) is a fixed array inside the
 * library, SCI_NOALLOC_MAX_PAIRS pairs (about 4.5 MiB).  The CUDA runtime loads the
 * array's module lazily, so sci_create() loads it on the context's device and looks up
 * the array's device address (cudaGetSymbolAddress) there: the device memory is
 * committed when the first context on that device is created and held until the process
 * exits, and no call of this function is the first touch.
 *   - rows and J must be non-NULL when cap > 0: the list is sorted in place in them.
 *   - More than SCI_NOALLOC_MAX_PAIRS connections in [row_begin, row_end) returns
 *     SCI_ERR_OVERFLOW, with *count set to the true number; split the range.
 *   - Every call shares the scratch array, which keeps the last call's contents; the
 *     call clears the counter itself.  Calls that overlap on the GPU (from two host
 *     threads, or on two streams) race and corrupt each other's results.
 * Synchronous. */
#define SCI_NOALLOC_MAX_PAIRS 524288
int sci_connections_noalloc(sci_ctx *ctx, int64_t row_begin, int64_t row_end, int64_t *count,
                            int64_t *rows, int64_t *J, int8_t *degree, int8_t *phase,
                            int64_t cap);

/* Number of connected ordered pairs (I, J), I != J, excitation degree <= 2 (every
 * off-diagonal element that sigma evaluates, counted whether or not its value is 0);
 * with a row range set (sci_set_row_range), the pairs with I in the range. */
int sci_count_pairs(sci_ctx *ctx, int64_t *pairs);

/* sigma for callers holding HOST buffers: C_host [M][nvec] is copied to the device, S
 * is computed as by sci_sigma() and copied back into S_host [M][nvec].  Staging buffers
 * are allocated by the context on first use (and grown when nvec grows).  Synchronous.
 * Host buffers may be pageable; pinned ones copy faster. */
int sci_sigma_host(sci_ctx *ctx, const void *C_host, void *S_host, int nvec, int prec);

/* Table sizes, for reports: out[0..n) receives, in order, M, pairs, entries and buckets
 * of the (N-2)-hole table, entries and buckets of the (N-1)-hole table, the largest
 * bucket, the device bytes held by the context, the double-excitation pairs and the
 * single-excitation pairs (with a row range set, the three pair counts are the range's:
 * pairs (I, J) with I in the range).  n <= 10. */
int sci_info(sci_ctx *ctx, int64_t *out, int n);

/* Kernel timing for reports.  sci_profile(ctx, 1) makes later sci_sigma() calls record
 * CUDA events on the context stream around each of their kernels; sci_kernel_times()
 * waits for the last such call and writes the durations in milliseconds of its diagonal
 * initialisation, double-excitation and single-excitation kernels and, in deterministic
 * mode (sci_set_deterministic), of the per-row sums (0 otherwise) to ms[0..n), n <= 4. */
int sci_profile(sci_ctx *ctx, int enable);
int sci_kernel_times(sci_ctx *ctx, float *ms, int n);

/* One- and two-particle reduced density matrices (Sec. 3.4), summed over the columns of
 * C with weights:
 *   rdm1[p][q]       = sum_k w_k <c_k| a+_p a_q |c_k>
 *   rdm2[p][q][r][s] = sum_k w_k <c_k| a+_p a+_r a_s a_q |c_k>
 * over the norb = 2n spin-orbitals (spin-orbital mode, bit order of the keys) or the n
 * spinors, norb <= 256 (one- to four-word keys), unnormalised: for a normalised c the
 * energy of Eq. Hamiltonian is
 * sum h_pq rdm1_pq + 1/2 sum (pq|rs) rdm2_pqrs (spin-orbital integrals).
 *   C: device, [M][nvec], double (real mode) or complex128 (complex mode), nvec >= 1.
 *   weights: HOST, nvec doubles, or NULL for all ones.
 *   rdm1: device, [norb][norb] scalars, overwritten.
 *   rdm2: device, [norb]^4 scalars, overwritten; or NULL to skip the double-excitation
 *     walk (then only rdm1 is formed).
 * Connections are recomputed from the tables built by sci_set_determinants(); the context
 * allocates a scratch buffer (about norb^3 + the pair-table size scalars) on first use and
 * grows it when needed, so calls that grow it are not graph-capturable.  Queued on the
 * context stream (the weights are copied synchronously).  The summation order of the
 * device atomics is not fixed: results agree with a fixed-order sum to rounding.
 * Errors: SCI_ERR_STATE before integrals and determinants, SCI_ERR_ARG for NULL C/rdm1 or
 * nvec < 1, SCI_ERR_OVERFLOW if the largest (N-2) bucket does not fit the staging window,
 * SCI_ERR_NOMEM. */
int sci_rdm12(sci_ctx *ctx, const void *C, int nvec, const double *weights, void *rdm1, void *rdm2);

/* Gradients of weighted Rayleigh quotients with respect to the integrals, from the density
 * matrices of sci_rdm12 (Sec. 3.4) contracted on the device.  Real spin-orbital mode.
 * With g1, g2 the spin-orbital density matrices of sum_k w_k |c_k><c_k| (see sci_rdm12):
 *   gamma[p][q]       = sum_s g1[ps][qs]                    (dE/dh_pq for E = c^T H c)
 *   Gamma[p][q][r][s] = sum_{s1,s2} g2[p s1][q s1][r s2][s s2]  (dE/d(pq|rs) = Gamma / 2)
 *   gchol[P][p][q]    = sum_rs Gamma[p][q][r][s] chol[P][r][s]
 *                                   (dE/dL^P_pq for (pq|rs) = sum_P L^P_pq L^P_rs)
 * over the n spatial orbitals (bit p < n alpha p, bit n + p beta p).
 *   C: device [M][nvec] doubles; weights: HOST, nvec doubles or NULL (all ones).
 *   gamma: device [n][n] or NULL.  Gamma: device [n]^4 or NULL.
 *   chol: device [naux][n][n] and gchol: device [naux][n][n] (overwritten), or both NULL.
 * The 2-RDM walk runs only when Gamma or chol is given.  Synchronous; allocates and frees
 * a scratch buffer (the spin-orbital matrices, (2n)^4 doubles).  Errors: SCI_ERR_STATE,
 * SCI_ERR_ARG (mode, NULL operands, naux < 1), SCI_ERR_NOMEM, and those of sci_rdm12. */
int sci_rdm_grads(sci_ctx *ctx, const double *C, int nvec, const double *weights, double *gamma,
                  double *Gamma, int naux, const double *chol, double *gchol);

/* Epstein-Nesbet second-order energy of roots of the variational space (Sec. 2.4,
 * constraint-based ENPT2, with P_m = P):
 *   E2_k[Q] = E2_k[W] - E2_k[P]                                         (Eq. PT2final)
 *   E2_k[W] = sum_{I in W} (sum_{J in P} H_IJ c_Jk)^2 / (E0_k - H_II)    (Eq. EW1)
 *   E2_k[P] = sum_{I in P} (<I|H|c_k> - c_Ik H_II)^2 / (E0_k - H_II)     (Eq. EP1)
 * over W, the determinants within a single or double excitation of the list.  Real
 * spin-orbital mode (batches by a code of the beta string) or complex spinor mode (no
 * spin conservation, the 4C workloads of Sec. 4; batches by a code of the whole string;
 * the squares are |.|^2 of complex numerators), on one-word lists (n <= 32 spatial
 * orbitals or n <= 64 spinors) or two-word lists (sci_set_determinants_w: n <= 64 or
 * n <= 128; the table keys are then 128-bit, claimed by a 16-byte compare-and-swap), or
 * three-word lists (n <= 96 or n <= 192, fewer than 64 electrons when the list has 192
 * spin-orbitals or spinors: words 0-1 of a key are claimed by the 16-byte
 * compare-and-swap and word 2 by an 8-byte one).
 * Spinor mode with real integrals returns SCI_ERR_ARG.
 *   C: device, [M][nroots] doubles (complex mode: complex128, interleaved), 1 <= nroots
 *      <= 8 (need not be normalised; the formulas use c as given, so pass normalised
 *      eigenvectors for energies).
 *   E0: HOST, nroots doubles (the zeroth-order energies E0_k).
 *   eps: screening; a generated contribution with |H_IJ| max_k |c_Jk| < eps is dropped
 *      (0 = exact).
 *   table_bytes: device memory for the hash table of one batch (8 + 8 nroots bytes per
 *      entry, 8 + 16 nroots in complex mode; with two- or three-word keys 16 or 24 bytes
 *      of key and the entry rounded up to a multiple of 16 bytes; capacity the largest power of two
 *      within the budget, at least 256).  W is split into
 *      2^t batches (t <= 10) so that a batch's generated excitations fill at most 60% of
 *      it; a batch that still overflows (or probes too far) restarts the sum with twice
 *      the batches.  Larger is not always faster: the inserts are random accesses, and a
 *      table of tens of GB makes them slower than the extra passes of a smaller one
 *      (measured on a 200k-determinant 64-spinor space: 1.9 s with 2-24 GB, 3.2 s with
 *      96 GB; a 2M-determinant real space: 7.9-8.0 s with 16-96 GB, 8.7 s with 4 GB).
 *   E2: HOST, 3 x nroots doubles, overwritten: E2[W], then E2[P], then E2[Q].
 *   stats: HOST, 8 int64 or NULL: batches, distinct W determinants summed, passes run
 *      (with restarts), table capacity, microseconds spent clearing the table,
 *      generating and evaluating (CUDA events), and the distinct count of the sampling
 *      batch (-1 if none).  Before the sum, one batch of a four-times finer split is
 *      generated to estimate the distinct determinants; the batch count is chosen from
 *      that estimate (25% margin) and never exceeds the bound from the generated count.
 * Synchronous.  Allocates sigma scratch (M x nroots doubles) and the table for the call.
 * Errors: SCI_ERR_ARG (mode, sizes, NULL), SCI_ERR_STATE, SCI_ERR_NOMEM, SCI_ERR_OVERFLOW
 * (the table is too small even at 1024 batches). */
int sci_enpt2(sci_ctx *ctx, const double *C, int nroots, const double *E0, double eps,
              size_t table_bytes, double *E2, int64_t *stats);

/* ---------------------------------------------------------------- batched instances
 * Many small real spin-orbital Hamiltonians (each a sci_ctx with integrals and
 * determinants set) applied to their vectors in ONE persistent kernel launch, the GPU
 * form of the paper's dynamic task scheduling (Sec. 3.1).  The paper has no batched
 * entry point; its tasks are oCFG pairs of one Hamiltonian.
 *
 * Vectors: all instances' C (and S) live in one device array of sum_i M_i doubles,
 * instance i at offset sum_{j<i} M_j (its add order); one vector per instance.
 * Schedules: SCI_SCHED_TILE walks the bucket tables (any determinant list, atomics into
 * S); SCI_SCHED_WARP gives each determinant a warp that generates its excitations and
 * indexes them by combinatorial ranking (full-CI instances of at most 20 orbitals, S stored directly);
 * SCI_SCHED_AUTO times both on each instance and keeps the faster (decisions and times
 * cached by (n, n_alpha, n_beta, M) in the batch, so equal shapes are timed once).
 * The batch keeps pointers into the instances' tables: an instance must outlive the
 * batch and must not be re-set after sci_batch_plan().  Work runs on a stream of the
 * batch, ordered after the work queued on the caller's stream at the time of the call
 * and before later work queued there. */
typedef struct sci_batch sci_batch;
enum { SCI_SCHED_AUTO = 0, SCI_SCHED_TILE = 1, SCI_SCHED_WARP = 2 };
int sci_batch_create(sci_batch **out, int device, void *cuda_stream);
int sci_batch_destroy(sci_batch *b);
/* Append an instance; returns its index (>= 0) or a negative error code. */
int sci_batch_add(sci_batch *b, sci_ctx *instance);
/* Choose the schedules and build the work list (items ordered by decreasing cost).  AUTO
 * runs both schedules on C -> S (device arrays as above; S is overwritten) to time them;
 * TILE and WARP need no vectors (C, S may be NULL).  Synchronous. */
int sci_batch_plan(sci_batch *b, int schedule, const double *C, double *S);
/* S = H_i C_i for every instance, one persistent launch (after a counter reset and a
 * clear of S). */
int sci_batch_sigma(sci_batch *b, const double *C, double *S);
/* Capture that launch for fixed C and S in a CUDA graph owned by the batch; replay it. */
int sci_batch_capture(sci_batch *b, const double *C, double *S);
int sci_batch_replay(sci_batch *b);
/* Instances taking part in later sigma launches and replays (captured graphs included):
 * active (host, n = instance count) nonzero = computed, 0 = skipped (its S stays zero).
 * Copied on the batch stream, ordered after the launches already queued there.
 * sci_batch_plan() makes every instance active. */
int sci_batch_set_active(sci_batch *b, const int32_t *active, int n);
/* Per instance: chosen schedule, autotuner times in ms (-1 if not timed), offset. */
int sci_batch_info(sci_batch *b, int i, int *schedule, float *ms_tile, float *ms_warp, int64_t *offset);
/* out[0..n): work items, persistent CTAs, total determinants, total pairs; n <= 4. */
int sci_batch_items(sci_batch *b, int64_t *out, int n);
const char *sci_batch_last_error(const sci_batch *b);

/* Block-vector products for the subspace algebra of a block Davidson solver around
 * sigma (Sec. 2.4, the diagonalisation paragraph: the eigenproblem is solved through
 * matrix-vector products; the paper leaves the solver's linear algebra unspecified).
 * Real FP64 data only.  All matrices are device pointers, row-major with the given
 * leading dimension (in elements; lda >= width).  Asynchronous on the context stream;
 * they need no Hamiltonian or determinant list.
 * prec: SCI_PREC_F64 (FP64 FMA) or SCI_PREC_F64_DS (paired FP32 on the FP32 pipes,
 * inputs carried to 2^-47 relative, sums folded into FP64 every 32 rows).
 *
 * sci_bv_gemm_tn: P[k][a] = A^T B for A [M][lda] (first k columns) and B [M][ldb] (first
 *   a columns).  1 <= a <= 16 and k <= 8 * 256 / pow2(a) (256 for a <= 8, 128 for a <= 16).
 *   Deterministic (fixed reduction order).  The context holds a partial-sum buffer of
 *   (CTAs x k x a) doubles, allocated on first use and grown when k x a grows; calls that
 *   grow it are not graph-capturable.
 * sci_bv_gemm_nn: C[m][j] = sum_i A1[m][i] S1[i][j] + sum_i A2[m][i] S2[i][j]
 *   (+ beta C[m][j] when beta != 0) for j < a, S1 [k1][a] and S2 [k2][a] row-major on the
 *   device, 1 <= a <= 16, k1 + k2 <= 256 (either may be 0 with a NULL operand).  Each row
 *   is computed from its own inputs only, so C may alias A1 or A2 (same base and stride)
 *   for an in-place update.  Optional epilogue for residuals:
 *     colsq (device [a], or NULL): += sum_m C[m][j]^2 of the value before preconditioning
 *       (FP64 atomics; the order of the additions is not fixed);
 *     dg (device [M]) and shift (device [a]), or NULL: the stored value becomes
 *       C[m][j] / (shift[j] - dg[m]) with a denominator below 1e-8 in magnitude replaced
 *       by 1e-8 (the Davidson diagonal preconditioner), the quotient taken in FP32.
 * Errors: SCI_ERR_ARG for sizes out of range or NULL operands; SCI_ERR_NOMEM if the
 * partial-sum buffer cannot be grown. */
int sci_bv_gemm_tn(sci_ctx *ctx, int64_t M, int k, int a, const double *A, int64_t lda,
                   const double *B, int64_t ldb, double *P, int prec);
int sci_bv_gemm_nn(sci_ctx *ctx, int64_t M, int a, const double *A1, int64_t lda1, int k1,
                   const double *S1, const double *A2, int64_t lda2, int k2, const double *S2,
                   double beta, double *C, int64_t ldc, const double *dg, const double *shift,
                   double *colsq, int prec);

/* Segmented block-vector products: the subspace algebra of many independent solvers
 * (the instances of a batch) whose vectors lie end to end in one device array, instance
 * s on rows [offsets[s], offsets[s+1]).  A block of k such vectors is column-major:
 * column j starts at A + j * lda (lda >= offsets[nseg] when k > 1).  FP64, device
 * pointers, asynchronous on the stream given at creation (NULL: the legacy default
 * stream).  Same role as the sci_bv_* products for one instance (Sec. 2.4, the
 * diagonalisation paragraph).
 *
 * sci_seg_create: offsets (host, nseg + 1 values, offsets[0] = 0, non-decreasing; empty
 *   instances allowed); kmax (1..256) bounds k, k1 and k2.  Allocates the work list and
 *   a partial-sum buffer ((total rows / 2048 + nseg) x kmax doubles).  Synchronous.
 *   Errors: SCI_ERR_ARG, SCI_ERR_OVERFLOW, SCI_ERR_NOMEM.
 * sci_seg_tn: out[s * k + j] = sum_{i in s} A[j * lda + i] t[i] for j < k (out: device,
 *   nseg x k; 0 for an empty instance).  Deterministic: per-item partials summed in item
 *   order.
 * sci_seg_nn: y[i] = beta[s] y[i] + alpha1 sum_{j<k1} A1[j * lda1 + i] c1[s * k1 + j]
 *                                 + alpha2 sum_{j<k2} A2[j * lda2 + i] c2[s * k2 + j]
 *   for i in instance s (beta, c1, c2: device arrays [nseg], [nseg x k1], [nseg x k2];
 *   beta NULL means 0; y is not read where beta[s] = 0).  k1 or k2 may be 0 with NULL
 *   operands.  If dg (device [total rows]) is given, the stored value is then divided by
 *   shift[s] - dg[i] (shift: device [nseg]), a denominator below 1e-8 in magnitude
 *   replaced by 1e-8 (the Davidson diagonal preconditioner).  y must not overlap A1, A2
 *   or dg.
 * Errors: SCI_ERR_ARG for k out of range, NULL operands or lda below the total rows. */
typedef struct sci_seg sci_seg;
int sci_seg_create(sci_seg **out, int device, int nseg, const int64_t *offsets, int kmax, void *cuda_stream);
int sci_seg_destroy(sci_seg *s);
int sci_seg_tn(sci_seg *s, int k, const double *A, int64_t lda, const double *t, double *out);
int sci_seg_nn(sci_seg *s, double *y, const double *beta, int k1, const double *A1, int64_t lda1,
               const double *c1, double alpha1, int k2, const double *A2, int64_t lda2,
               const double *c2, double alpha2, const double *dg, const double *shift);
const char *sci_seg_last_error(const sci_seg *s);

/* Eigenpairs of nb real symmetric n x n matrices (the projected matrices of the solvers
 * above), one CTA each: cyclic Jacobi with the parallel round-robin ordering (Golub and
 * Van Loan, Matrix Computations, Sec. 8.5).  Device pointers, asynchronous on
 * cuda_stream (NULL: the legacy default stream).
 *   A: matrix b at A + b * strideA, row-major with leading dimension lda; both triangles
 *      are read and (a_ij + a_ji) / 2 is used.  Not modified.
 *   w: eigenvalues of matrix b, ascending, at w + b * stridew.
 *   V: eigenvectors as columns (V[i][j] = component i of eigenvector j, same order as w),
 *      matrix b at V + b * strideV with leading dimension ldv.
 *   Sweeps stop when the off-diagonal sum of squares is below 1e-30 of the total, or
 *   after max_sweeps; not_converged (device int, or NULL) is then incremented per matrix.
 * 1 <= n <= 64 (n = 0 or nb = 0: nothing to do).  Errors: SCI_ERR_ARG for sizes, strides
 * or NULL pointers; SCI_ERR_CUDA. */
int sci_syev_batched(int device, int nb, int n, const double *A, int64_t lda, int64_t strideA,
                     double *w, int64_t stridew, double *V, int64_t ldv, int64_t strideV,
                     int max_sweeps, int *not_converged, void *cuda_stream);

/* Measured FMA throughput of the GPU, for the benchmark's pipe fractions (the paper has
 * no counterpart: its timings are CPU wall times).  prec SCI_PREC_F64 times FP64 FMAs,
 * SCI_PREC_F32_STORE_F64_ACC FP32 FMAs: 8 CTAs of 256 threads per SM, 8 independent FMA
 * chains of `iters` (>= 8) steps per thread, one untimed warm-up launch, then one launch
 * timed with CUDA events on cuda_stream (NULL: the legacy default stream).
 * *fma_per_s receives the FMAs per second (one FMA = 2 flops).  Synchronous; allocates
 * and frees a small output buffer.  Errors: SCI_ERR_ARG, SCI_ERR_NOMEM, SCI_ERR_CUDA. */
int sci_peak_fma(int device, int prec, int iters, void *cuda_stream, double *fma_per_s);

/* Wait for the context stream and return the device status word (SCI_OK or the first
 * device-side error code). */
int sci_sync_status(sci_ctx *ctx);

/* Message of the last error of this context ("" if none).  Valid until the next call. */
const char *sci_last_error(const sci_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SCI_H */
