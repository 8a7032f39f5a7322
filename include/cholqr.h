/*
 * cholqr.h -- C ABI of libcholqr: shifted Cholesky QR (sCholQR3 with the
 * recomputed shift) and the Cholesky-QR updating scheme on one GB300 GPU.
 *
 * Paper: M. Bindhak, A. J. R. Pelling, J. Saak, "Towards an Efficient Shifted
 * Cholesky QR for Applications in Model Order Reduction using pyMOR",
 * arXiv 2507.07788.
 *
 * Conventions for every entry point
 *   - Matrices are FP64 and column-major: element (i, j) of M with leading
 *     dimension ld is M[i + j*ld].  A "vector" of the paper is one column.
 *   - Pointers named A, Q, R, A_in are DEVICE pointers (memory of the current
 *     CUDA device) unless the function name ends in _host.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is queued on it; each call synchronises that stream once
 *     at its end to read the status and fill `info`, so on return the outputs
 *     are complete.
 *   - The library allocates its own scratch memory stream-ordered
 *     (cudaMallocAsync on `stream`) and frees it before returning; basis
 *     handles own their storage until basis_free.
 *   - Errors are reported by the return value; no function aborts the
 *     process.  On an error return (< 0) output buffers hold unspecified data,
 *     except where stated.
 *   - Calls on different streams may run concurrently; calls sharing a basis
 *     handle must be serialised by the caller.
 */
#ifndef CHOLQR_H
#define CHOLQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  CQR_NOT_CONVERGED still returns a valid factorisation
 * (Q R = A to working accuracy) whose orthogonality did not reach `tol`
 * within `max_iter` passes (the paper caps iterations at 10, Sec. 4.1). */
typedef enum cqr_status {
  CQR_OK = 0,
  CQR_NOT_CONVERGED = 1,
  CQR_ERR_INVALID = -1,   /* bad argument (sizes, leading dims, NULL, opts) */
  CQR_ERR_BREAKDOWN = -2, /* Cholesky failed after every permitted shift */
  CQR_ERR_OOM = -3,       /* device allocation failed */
  CQR_ERR_CAPACITY = -4,  /* basis_append: q + p > n_max */
  CQR_ERR_CUDA = -5,      /* a CUDA runtime call or launch failed */
  CQR_ERR_TIMEOUT = -6,   /* reserved for waits that give up */
  CQR_ERR_REDUCE = -7     /* cholqr_factor_sharded: the reducer reported a failure */
} cqr_status;

/* Shift policy of the factorisation (Alg. 1, Sec. 2.1, and Sec. 4.1 item 2):
 *   CQR_SHIFT_SCHOLQR3      first pass always shifted (sCholQR3), later
 *                           passes unshifted; a later breakdown recomputes
 *                           the shift from the current Gramian (Alg. 1).
 *                           Default.
 *   CQR_SHIFT_ON_BREAKDOWN  Alg. 1 exactly as printed.
 *   CQR_SHIFT_NONE          no shift at all (CholQR / CholQR2); a breakdown
 *                           returns CQR_ERR_BREAKDOWN.
 *   CQR_SHIFT_SCHOLQR3_STRICT  first pass shifted, a later breakdown returns
 *                           CQR_ERR_BREAKDOWN (the sCholQR3 of Fukaya et al.
 *                           that Fig. 1 compares against).
 *   CQR_SHIFT_ISCHOLQR      no first shift; the shift is computed once, from
 *                           the Gramian of the first breakdown, and reused at
 *                           every later breakdown (isCholQR, Fig. 1).  Sized
 *                           from ||A||^2, that shift is too large for later
 *                           Gramians when ||A|| >> 1 (Sec. 2.1): from
 *                           kappa ~ 1e16 the policy fails for such A.
 * The last two are comparison policies for Fig. 1; the factorisation's
 * other rules (stop test, x10 escalation of a failing shift) are shared. */
enum {
  CQR_SHIFT_SCHOLQR3 = 0,
  CQR_SHIFT_ON_BREAKDOWN = 1,
  CQR_SHIFT_NONE = 2,
  CQR_SHIFT_SCHOLQR3_STRICT = 3,
  CQR_SHIFT_ISCHOLQR = 4
};

/* Stopping rule: ||X - I||_F < tol (Sec. 4.1, default tol = 1e-13), or the
 * literal u*sqrt(n) of Alg. 1 / Alg. 2. */
enum { CQR_STOP_FROB_TOL = 0, CQR_STOP_U_SQRT_N = 1 };

/* Arithmetic of the row-sweeping kernels.  CQR_PREC_FP64: every step in FP64.
 * CQR_PREC_MIXED (cholqr_factor only): the Gramian of the first (shifted)
 * pass is formed at reduced precision and the first shift is sized for its
 * error bound, in the form of Alg. 1; the norm estimate, Cholesky,
 * solves and all later passes stay FP64.  With the digit kernels (n <= 128,
 * emulation not CQR_EMU_OFF, no reducer) that Gramian keeps 5 balanced
 * base-256 digits (40 bits relative to each column's largest binary
 * exponent E_j) and the digit orders <= 4 on the tensor cores, and
 *   sigma = 11 (m e sum_j 4^(E_j - 1022) + n (n + 1 + G + 9) u ||X||),
 * e = 2.0324e-12 (a row's error bound in units of 2^(E_i + E_j - 2044)),
 * G = the kernel's partial count, u = 2^-53.  Otherwise (emulation off, wider
 * n, or cholqr_factor_sharded, whose shift must not depend on the rank's
 * rows) it is formed from inputs truncated to FP32 with FP32 products and
 *   sigma = 11 (n (2 2^-23 + 66 2^-24) + n (n + 1) u) ||X||. */
enum { CQR_PREC_FP64 = 0, CQR_PREC_MIXED = 1 };

typedef struct cqr_opts {
  double tol;              /* stop when ||X - I||_F < tol            (1e-13) */
  int32_t max_iter;        /* passes / outer iterations cap              (10) */
  int32_t min_iter;        /* minimum passes of cholqr_factor             (0) */
  int32_t update_min_iter; /* minimum outer iterations of basis_append:
                              2 = the projection is applied twice       (2) */
  int32_t precision;       /* CQR_PREC_*                         (FP64) */
  int32_t shift_policy;    /* CQR_SHIFT_*                    (SCHOLQR3) */
  int32_t stop_rule;       /* CQR_STOP_*                     (FROB_TOL) */
  int32_t max_escalations; /* cap on x10 shift escalations           (40) */
  int32_t emulation;       /* CQR_EMU_*                          (AUTO) */
} cqr_opts;

/* How the FP64 products of a pass are formed.  CQR_EMU_AUTO: on the tensor
 * cores with the Ozaki splitting scheme (exact digit products, each entry
 * rounded to FP64 once) where the kernels support it: the Gramians of
 * cholqr_factor and cholqr_gram for n <= 128 and the factorisation's
 * triangular solve for 17 <= n <= 128; for basis_append and cholqr_pn on
 * more than 262144 rows, an append to an empty basis (the factorisation's
 * pipeline), the cross Gramian of appends of 32..64 columns, and the cross
 * Gramian and projection of appends of <= 16 columns to a basis with a digit
 * cache (basis_enable_digit_cache; cholqr_pn keeps one for panels of <= 16
 * columns; q <= 256 for the projection); FP64 CUDA cores elsewhere.  For
 * 33 <= n <= 64 the Gramian of cholqr_factor (and of an append to an empty
 * basis) and of cholqr_gram runs on a tcgen05 kernel with TMEM accumulators
 * and TMA-loaded tiles when the block is 16-byte aligned with an even
 * leading dimension; the other kernels issue warp-level mma.sync.
 * CQR_EMU_OFF: FP64 CUDA cores everywhere.  CQR_EMU_TCGEN05: as AUTO, with
 * the tcgen05 Gramian from n = 17 and the factorisation's solve for
 * 17 <= n <= 64 on a tcgen05 kernel too (one row chunk per pass); the same
 * exact digit products. */
enum { CQR_EMU_AUTO = 0, CQR_EMU_OFF = 1, CQR_EMU_TCGEN05 = 2 };

/* Per-call report.  orth_frob is ||X - I||_F of the last Gramian formed
 * (for basis_append: of the projected Gramian Q^T Q - B~^T B~), proj_frob is
 * ||B~||_F = ||Q_in^T Q||_F after the last iteration (0 for factor). */
typedef struct cqr_info {
  int32_t iters;         /* passes (factor) or outer iterations (append) */
  int32_t chol_attempts; /* Cholesky factorisations attempted */
  int32_t shifts;        /* shifts computed from ||X|| */
  int32_t escalations;   /* x10 shift escalations */
  double sigma_first;    /* first shift applied (0 if none) */
  double sigma_last;     /* last shift applied (0 if none) */
  double orth_frob;
  double proj_frob;
} cqr_info;

/* Largest Gramian width handled by the kernels: n of cholqr_factor and p of
 * basis_append must not exceed it.  Basis capacity (q + p) up to
 * CQR_MAX_BASIS.  Above 128 columns the Gramian of cholqr_factor,
 * cholqr_gram and of an append to an empty basis is formed by 64 x 64 block
 * pairs on the tensor cores (exact digit products, unless
 * opts->emulation is CQR_EMU_OFF: then, and for appends to a non-empty
 * basis, the FP64 row sweep, split over several sweeps of its entries); the
 * triangular solve Q = Y R~^{-1} is an exact digit product with the
 * contraction in blocks of 64 (the FP64 row substitution under the same
 * exceptions); the control step keeps its n x n working storage in global
 * memory and shares each Cholesky among one CTA per SM (a cooperative
 * launch, whose grid barriers wait at most 5 s each: a wait that runs out
 * ends the call with CQR_ERR_TIMEOUT).  The cooperative steps of all calls
 * on a device run on one internal stream, ordered after the caller's
 * stream by events, so concurrent wide calls take turns there. */
#define CQR_MAX_N 512
#define CQR_MAX_BASIS 1024

/* Fills *o with the defaults listed above.  o must not be NULL. */
void cqr_default_opts(cqr_opts *o);

/* Static string naming a status code (never NULL). */
const char *cqr_status_string(int status);

/*
 * cholqr_factor -- QR factorisation A = Q R of a tall-skinny m x n block by
 * iterated shifted Cholesky QR: Alg. 1 (rsCholQR, Sec. 2.1) with the shift of
 * Alg. 1, sigma = max{11 (m n + n (n+1)) u ||X||, 2u}, and the
 * sCholQR3 first-pass shift named in Sec. 4.1 (opts->shift_policy).
 *
 *   opts      host pointer, may be NULL (defaults).
 *   m, n      1 <= n <= CQR_MAX_N, m >= n.
 *   A, lda    device, m x n input, lda >= m.  Read only, unless it aliases Q.
 *   Q, ldq    device, m x n output, ldq >= m.  Q may be A (in place) when
 *             ldq == lda; otherwise the two must not overlap.
 *   R, ldr    device, n x n output, ldr >= n; upper triangular with positive
 *             diagonal, zeros below it.
 *   info      host pointer, may be NULL.
 *   stream    cudaStream_t as void*.
 * Returns CQR_OK, CQR_NOT_CONVERGED (valid Q, R), or an error code.
 */
cqr_status cholqr_factor(const cqr_opts *opts, int64_t m, int64_t n, const double *A,
                         int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr,
                         cqr_info *info, void *stream);

/*
 * cholqr_gram -- the Gramian X = A^T A of Alg. 1, formed by the same
 * row sweep and fixed-order reduction as the factorisation's first pass
 * (tensor-core digit arithmetic for n <= 128 unless opts->emulation is
 * CQR_EMU_OFF; FP64 CUDA cores otherwise).  With opts->precision =
 * CQR_PREC_MIXED it is the first-pass Gramian of the mixed factorisation
 * (5-digit on the tensor cores, or FP32 with CQR_EMU_OFF; see CQR_PREC_MIXED).
 *   A, lda    device, m x n, lda >= m (read only).
 *   X, ldx    device, n x n output (both triangles), ldx >= n.
 *   1 <= n <= CQR_MAX_N, m >= 1.
 */
cqr_status cholqr_gram(const cqr_opts *opts, int64_t m, int64_t n, const double *A, int64_t lda,
                       double *X, int64_t ldx, void *stream);

/*
 * cholqr_factor_host -- the same factorisation on HOST buffers: A is copied
 * to the device and factored exactly as cholqr_factor factors it (Q and R
 * agree bit for bit).  Where the tensor-core path runs (n <= 128,
 * CQR_PREC_FP64, emulation CQR_EMU_AUTO) and Q is page-locked
 * (cudaHostAlloc / cudaHostRegister), the pass expected to be the last
 * (its input has ||Q^T Q - I||_F < 1/2) writes each solved row chunk of Q
 * straight into the host Q while the next chunks run, and only chunks that
 * missed the final pass are copied after the stop.  Otherwise Q is copied
 * whole after the stop.
 *   A, lda    host, m x n, lda >= m (read only; pinned for full bandwidth).
 *   Q, ldq    host, m x n output, ldq >= m; must not overlap A (else
 *             CQR_ERR_INVALID).  Its contents are undefined while the
 *             call runs and after an error.
 *   R, ldr    host, n x n output, ldr >= n.
 * The device copies are stream-ordered scratch freed before return; the call
 * returns after the stream has drained.  Status as cholqr_factor.
 */
cqr_status cholqr_factor_host(const cqr_opts *opts, int64_t m, int64_t n, const double *A,
                              int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr,
                              cqr_info *info, void *stream);

/*
 * cholqr_factor_noalloc -- cholqr_factor for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a deployment variant.
 * Some callers cannot call cudaMalloc: processes that have already handed all
 * device memory to their own allocator (a framework caching allocator, or a
 * serving loop that admits work against a fixed HBM budget), where a
 * library-side allocation could fail or fragment their pool, and
 * latency-critical loops that must never pay for, or risk the failure of, an
 * allocation inside a call.  This entry point calls no allocating routine:
 * all of its device scratch lives in one fixed 8 MiB array compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits, and the status is read back into host stack memory.
 *   Arguments, layout and results are those of cholqr_factor, but it always
 *   runs the FP64 CUDA-core path: the fused row sweep (triangular solve +
 *   Gramian), its reduction and the control kernel, exactly as cholqr_factor
 *   does with opts->emulation = CQR_EMU_OFF (same kernels, same launch
 *   geometry, so Q and R are bitwise equal to that call's).  It is therefore
 *   slower than cholqr_factor's default tensor-core path for n >= 17.
 *   opts->emulation is ignored; opts->precision = CQR_PREC_MIXED returns
 *   CQR_ERR_INVALID.  Limit: n <= 64; larger n returns CQR_ERR_CAPACITY
 *   without touching the device.
 *   A, Q and R must be memory of the current device (else CQR_ERR_INVALID).
 *   Each call looks up the array's device address with the current device
 *   current.  All calls share the array and it keeps the last call's
 *   contents; each call clears what must start at zero.  Calls whose work
 *   overlaps on the GPU (for example on two streams at once) race on the
 *   array and must be serialised by the caller.
 */
cqr_status cholqr_factor_noalloc(const cqr_opts *opts, int64_t m, int64_t n, const double *A,
                                 int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr,
                                 cqr_info *info, void *stream);

/*
 * Row-sharded factorisation (communication-avoiding Cholesky QR, Sec. 1):
 * the m rows of A are split into contiguous blocks, one per rank (one GPU or
 * one process each).  Each rank forms the partial Gramian of its own rows;
 * the partials are exchanged through the caller's reducer and summed in
 * rank order 0, 1, ..., world-1 by a library kernel, so every rank holds the
 * bitwise same Gramian and takes the same shift, breakdown and stop
 * decisions; the triangular solves are row-local.  One exchange of n x n
 * doubles per pass (and one for the first Gramian).
 *
 * cqr_reducer: caller-owned exchange buffers and callback.
 *   world, rank   number of ranks and this rank (0 <= rank < world).
 *   send          device, at least `capacity` doubles: the library writes its
 *                 local block (count doubles) there before each call.
 *   recv          device, at least world * capacity doubles: on return of
 *                 allgather (or, for work queued on `stream`, when that work
 *                 completes) recv[r * count .. (r + 1) * count) must hold rank
 *                 r's block, on every rank.
 *   capacity      doubles available in send (n * n is enough).
 *   allgather     called by the library on every rank the same number of
 *                 times, in the same order; its work must be ordered on
 *                 `stream` (queued there, or complete before it returns).
 *                 Returns 0 on success; any other value makes the call stop
 *                 and return CQR_ERR_REDUCE.
 *   ctx           passed through to allgather.
 */
typedef struct cqr_reducer {
  int32_t world;
  int32_t rank;
  double *send;
  double *recv;
  int64_t capacity;
  int (*allgather)(void *ctx, int64_t count, void *stream);
  void *ctx;
} cqr_reducer;

/*
 * cholqr_factor_sharded -- cholqr_factor (Alg. 1 with the sCholQR3 first
 * shift, Sec. 2.1 and 4.1) on this rank's row block of a matrix with m_total
 * rows.  The shift uses m_total (Alg. 1).  Every rank must call it
 * with the same opts, n and m_total; the results are this rank's rows of Q
 * and the full R (the same on every rank).
 *   m_local   rows of this rank's block, 1 <= m_local <= m_total, m_total >= n.
 *   A, Q      device, m_local x n blocks (lda, ldq >= m_local), as in
 *             cholqr_factor (Q may be A).
 *   R         device, n x n (ldr >= n).
 *   red       reducer (see above), not NULL; capacity >= n * n.
 * Returns the status of cholqr_factor, or CQR_ERR_REDUCE if a reducer call
 * failed (outputs unspecified; every rank's later reducer calls are skipped,
 * so peers must detect the failure through their own reducer).
 */
cqr_status cholqr_factor_sharded(const cqr_opts *opts, int64_t m_local, int64_t m_total, int64_t n,
                                 const double *A, int64_t lda, double *Q, int64_t ldq, double *R,
                                 int64_t ldr, const cqr_reducer *red, cqr_info *info, void *stream);

/*
 * cholqr_pn -- pnCholQR, Alg. 3 (Sec. 2.3): QR of A (m x n) by r column
 * panels, the first factored and each later one appended to the growing
 * basis by the Cholesky-QR update (Alg. 2, as basis_append).  Panel k has
 * n/r columns, plus one for k < n mod r.
 *   opts      host pointer, may be NULL (defaults; update_min_iter applies to
 *             every panel).
 *   m, n, r   1 <= r <= n <= CQR_MAX_BASIS, m >= n, every panel at most
 *             CQR_MAX_N columns (ceil(n/r) <= CQR_MAX_N).
 *   A, lda    device, m x n, lda >= m, read only; must not overlap Q.
 *   Q, ldq    device, m x n output, ldq >= m.
 *   R, ldr    device, n x n output, ldr >= n; upper triangular (the
 *             strictly lower part is set to zero).
 *   info      host pointer, may be NULL: iters, chol_attempts, shifts and
 *             escalations summed over the panels; sigma_first = the first
 *             nonzero shift, sigma_last = the last; orth_frob and proj_frob of
 *             the last panel.
 * With r > 1 panels of at most 16 columns on more than 262144 rows (and
 * CQR_EMU_AUTO), the call keeps a stream-ordered digit cache of the columns
 * already factored (14 bytes per entry of Q, freed before return), as a
 * basis with basis_enable_digit_cache does; without room for it the panels
 * take the FP64 path.
 * Returns the first error of a panel (later panels are not run), else
 * CQR_NOT_CONVERGED if any panel did not converge, else CQR_OK.
 */
cqr_status cholqr_pn(const cqr_opts *opts, int64_t m, int64_t n, int64_t r, const double *A,
                     int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr, cqr_info *info,
                     void *stream);

/* Opaque growing orthonormal basis (Q_in m x q, R_in q x q) of Sec. 2.2. */
typedef struct cqr_basis cqr_basis;

/*
 * basis_create -- allocate an empty basis (q = 0) for vectors of length m
 * with room for n_max columns: device Q (m x n_max, leading dimension m
 * rounded up to even) and R (n_max x n_max), both owned by the handle.
 *   1 <= n_max <= CQR_MAX_BASIS, m >= 1.  opts may be NULL (defaults); it is
 *   copied.  *out receives the handle (NULL on error).
 */
cqr_status basis_create(int64_t m, int64_t n_max, const cqr_opts *opts, void *stream,
                        cqr_basis **out);

/*
 * basis_append -- the Cholesky-QR update, Alg. 2 (cholQRUpdate, Sec. 2.2):
 * given the basis Q_in R_in = A_prev (m x q) and new columns A_in (m x p),
 * extend it to [Q_in Q] and [[R_in, B], [0, R]] with
 * [Q_in Q][[R_in, B], [0, R]] = [A_prev A_in] (Proposition 2.1).  The shift
 * loop is Alg. 2: sigma starts at 0, then
 * 11 (m q + q (q+1)) u ||X|| (Alg. 1's formula with p when q = 0), then x10,
 * floored at 2u.  At least opts->update_min_iter outer iterations are made.
 *   p         1 <= p <= CQR_MAX_N, q + p <= n_max (else CQR_ERR_CAPACITY).
 *   A_in, lda device, m x p, lda >= m, read only and caller-owned; it must not
 *             overlap the basis storage.
 * On CQR_OK / CQR_NOT_CONVERGED the basis grows by p columns; on an error the
 * basis keeps its previous q columns and R_in unchanged.
 */
cqr_status basis_append(cqr_basis *b, int64_t p, const double *A_in, int64_t lda,
                        cqr_info *info, void *stream);

/*
 * basis_enable_digit_cache -- keep a digit copy of the basis columns on the
 * device (7 bf16 digits per entry, 14 bytes: 1.75x the size of Q) so that
 * later appends of p <= 16 columns to a basis of more than 262144 rows form
 * their cross Gramian [Q_in A_in]^T A_in (Alg. 2) and, while
 * the basis has at most 256 columns, the projection Q_in B~ of the solve
 * (Alg. 2) on the tensor cores from the cached digits instead of
 * FP64 products.  Each column is written as sign * V * 2^(E_k - 1078) with
 * E_k its largest biased exponent and V < 2^56 in 7 balanced base-256
 * digits; the cache fills for the present columns now and for new ones at
 * each successful append (and, in the serving runtime, when a factor
 * request replaces the columns).  The result follows the same tolerances as
 * without the cache (the digit products are exact; each entry is rounded
 * once).
 *   Returns CQR_OK (also if the cache exists), CQR_ERR_OOM (the basis is
 *   unchanged and appends keep the FP64 path), or CQR_ERR_CUDA.
 */
cqr_status basis_enable_digit_cache(cqr_basis *b, void *stream);

/* basis_free -- release the handle and its device storage (NULL is a no-op).
 * The caller must make sure no queued work still uses the basis. */
cqr_status basis_free(cqr_basis *b);

/* Accessors.  basis_q / basis_r return DEVICE pointers owned by the basis
 * (valid until basis_free) and the leading dimension.  Q has basis_cols(b)
 * valid columns; R is upper triangular in its leading q x q block. */
int64_t basis_cols(const cqr_basis *b);
int64_t basis_rows(const cqr_basis *b);
int64_t basis_capacity(const cqr_basis *b);
cqr_status basis_q(const cqr_basis *b, const double **Q, int64_t *ldq);
cqr_status basis_r(const cqr_basis *b, const double **R, int64_t *ldr);

/*
 * Serving runtime (no counterpart in the paper; it serves the paper's two
 * modes of use, M1 = full factorisation and M2 = repeated updates, Sec. 1).
 * A server keeps many bases resident on the device and executes factor and
 * append requests with continuous batching:
 *   - requests are admitted in arrival order when their basis is idle, their
 *     transient device memory fits `hbm_budget_bytes` and an executor is free;
 *     requests on one basis run in submission order;
 *   - factor requests and large appends run on `slots` worker streams
 *     concurrently; appends of at most 32 columns to bases of at most
 *     `small_rows` rows that keep no digit cache are batched: one
 *     persistent launch per step covers every append of the batch, replayed
 *     from captured CUDA graphs;
 *   - a factor request replaces its basis's columns (and refills the
 *     basis's digit cache, if it keeps one);
 *   - each result is bitwise the same alone and in the mix (a batched problem
 *     uses the same per-CTA work and reduction order as alone).
 * Timestamps are seconds on the server's steady clock (cqr_server_now).
 */
typedef struct cqr_server cqr_server;

typedef struct cqr_server_opts {
  int32_t slots;            /* worker streams for factors / large appends (4) */
  int32_t batch_max;        /* appends per batched launch, 0 = no batching (16) */
  int64_t hbm_budget_bytes; /* transient device memory of admitted requests (8 GiB) */
  int64_t small_rows;       /* appends to bases with m <= small_rows are batched (262144) */
} cqr_server_opts;

typedef struct cqr_request_result {
  int32_t status;     /* cqr_status of the request */
  int32_t kind;       /* 0 factor, 1 append */
  int32_t batched;    /* 1 if it ran in a batched launch */
  int32_t batch_size; /* problems in that launch */
  double t_submit;    /* arrival (submit) time */
  double t_start;     /* admission time */
  double t_done;      /* completion time */
  cqr_info info;
} cqr_request_result;

void cqr_server_default_opts(cqr_server_opts *o);
/* Creates a server on the current device (allocates the batch workspace,
 * captures its graphs, starts the worker and batcher threads). */
cqr_status cqr_server_create(const cqr_server_opts *opts, cqr_server **out);
/* Factor request (M1): replaces basis b by the QR of A (device, b->m x n,
 * lda >= m, caller-owned and unchanged until the request completes).
 * n <= min(CQR_MAX_N, capacity).  *ticket identifies the request. */
cqr_status cqr_server_submit_factor(cqr_server *s, cqr_basis *b, int64_t n, const double *A,
                                    int64_t lda, const cqr_opts *opts, uint64_t *ticket);
/* Append request (M2): basis_append(b, p, A_in) when admitted.  A_in stays
 * caller-owned and unchanged until completion; it must not overlap the
 * basis storage (else CQR_ERR_INVALID at submission).  An append past the
 * basis capacity completes with CQR_ERR_CAPACITY. */
cqr_status cqr_server_submit_append(cqr_server *s, cqr_basis *b, int64_t p, const double *A_in,
                                    int64_t lda, uint64_t *ticket);
/* Blocks until the request completes and copies its result (out may be NULL). */
cqr_status cqr_server_wait(cqr_server *s, uint64_t ticket, cqr_request_result *out);
/* Blocks until every submitted request has completed. */
cqr_status cqr_server_drain(cqr_server *s);
/* Seconds since the server was created (the clock of the result stamps). */
double cqr_server_now(const cqr_server *s);
/* Drains, stops the threads and frees the server (not the bases). */
cqr_status cqr_server_destroy(cqr_server *s);

/*
 * Instrumentation (no counterpart in the paper).  When enabled, every call
 * brackets each row sweep (the Gramian sweep and each solve + Gramian pass)
 * with CUDA events on the caller's stream, and each FP64 row-solve kernel
 * and each tensor-core Gramian kernel with events on the stream it is
 * launched on; at the call's final synchronisation the elapsed times of the
 * launches that did work, with their algorithmic FLOPs and bytes, are added
 * to process-wide counters.  All kernel launches of the library are counted whether or not
 * timing is enabled.  Counters are protected by a mutex; reset clears them.
 */
typedef struct cqr_timing {
  int64_t kernel_launches;   /* every kernel launch of the library */
  int64_t sweep_launches;    /* timed row sweeps that did work */
  double sweep_ms;           /* their summed event time */
  double sweep_flops;        /* their algorithmic FLOPs */
  double sweep_bytes;        /* their algorithmic HBM bytes (read + write) */
  int64_t fused_launches;    /* of those, fused solve + Gramian sweeps */
  double fused_ms;
  double fused_flops;
  double fused_bytes;
  int64_t solve_launches;    /* FP64 row-solve kernels of the pass pipeline */
  double solve_ms;
  double solve_flops;
  double solve_bytes;
  int64_t gram_launches;     /* tensor-core Gramian kernels (each timed alone) */
  double gram_ms;
  double gram_flops;
  double gram_bytes;
  int64_t tsolve_launches;   /* tensor-core solve kernels Q = Y R~^{-1} */
  double tsolve_ms;
  double tsolve_flops;       /* FP64-equivalent FLOPs (n^2 per row) */
  double tsolve_bytes;
  double tsolve_tc_flops;    /* bf16 digit-product FLOPs on the tensor pipe */
} cqr_timing;

/* Enables (1) or disables (0) event timing of the row sweeps. */
cqr_status cqr_timing_enable(int enable);
/* Copies the counters to *out (host pointer, not NULL). */
cqr_status cqr_timing_read(cqr_timing *out);
/* Clears the counters. */
void cqr_timing_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* CHOLQR_H */
