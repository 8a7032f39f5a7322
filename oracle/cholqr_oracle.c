/*
 * Plain FP64 CPU oracle for shifted Cholesky QR and the Cholesky-QR update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Everything is written as the textbook definition or as the paper's
 * algorithm step by step, in IEEE double precision, with sums taken in index
 * order.  Compile with -ffp-contract=off so that no multiply-add is fused
 * behind our back (the same results on x86-64 and aarch64).
 *
 * Matrices are column-major: element (i, j) of M with leading dimension ld
 * is M[i + j*ld].
 *
 * Paper: Bindhak, Pelling, Saak, "Towards an Efficient Shifted Cholesky QR for
 * Applications in Model Order Reduction using pyMOR", arXiv 2507.07788.
 *   Alg. 1  rsCholQR (iterated Cholesky QR with shift recomputation), Sec. 2.1
 *   Alg. 2  cholQRUpdate (Cholesky-QR updating scheme), Sec. 2.2
 *   Alg. 3  pnCholQR (panel scheme), Sec. 2.3
 *   Sec. 4.1 stopping rule ||I - Q^T Q||_F <= 1e-13, at most 10 iterations,
 *            metrics LOO / RRR / RCR, test matrices A = U Sigma V^T.
 *
 * Parity pins: every function here is checked in tests/test_oracle_pins.py
 * against something other than itself (LAPACK through numpy, closed forms,
 * brute force, Proposition 2.1, the Fig. 1 robustness claims).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "cholqr_oracle.h"

#define AT(M, i, j, ld) ((M)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)])

/* Unit roundoff of IEEE binary64, 2^-53 (Sec. 4.1: u ~ 1.11e-16). */
static const double ORC_U = 1.1102230246251565404236316680908203125e-16;

/* ------------------------------------------------------------------------- */
/* Basic dense kernels, written as their definitions.                        */
/* ------------------------------------------------------------------------- */

/* X = A^T A (n x n, both triangles), A m x n.  Definition of the Gramian
 * (Alg. 1): X_ij = sum_k A_ki A_kj, k ascending. */
void orc_gram(int64_t m, int64_t n, const double *A, int64_t lda, double *X,
              int64_t ldx) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i <= j; ++i) {
      double s = 0.0;
      for (int64_t k = 0; k < m; ++k) s += AT(A, k, i, lda) * AT(A, k, j, lda);
      AT(X, i, j, ldx) = s;
      AT(X, j, i, ldx) = s;
    }
}

/* C = A^T B (p x q), A m x p, B m x q.  Used for B~ = Q_in^T Q (Alg. 2). */
void orc_gemm_tn(int64_t m, int64_t p, int64_t q, const double *A,
                 int64_t lda, const double *B, int64_t ldb, double *C,
                 int64_t ldc) {
  for (int64_t j = 0; j < q; ++j)
    for (int64_t i = 0; i < p; ++i) {
      double s = 0.0;
      for (int64_t k = 0; k < m; ++k) s += AT(A, k, i, lda) * AT(B, k, j, ldb);
      AT(C, i, j, ldc) = s;
    }
}

/* Cholesky factorisation R^T R = X + sigma I, R upper triangular (the
 * "chol" of Alg. 1 and Alg. 2).  Row-oriented textbook
 * algorithm reading only the upper triangle of X.
 * Breakdown: a pivot d_j = X_jj + sigma - sum_{k<j} R_kj^2 that is not
 * strictly positive (or not finite).  Returns 0 on success, else j+1 for the
 * first failing pivot.  The strictly lower part of R is set to zero. */
int orc_chol(int64_t n, const double *X, int64_t ldx, double sigma, double *R,
             int64_t ldr) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(R, i, j, ldr) = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double d = AT(X, j, j, ldx) + sigma;
    for (int64_t k = 0; k < j; ++k) d -= AT(R, k, j, ldr) * AT(R, k, j, ldr);
    if (!(d > 0.0) || !isfinite(d)) return (int)(j + 1);
    double rjj = sqrt(d);
    AT(R, j, j, ldr) = rjj;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = AT(X, j, i, ldx);
      for (int64_t k = 0; k < j; ++k) s -= AT(R, k, j, ldr) * AT(R, k, i, ldr);
      AT(R, j, i, ldr) = s / rjj;
    }
  }
  return 0;
}

/* Q = A R^{-1} for upper triangular R, one row at a time by forward
 * substitution on R^T q^T = a^T (Alg. 1, Alg. 2).  Q may
 * alias A: each row is read before it is overwritten. */
void orc_trsm_runn(int64_t m, int64_t n, const double *A, int64_t lda,
                   const double *R, int64_t ldr, double *Q, int64_t ldq) {
  for (int64_t r = 0; r < m; ++r)
    for (int64_t j = 0; j < n; ++j) {
      double s = AT(A, r, j, lda);
      for (int64_t k = 0; k < j; ++k) s -= AT(Q, r, k, ldq) * AT(R, k, j, ldr);
      AT(Q, r, j, ldq) = s / AT(R, j, j, ldr);
    }
}

/* C = T R for upper triangular T (n x n) and R (n x n): the R <- R~ R of
 * Alg. 1 / Alg. 2.  C must not alias T or R. */
void orc_trmm_upper(int64_t n, const double *T, int64_t ldt, const double *R,
                    int64_t ldr, double *C, int64_t ldc) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t k = i; k <= j; ++k) s += AT(T, i, k, ldt) * AT(R, k, j, ldr);
      AT(C, i, j, ldc) = (i <= j) ? s : 0.0;
    }
}

/* ||X - I||_F (Alg. 1, Alg. 2, and the Sec. 4.1 stop rule). */
double orc_frob_minus_identity(int64_t n, const double *X, int64_t ldx) {
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double d = AT(X, i, j, ldx) - (i == j ? 1.0 : 0.0);
      s += d * d;
    }
  return sqrt(s);
}

/* Eigenvalues of a symmetric n x n matrix by the cyclic Jacobi method
 * (Golub & Van Loan, Sec. 8.5): sweeps of plane rotations that zero each
 * off-diagonal entry in row order, until the off-diagonal Frobenius mass is
 * below 1e-300 or below u times the diagonal mass.  w receives the
 * eigenvalues (unsorted).  Returns the number of sweeps. */
int orc_sym_eigvals(int64_t n, const double *X, int64_t ldx, double *w) {
  double *a = (double *)malloc(sizeof(double) * (size_t)(n * n + 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) a[i + j * n] = AT(X, i, j, ldx);
  int sweep = 0;
  for (; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) {
        if (i == j)
          diag += a[i + j * n] * a[i + j * n];
        else
          off += a[i + j * n] * a[i + j * n];
      }
    if (off <= 1e-300 || off <= ORC_U * ORC_U * diag) break;
    for (int64_t p = 0; p < n - 1; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        double apq = a[p + q * n];
        if (apq == 0.0) continue;
        double app = a[p + p * n], aqq = a[q + q * n];
        /* Symmetric Schur decomposition of the 2x2 block (GVL Alg. 8.5.1). */
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* A <- J^T A J with J = rotation in the (p, q) plane. */
        for (int64_t k = 0; k < n; ++k) {
          double akp = a[k + p * n], akq = a[k + q * n];
          a[k + p * n] = c * akp - s * akq;
          a[k + q * n] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; ++k) {
          double apk = a[p + k * n], aqk = a[q + k * n];
          a[p + k * n] = c * apk - s * aqk;
          a[q + k * n] = s * apk + c * aqk;
        }
        a[p + q * n] = 0.0;
        a[q + p * n] = 0.0;
      }
  }
  for (int64_t i = 0; i < n; ++i) w[i] = a[i + i * n];
  free(a);
  return sweep;
}

/* Spectral norm of a symmetric matrix, max_i |lambda_i|.  This is the
 * ||X|| of Alg. 1 and Alg. 2; the paper estimates it with a
 * Lanczos eigensolver to 1e-2 relative accuracy (App. A, Listing 1), the
 * oracle computes it to full accuracy. */
double orc_sym_norm2(int64_t n, const double *X, int64_t ldx) {
  if (n <= 0) return 0.0;
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  orc_sym_eigvals(n, X, ldx, w);
  double mx = 0.0;
  for (int64_t i = 0; i < n; ++i) mx = fmax(mx, fabs(w[i]));
  free(w);
  return mx;
}

/* Shift of Alg. 1: sigma = max{11 (m n + n (n + 1)) u ||X||, 2u}.
 * The 2u floor is the paper's guard against a vanishing shift (Sec. 2.1). */
double orc_shift(int64_t m, int64_t n, double normX) {
  double c = 11.0 * ((double)m * (double)n + (double)n * ((double)n + 1.0));
  double s = c * ORC_U * normX;
  return fmax(s, 2.0 * ORC_U);
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 (rsCholQR) with the sCholQR3 first-pass shift.                      */
/* ------------------------------------------------------------------------- */

void orc_default_opts(orc_opts *o) {
  o->tol = 1e-13;             /* Sec. 4.1 */
  o->max_iter = 10;           /* Sec. 4.1 */
  o->min_iter = 0;
  o->shift_policy = ORC_SHIFT_SCHOLQR3;
  o->stop_rule = ORC_STOP_FROB_TOL;
  o->max_escalations = 40;
}

static void set_identity(int64_t n, double *M, int64_t ld) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(M, i, j, ld) = (i == j) ? 1.0 : 0.0;
}

static double stop_tol(const orc_opts *o, int64_t n) {
  if (o->stop_rule == ORC_STOP_U_SQRT_N) return ORC_U * sqrt((double)n);
  return o->tol;
}

/*
 * Iterated Cholesky QR, Alg. 1, generalised by a shift policy:
 *   ORC_SHIFT_SCHOLQR3     pass 1 always shifted by sigma(||X||) (the
 *                          sCholQR3 of Fukaya et al. 2020, Alg. 4.2, named
 *                          in Sec. 4.1); later passes unshifted unless the
 *                          Cholesky breaks down, then the shift is recomputed
 *                          from the current X (Alg. 1).
 *   ORC_SHIFT_ON_BREAKDOWN Alg. 1 as printed.
 *   ORC_SHIFT_SCHOLQR3_STRICT  pass 1 shifted, later breakdown = failure
 *                          (Fukaya's sCholQR3, a Fig. 1 comparison system).
 *   ORC_SHIFT_ISCHOLQR     shift computed once from the first X and reused
 *                          on every breakdown (isCholQR, Fukaya Alg. 4.1).
 *   ORC_SHIFT_NONE         no shift; breakdown = failure (CholQR, CholQR2).
 * The loop runs while ||X - I||_F >= tol (Alg. 1; the tolerance of
 * Sec. 4.1) or fewer than min_iter passes were made, for at most max_iter
 * passes.  If a shifted Cholesky still breaks down (Alg. 1 is silent), the
 * shift is multiplied by 10 as in Alg. 2, at most max_escalations
 * times.
 * Returns ORC_OK, ORC_NOT_CONVERGED (valid Q, R; tolerance not met) or
 * ORC_ERR_BREAKDOWN.  Q may alias A.
 */
int orc_cholqr(const orc_opts *o, int64_t m, int64_t n, const double *A,
               int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr,
               orc_info *info) {
  orc_info inf;
  memset(&inf, 0, sizeof(inf));
  double *X = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *Rt = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *Rn = (double *)malloc(sizeof(double) * (size_t)(n * n));
  int status = ORC_OK;
  const double tol = stop_tol(o, n);
  double sigma_once = -1.0; /* isCholQR's single shift */

  /* Q <- A */
  if (Q != A)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < m; ++i) AT(Q, i, j, ldq) = AT(A, i, j, lda);
  /* R <- I */
  set_identity(n, R, ldr);
  /* X <- Q^T Q */
  orc_gram(m, n, Q, ldq, X, n);
  double orth = orc_frob_minus_identity(n, X, n);
  /* A non-finite Gramian (NaN or Inf in A) leaves the loop's stop test
   * undefined; it cannot be factored, so it is reported as a breakdown. */
  if (!isfinite(orth)) status = ORC_ERR_BREAKDOWN;

  int it = 0;
  while (status == ORC_OK && (orth >= tol || it < o->min_iter) && it < o->max_iter) {
    int first = (it == 0);
    double sigma = 0.0;
    int shifted_first = first && (o->shift_policy == ORC_SHIFT_SCHOLQR3 ||
                                  o->shift_policy == ORC_SHIFT_SCHOLQR3_STRICT);
    int rc;
    if (shifted_first) {
      sigma = orc_shift(m, n, orc_sym_norm2(n, X, n));
      inf.shifts++;
      if (inf.shifts == 1) inf.sigma_first = sigma;
      inf.sigma_last = sigma;
      inf.chol_attempts++;
      rc = orc_chol(n, X, n, sigma, Rt, n);
    } else {
      /* try the unshifted Cholesky factorisation */
      inf.chol_attempts++;
      rc = orc_chol(n, X, n, 0.0, Rt, n);
      if (rc != 0) {
        if (o->shift_policy == ORC_SHIFT_NONE ||
            o->shift_policy == ORC_SHIFT_SCHOLQR3_STRICT) {
          status = ORC_ERR_BREAKDOWN;
          break;
        }
        /* recompute the shift from the current X */
        if (o->shift_policy == ORC_SHIFT_ISCHOLQR) {
          if (sigma_once < 0.0) sigma_once = orc_shift(m, n, orc_sym_norm2(n, X, n));
          sigma = sigma_once;
        } else {
          sigma = orc_shift(m, n, orc_sym_norm2(n, X, n));
        }
        inf.shifts++;
        if (inf.shifts == 1) inf.sigma_first = sigma;
        inf.sigma_last = sigma;
        /* shifted Cholesky */
        inf.chol_attempts++;
        rc = orc_chol(n, X, n, sigma, Rt, n);
      }
    }
    /* Shifted factorisation failed as well: escalate by 10 (reading). */
    int esc = 0;
    while (rc != 0 && esc < o->max_escalations) {
      sigma *= 10.0;
      inf.escalations++;
      inf.sigma_last = sigma;
      inf.chol_attempts++;
      rc = orc_chol(n, X, n, sigma, Rt, n);
      esc++;
    }
    if (rc != 0) {
      status = ORC_ERR_BREAKDOWN;
      break;
    }
    /* Q <- Q R~^{-1} */
    orc_trsm_runn(m, n, Q, ldq, Rt, n, Q, ldq);
    /* R <- R~ R */
    orc_trmm_upper(n, Rt, n, R, ldr, Rn, n);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) AT(R, i, j, ldr) = AT(Rn, i, j, n);
    /* X <- Q^T Q */
    orc_gram(m, n, Q, ldq, X, n);
    orth = orc_frob_minus_identity(n, X, n);
    ++it;
    if (!isfinite(orth)) status = ORC_ERR_BREAKDOWN;
  }
  inf.iters = it;
  inf.orth_frob = orth;
  if (status == ORC_OK && orth >= tol) status = ORC_NOT_CONVERGED;
  if (info) *info = inf;
  free(X);
  free(Rt);
  free(Rn);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Alg. 2 (cholQRUpdate).                                                     */
/* ------------------------------------------------------------------------- */

/* Shift of Alg. 2, first attempt: 11 (m q + q (q + 1)) u ||X||, with
 * q the number of existing basis columns.  For q = 0 this is zero; the
 * oracle then uses Alg. 1's formula with the block width p (a reading: with
 * no basis the update is a plain shifted CholQR of the block). */
double orc_update_shift(int64_t m, int64_t q, int64_t p, double normX) {
  if (q == 0) return orc_shift(m, p, normX);
  double c = 11.0 * ((double)m * (double)q + (double)q * ((double)q + 1.0));
  return c * ORC_U * normX;
}

/* X = Q^T Q - Bt^T Bt (Alg. 2); Q m x p, Bt q x p. */
static void update_gram(int64_t m, int64_t q, int64_t p, const double *Q,
                        int64_t ldq, const double *Bt, double *X) {
  orc_gram(m, p, Q, ldq, X, p);
  for (int64_t j = 0; j < p; ++j)
    for (int64_t i = 0; i < p; ++i) {
      double s = 0.0;
      for (int64_t k = 0; k < q; ++k) s += AT(Bt, k, i, q) * AT(Bt, k, j, q);
      AT(X, i, j, p) -= s;
    }
}

/*
 * Alg. 2.  Given Q_in (m x q, orthonormal) and new columns A_in (m x p),
 * computes Q (m x p), B (q x p) and R (p x p) with
 *   [Q_in Q] [[R_in, B], [0, R]] = [Q_in R_in, A_in]  (Proposition 2.1).
 * The loop runs while ||X - I||_F >= tol or fewer than min_iter outer
 * iterations were made, at most max_iter.  The inner shift loop starts at
 * sigma = 0 and follows Alg. 2 (first shift from ||X||, then
 * times 10, floored at 2u), at most max_escalations shifted attempts.
 * Q_out may not alias A_in or Q_in.
 */
int orc_cholqr_update(const orc_opts *o, int64_t m, int64_t q,
                      const double *Qin, int64_t ldqin, int64_t p,
                      const double *Ain, int64_t lda, double *Q, int64_t ldq,
                      double *B, int64_t ldb, double *R, int64_t ldr,
                      orc_info *info) {
  orc_info inf;
  memset(&inf, 0, sizeof(inf));
  int status = ORC_OK;
  const double tol = stop_tol(o, p);
  int64_t qq = q > 0 ? q : 1;
  double *Bt = (double *)calloc((size_t)(qq * p), sizeof(double));
  double *X = (double *)malloc(sizeof(double) * (size_t)(p * p));
  double *Rt = (double *)malloc(sizeof(double) * (size_t)(p * p));
  double *Rn = (double *)malloc(sizeof(double) * (size_t)(p * p));
  double *Bn = (double *)malloc(sizeof(double) * (size_t)(qq * p));
  double *row = (double *)malloc(sizeof(double) * (size_t)p);

  /* Q <- A_in */
  for (int64_t j = 0; j < p; ++j)
    for (int64_t i = 0; i < m; ++i) AT(Q, i, j, ldq) = AT(Ain, i, j, lda);
  /* B <- 0 */
  for (int64_t j = 0; j < p; ++j)
    for (int64_t i = 0; i < q; ++i) AT(B, i, j, ldb) = 0.0;
  /* R <- I_p */
  set_identity(p, R, ldr);
  /* Bt <- Q_in^T Q */
  if (q > 0) orc_gemm_tn(m, q, p, Qin, ldqin, Q, ldq, Bt, q);
  /* X <- Q^T Q - Bt^T Bt */
  update_gram(m, q, p, Q, ldq, Bt, X);
  double orth = orc_frob_minus_identity(p, X, p);
  if (!isfinite(orth)) status = ORC_ERR_BREAKDOWN; /* as in orc_cholqr */

  int it = 0;
  while (status == ORC_OK && (orth >= tol || it < o->min_iter) && it < o->max_iter) {
    /* shift loop */
    double sigma = 0.0;
    double normX = -1.0;
    inf.chol_attempts++;
    int rc = orc_chol(p, X, p, sigma, Rt, p);
    int esc = 0;
    while (rc != 0 && esc < o->max_escalations) {
      if (sigma == 0.0) {
        if (normX < 0.0) normX = orc_sym_norm2(p, X, p);
        sigma = orc_update_shift(m, q, p, normX);
        inf.shifts++;
        if (inf.shifts == 1) inf.sigma_first = sigma;
      } else {
        sigma = 10.0 * sigma;
        inf.escalations++;
      }
      sigma = fmax(sigma, 2.0 * ORC_U);
      inf.sigma_last = sigma;
      inf.chol_attempts++;
      rc = orc_chol(p, X, p, sigma, Rt, p);
      esc++;
    }
    if (rc != 0) {
      status = ORC_ERR_BREAKDOWN;
      break;
    }
    /* Q <- (Q - Q_in Bt) R~^{-1}, row by row */
    for (int64_t r = 0; r < m; ++r) {
      for (int64_t j = 0; j < p; ++j) {
        double s = AT(Q, r, j, ldq);
        for (int64_t k = 0; k < q; ++k) s -= AT(Qin, r, k, ldqin) * AT(Bt, k, j, q);
        row[j] = s;
      }
      for (int64_t j = 0; j < p; ++j) AT(Q, r, j, ldq) = row[j];
    }
    orc_trsm_runn(m, p, Q, ldq, Rt, p, Q, ldq);
    /* B <- B + Bt R */
    for (int64_t j = 0; j < p; ++j)
      for (int64_t i = 0; i < q; ++i) {
        double s = 0.0;
        for (int64_t k = 0; k <= j; ++k) s += AT(Bt, i, k, q) * AT(R, k, j, ldr);
        AT(Bn, i, j, q) = AT(B, i, j, ldb) + s;
      }
    for (int64_t j = 0; j < p; ++j)
      for (int64_t i = 0; i < q; ++i) AT(B, i, j, ldb) = AT(Bn, i, j, q);
    /* R <- R~ R */
    orc_trmm_upper(p, Rt, p, R, ldr, Rn, p);
    for (int64_t j = 0; j < p; ++j)
      for (int64_t i = 0; i < p; ++i) AT(R, i, j, ldr) = AT(Rn, i, j, p);
    /* Bt <- Q_in^T Q */
    if (q > 0) orc_gemm_tn(m, q, p, Qin, ldqin, Q, ldq, Bt, q);
    /* X <- Q^T Q - Bt^T Bt */
    update_gram(m, q, p, Q, ldq, Bt, X);
    orth = orc_frob_minus_identity(p, X, p);
    ++it;
    if (!isfinite(orth)) status = ORC_ERR_BREAKDOWN;
  }
  inf.iters = it;
  inf.orth_frob = orth;
  {
    double bs = 0.0;
    for (int64_t j = 0; j < p; ++j)
      for (int64_t i = 0; i < q; ++i) bs += AT(Bt, i, j, q) * AT(Bt, i, j, q);
    inf.proj_frob = sqrt(bs);
  }
  if (status == ORC_OK && orth >= tol) status = ORC_NOT_CONVERGED;
  if (info) *info = inf;
  free(Bt);
  free(X);
  free(Rt);
  free(Rn);
  free(Bn);
  free(row);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Alg. 3 (pnCholQR): Alg. 2 applied panel by panel.                          */
/* ------------------------------------------------------------------------- */

/* Splits A (m x n) into r panels of widths w_i = n/r (the first n mod r
 * panels one wider) and appends them in order with Alg. 2.  Q is m x n, R is
 * n x n upper triangular.  Returns the worst status over the panels;
 * info accumulates iterations and shifts, orth_frob is the last panel's. */
int orc_pncholqr(const orc_opts *o, int64_t m, int64_t n, int64_t r,
                 const double *A, int64_t lda, double *Q, int64_t ldq,
                 double *R, int64_t ldr, orc_info *info) {
  orc_info tot;
  memset(&tot, 0, sizeof(tot));
  int status = ORC_OK;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(R, i, j, ldr) = 0.0;
  int64_t q = 0;
  for (int64_t k = 0; k < r; ++k) {
    int64_t p = n / r + (k < n % r ? 1 : 0);
    if (p == 0) continue;
    orc_info pi;
    int rc = orc_cholqr_update(o, m, q, Q, ldq, p, &AT(A, 0, q, lda), lda,
                               &AT(Q, 0, q, ldq), ldq, &AT(R, 0, q, ldr), ldr,
                               &AT(R, q, q, ldr), ldr, &pi);
    tot.iters += pi.iters;
    tot.chol_attempts += pi.chol_attempts;
    tot.shifts += pi.shifts;
    tot.escalations += pi.escalations;
    if (tot.sigma_first == 0.0) tot.sigma_first = pi.sigma_first;
    if (pi.sigma_last != 0.0) tot.sigma_last = pi.sigma_last;
    tot.orth_frob = pi.orth_frob;
    tot.proj_frob = pi.proj_frob;
    if (rc < 0) {
      status = rc;
      break;
    }
    if (rc == ORC_NOT_CONVERGED) status = ORC_NOT_CONVERGED;
    q += p;
  }
  if (info) *info = tot;
  return status;
}

/* ------------------------------------------------------------------------- */
/* Checker: Householder QR (Golub & Van Loan, Alg. 5.2.1 + 5.1.1).            */
/* ------------------------------------------------------------------------- */

/* Economy QR of A (m x n, m >= n) by Householder reflections, with the signs
 * normalised so that R has a non-negative diagonal.  Q is m x n, R is n x n.
 * For full-rank A this QR is unique, which makes it the reference for the
 * Cholesky-based factors on small inputs. */
void orc_householder_qr(int64_t m, int64_t n, const double *A, int64_t lda,
                        double *Q, int64_t ldq, double *R, int64_t ldr) {
  double *a = (double *)malloc(sizeof(double) * (size_t)(m * n));
  double *v = (double *)malloc(sizeof(double) * (size_t)(m * n));
  double *beta = (double *)malloc(sizeof(double) * (size_t)n);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) a[i + j * m] = AT(A, i, j, lda);
  for (int64_t j = 0; j < n; ++j) {
    /* house(x) for x = a[j:m, j] (GVL Alg. 5.1.1) */
    double sigma = 0.0;
    for (int64_t i = j + 1; i < m; ++i) sigma += a[i + j * m] * a[i + j * m];
    double x0 = a[j + j * m];
    double *vj = v + j * m;
    for (int64_t i = 0; i < m; ++i) vj[i] = 0.0;
    vj[j] = 1.0;
    for (int64_t i = j + 1; i < m; ++i) vj[i] = a[i + j * m];
    double b;
    if (sigma == 0.0) {
      b = 0.0;
    } else {
      double mu = sqrt(x0 * x0 + sigma);
      double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
      b = 2.0 * v0 * v0 / (sigma + v0 * v0);
      for (int64_t i = j + 1; i < m; ++i) vj[i] /= v0;
    }
    beta[j] = b;
    /* a[j:m, j:n] <- (I - b v v^T) a[j:m, j:n] */
    for (int64_t c = j; c < n; ++c) {
      double s = 0.0;
      for (int64_t i = j; i < m; ++i) s += vj[i] * a[i + c * m];
      s *= b;
      for (int64_t i = j; i < m; ++i) a[i + c * m] -= s * vj[i];
    }
  }
  /* R = upper part of a; Q = H_1 ... H_n [I_n; 0] (backward accumulation) */
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(R, i, j, ldr) = (i <= j) ? a[i + j * m] : 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(Q, i, j, ldq) = (i == j) ? 1.0 : 0.0;
  for (int64_t j = n - 1; j >= 0; --j) {
    double *vj = v + j * m;
    for (int64_t c = 0; c < n; ++c) {
      double s = 0.0;
      for (int64_t i = j; i < m; ++i) s += vj[i] * AT(Q, i, c, ldq);
      s *= beta[j];
      for (int64_t i = j; i < m; ++i) AT(Q, i, c, ldq) -= s * vj[i];
    }
  }
  /* sign normalisation: make diag(R) >= 0 */
  for (int64_t j = 0; j < n; ++j)
    if (AT(R, j, j, ldr) < 0.0) {
      for (int64_t c = j; c < n; ++c) AT(R, j, c, ldr) = -AT(R, j, c, ldr);
      for (int64_t i = 0; i < m; ++i) AT(Q, i, j, ldq) = -AT(Q, i, j, ldq);
    }
  free(a);
  free(v);
  free(beta);
}

/* ------------------------------------------------------------------------- */
/* Metrics of Sec. 4.1 (spectral norms through Jacobi on n x n Gramians).     */
/* ------------------------------------------------------------------------- */

/* ||M||_2 for an m x n matrix: sqrt(lambda_max(M^T M)). */
static double mat_norm2(int64_t m, int64_t n, const double *M, int64_t ldm) {
  double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
  orc_gram(m, n, M, ldm, G, n);
  double l = orc_sym_norm2(n, G, n);
  free(G);
  return sqrt(l);
}

/* LOO(Q) = ||I - Q^T Q||_2 */
double orc_loo(int64_t m, int64_t n, const double *Q, int64_t ldq) {
  double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
  orc_gram(m, n, Q, ldq, G, n);
  for (int64_t i = 0; i < n; ++i) G[i + i * n] -= 1.0;
  double l = orc_sym_norm2(n, G, n);
  free(G);
  return l;
}

/* ||I - Q^T Q||_F (the Sec. 4.1 stopping quantity) */
double orc_loo_frob(int64_t m, int64_t n, const double *Q, int64_t ldq) {
  double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
  orc_gram(m, n, Q, ldq, G, n);
  double f = orc_frob_minus_identity(n, G, n);
  free(G);
  return f;
}

/* RRR(A, Q, R) = ||A - Q R||_2 / ||A||_2 */
double orc_rrr(int64_t m, int64_t n, const double *A, int64_t lda,
               const double *Q, int64_t ldq, const double *R, int64_t ldr) {
  double *D = (double *)malloc(sizeof(double) * (size_t)(m * n));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t k = 0; k <= j; ++k) s += AT(Q, i, k, ldq) * AT(R, k, j, ldr);
      D[i + j * m] = AT(A, i, j, lda) - s;
    }
  double num = mat_norm2(m, n, D, m);
  double den = mat_norm2(m, n, A, lda);
  free(D);
  return num / den;
}

/* RCR(A, R) = ||A^T A - R^T R||_2 / ||A||_2^2 */
double orc_rcr(int64_t m, int64_t n, const double *A, int64_t lda,
               const double *R, int64_t ldr) {
  double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
  orc_gram(m, n, A, lda, G, n);
  double den = orc_sym_norm2(n, G, n);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      int64_t kmax = i < j ? i : j;
      for (int64_t k = 0; k <= kmax; ++k) s += AT(R, k, i, ldr) * AT(R, k, j, ldr);
      G[i + j * n] -= s;
    }
  double num = orc_sym_norm2(n, G, n);
  free(G);
  return num / den;
}
