/* Plain FP64 CPU oracle for shifted Cholesky QR (test infrastructure only).
 * Declarations for oracle/cholqr_oracle.c; used by nothing but that file and
 * its ctypes wrapper oracle/__init__.py. */
#ifndef CHOLQR_ORACLE_H
#define CHOLQR_ORACLE_H
#include <stdint.h>

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_ERR_BREAKDOWN = -2 };
enum {
  ORC_SHIFT_SCHOLQR3 = 0,        /* pass 1 shifted, later shifts on breakdown */
  ORC_SHIFT_ON_BREAKDOWN = 1,    /* Alg. 1 as printed */
  ORC_SHIFT_NONE = 2,            /* CholQR / CholQR2 */
  ORC_SHIFT_SCHOLQR3_STRICT = 3, /* Fukaya sCholQR3: later breakdown fails */
  ORC_SHIFT_ISCHOLQR = 4         /* one shift, reused (Fukaya isCholQR) */
};
enum { ORC_STOP_FROB_TOL = 0, ORC_STOP_U_SQRT_N = 1 };

typedef struct {
  double tol;
  int max_iter;
  int min_iter;
  int shift_policy;
  int stop_rule;
  int max_escalations;
} orc_opts;

typedef struct {
  int iters;
  int chol_attempts;
  int shifts;
  int escalations;
  double sigma_first;
  double sigma_last;
  double orth_frob;
  double proj_frob;
} orc_info;

void orc_default_opts(orc_opts *o);
void orc_gram(int64_t m, int64_t n, const double *A, int64_t lda, double *X, int64_t ldx);
void orc_gemm_tn(int64_t m, int64_t p, int64_t q, const double *A, int64_t lda,
                 const double *B, int64_t ldb, double *C, int64_t ldc);
int orc_chol(int64_t n, const double *X, int64_t ldx, double sigma, double *R, int64_t ldr);
void orc_trsm_runn(int64_t m, int64_t n, const double *A, int64_t lda, const double *R,
                   int64_t ldr, double *Q, int64_t ldq);
void orc_trmm_upper(int64_t n, const double *T, int64_t ldt, const double *R, int64_t ldr,
                    double *C, int64_t ldc);
double orc_frob_minus_identity(int64_t n, const double *X, int64_t ldx);
int orc_sym_eigvals(int64_t n, const double *X, int64_t ldx, double *w);
double orc_sym_norm2(int64_t n, const double *X, int64_t ldx);
double orc_shift(int64_t m, int64_t n, double normX);
double orc_update_shift(int64_t m, int64_t q, int64_t p, double normX);
int orc_cholqr(const orc_opts *o, int64_t m, int64_t n, const double *A, int64_t lda,
               double *Q, int64_t ldq, double *R, int64_t ldr, orc_info *info);
int orc_cholqr_update(const orc_opts *o, int64_t m, int64_t q, const double *Qin,
                      int64_t ldqin, int64_t p, const double *Ain, int64_t lda, double *Q,
                      int64_t ldq, double *B, int64_t ldb, double *R, int64_t ldr,
                      orc_info *info);
int orc_pncholqr(const orc_opts *o, int64_t m, int64_t n, int64_t r, const double *A,
                 int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr,
                 orc_info *info);
void orc_householder_qr(int64_t m, int64_t n, const double *A, int64_t lda, double *Q,
                        int64_t ldq, double *R, int64_t ldr);
double orc_loo(int64_t m, int64_t n, const double *Q, int64_t ldq);
double orc_loo_frob(int64_t m, int64_t n, const double *Q, int64_t ldq);
double orc_rrr(int64_t m, int64_t n, const double *A, int64_t lda, const double *Q,
               int64_t ldq, const double *R, int64_t ldr);
double orc_rcr(int64_t m, int64_t n, const double *A, int64_t lda, const double *R,
               int64_t ldr);
#endif
