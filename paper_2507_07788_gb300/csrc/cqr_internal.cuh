// Internal declarations shared by the translation units of libcholqr.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "cholqr.h"

// A growing basis (Q m x n_max with q valid columns, R n_max x n_max).
struct cqr_basis {
  int device;
  int64_t m, n_max, q, ldq, ldr;
  double *Q;
  double *R;
  cqr_opts opts;
  // digit cache of Q's columns (basis_enable_digit_cache): 7 bf16 planes of
  // n_max x ldc (ldc = m rounded up to 64) and one exponent per column
  uint16_t *Qd;
  int *Qe;
  int64_t ldc;
};

namespace cqr {

// Shared-memory attributes of a kernel belong to each device's context: this
// sets them once per device (bit d of `done` for device d < 64; devices
// beyond 64 set them on every launch).  Safe from several host threads.
struct KernelAttr {
  std::atomic<uint64_t> done{0};
};
template <typename K>
inline void set_smem_attr(KernelAttr &ka, K *kernel, int bytes, bool max_carveout) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit != 0 && (ka.done.load(std::memory_order_acquire) & bit) != 0) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (max_carveout)
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (bit != 0) ka.done.fetch_or(bit, std::memory_order_release);
}

constexpr double kU64 = 1.1102230246251565404236316680908203125e-16;  // 2^-53
constexpr int kThreads = 256;        // block size of the row-sweeping kernels
constexpr int kCtrlThreads = 512;    // block size of the single-CTA control kernel

// Device-resident status of one factorisation / append, written by the
// control kernel and read by the host once per call (and by every
// row-sweeping kernel, which returns at once when `done` is set).
struct DevState {
  int32_t done;
  int32_t status;
  int32_t iters;
  int32_t chol_attempts;
  int32_t shifts;
  int32_t escalations;
  int32_t active;  // the control kernel asked for another row pass
  int32_t pad;
  double sigma_first;
  double sigma_last;
  double orth_frob;
  double proj_frob;
  double sigma_once;  // isCholQR: the one shift, 0 until the first breakdown
};

// One sweep over the m rows.  The block being orthogonalised is Y (m x p);
// Q_in (m x q, q may be 0) is the fixed basis of an update.  With do_trsm the
// sweep first replaces each row y by (y - q_in B~) R~^{-1} (Alg. 1,
// Alg. 2) and writes it to Yout; in every case it accumulates the
// per-CTA partial sums of C = [Q_in Y]^T Y restricted to the B~ part
// (q x p) and the upper triangle of Y^T Y, in a fixed row order.
struct RowSweep {
  int64_t m;
  int32_t q, p;
  const double *Qin;
  int64_t ldqin;
  const double *Yin;
  int64_t ldyin;
  double *Yout;
  int64_t ldyout;
  const double *Rt;     // p x p upper (ld p): R~ of the current pass
  const double *Rdinv;  // p: 1 / R~_jj
  const double *Bt;     // q x p (ld q): B~ of the current iteration
  double *partials;     // [grid][E]
  int64_t E;            // q p + p (p + 1) / 2
  int64_t rows_per_cta; // multiple of tile_rows
  int32_t tile_rows;
  int32_t lds;          // shared-memory row stride (doubles), odd
  int32_t do_trsm;
  int32_t accumulate;  // tensor-core Gramian: add into the partials (later chunks of a pass)
  const double *Tinv;   // p x p upper (ld p): D R~^{-1} (tensor-core product Q = (Y D^-1)(D T))
  const int *Tscale;    // p: log2 of D (column k of Y is divided, row k of T multiplied, by 2^Tscale[k])
  const DevState *st;
  int32_t tc05;         // kTc05Gram | kTc05Solve: the tcgen05 kernels that may be used where they apply
  int32_t digits;       // digit Gramian: 0 (= 7, exact FP64) or kOzMixedDigits
  int *emax;            // digit Gramian: atomicMax of the final column exponents (or null)
};

struct Reduce {
  const double *partials;
  int32_t G;
  int64_t E;
  int32_t q, p;
  double *C;  // (q + p) x p, ld q + p
  const DevState *st;
};

enum { MODE_FACTOR = 0, MODE_UPDATE = 1 };

struct Ctrl {
  int64_t m;
  int32_t q, p;
  int32_t mode;
  int32_t shift_policy, max_iter, min_iter, max_escalations, stop_rule;
  double tol;
  // Mixed precision: when > 0 the first pass is always shifted by
  // max(first_shift_coeff * ||X|| + emax_coeff * sum_j 4^(emax_j - 1022), 2u)
  // (the Gramian came from FP32 data, emax null, or from the reduced-digit
  // Gramian, whose error bound is per row emax_coeff / m Ubar_i Ubar_j with
  // Ubar_j = 2^(emax_j - 1022)).
  double first_shift_coeff;
  const int *emax;      // p column exponents of the first Gramian (or null)
  double emax_coeff;
  int32_t r_external;  // 1: R <- R~ R is left to launch_rupdate (factor mode)
  const double *C;  // (q + p) x p, ld q + p
  double *Rt;       // p x p, ld p
  double *Rdinv;    // p
  double *Bt;       // q x p, ld q (update only)
  double *R;        // accumulated R (p x p block), ld ldr
  int64_t ldr;
  double *B;        // accumulated B (q x p block), ld ldb (update only)
  int64_t ldb;
  DevState *st;
  // Working storage of the control step (X, packed R~, two vectors and the
  // cooperative launch's control words: ctrl_work_bytes(p) bytes) in global
  // memory, for widths whose working set does not fit in shared memory
  // (p > kCtrlSmemMaxP); null otherwise.
  double *work;
};
// Widest p whose control step works in shared memory (197 KB at 128).
constexpr int kCtrlSmemMaxP = 128;

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_init(double *R, int64_t ldr, int p, double *B, int64_t ldb, int q,
                        DevState *st, cudaStream_t s);
cudaError_t launch_rowsweep(const RowSweep &a, int grid, cudaStream_t s);
// FP32 Gramian sweep of the mixed-precision first pass (no solve): inputs
// truncated to FP32 on the integer pipe, FP32 products summed per tile,
// tiles combined with Kahan compensation, partials written as FP64.
cudaError_t launch_gram32(const RowSweep &a, int grid, cudaStream_t s);
void gram32_geometry(int q, int p, int *tile_rows, int *lds, size_t *smem);
// Summation depth of one FP32 partial (tile rows + Kahan), for the shift.
constexpr int kGram32Depth = 64 + 2;
cudaError_t launch_reduce(const Reduce &a, cudaStream_t s);
cudaError_t launch_ctrl(const Ctrl &a, cudaStream_t s);
size_t ctrl_smem_bytes(int p);
size_t ctrl_work_bytes(int p);  // Ctrl::work bytes for p > kCtrlSmemMaxP
// R <- R~ R (Alg. 1) with one CTA per column of R, after the control
// kernel of a pass that continues (for controls run with r_external = 1).
cudaError_t launch_rupdate(const double *Rt, int p, double *R, int64_t ldr, const DevState *st,
                           cudaStream_t s);
// T = D R~^{-1} and the exponents of D (for the tensor-core solve), one
// warp per row, after the control kernel of a pass.
cudaError_t launch_tinv(const double *Rt, const double *Rdinv, const double *C, int ldc, int q, int p,
                        double *Tinv, int *Tscale, const DevState *st, cudaStream_t s);

// Batched persistent variants (descriptor arrays and counts in device
// memory, so a captured CUDA graph can be replayed with new contents).  A
// problem in a batch runs the same per-CTA work, in the same order, as alone.
constexpr int kBatchEPT = 33;  // entries per thread; problems need E <= 256 * 33
cudaError_t launch_rowsweep_batched(const RowSweep *reqs, const int *item_req, const int *item_cta,
                                    const int *nitems, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_reduce_batched(const Reduce *reqs, const int *item_req, const int *item_chunk,
                                  const int *nitems, int grid, cudaStream_t s);
cudaError_t launch_ctrl_batched(const Ctrl *reqs, const int *nreq, int grid, size_t smem,
                                cudaStream_t s);
cudaError_t launch_init_batched(const Ctrl *reqs, const int *nreq, int grid, cudaStream_t s);

// Tensor-core (Ozaki digit) Gramian sweep for q = 0, p <= 64: optional FP64
// row solve, then the exact-digit Gramian of the tile; per-CTA partials are
// full p x p (ld p) and reduce_oz returns X = sum_g (P_g + P_g^T).
cudaError_t launch_ozgram(const RowSweep &a, int grid, cudaStream_t s);
cudaError_t launch_reduce_oz(const double *partials, int G, int n, double *C, const DevState *st,
                             cudaStream_t s);
int ozgram_grid(int64_t m, int n, bool tc05 = true);
// Reduced-digit Gramian of the mixed-precision first pass: 5 balanced
// base-256 digits, orders <= 4; per row it adds less than
// kOzMixedRowErr Ubar_i Ubar_j to X_ij (Ubar_j = 2^(E_j - 1022) for the
// column's largest biased exponent E_j).
constexpr int kOzMixedDigits = 5;
constexpr double kOzMixedRowErr = 2.0324e-12;  // about 2^-38.84: 2^-38.99 plus the floor rescalings, with margin
// Q = Y T (T = R~^{-1}) on the tensor cores, exact digit products, 33 <= n <= 128.
cudaError_t launch_ozgemm(const RowSweep &a, int grid, cudaStream_t s);
int ozgemm_grid(int64_t m, int n, bool tc05 = true);
int ozgemm_tile_rows(int n, bool tc05 = true);
// Digit cache of a basis (csrc/ozcache.cu): fill columns k0 .. k0 + p - 1,
// and the cross Gramian [Q_in Y]^T Y of appends of p <= 16 columns that
// reads it (partials (q + p) x p per row group, for launch_reduce_dense).
cudaError_t launch_cache_fill(const double *Q, int64_t ldq, int64_t m, int k0, int p, int *Qe, uint16_t *Qd,
                              int64_t ldc, int64_t plane, cudaStream_t s);
cudaError_t launch_ozcgram(const RowSweep &a, const uint16_t *Qd, int64_t ldc, int64_t plane, const int *Qe,
                           int groups, cudaStream_t s);
int ozcgram_grid(int64_t m, int q, int p);
int ozcgram_tile_rows();
// Projection and solve of such appends from the same cache (q <= 256):
// P = Q_in B~ exactly on the tensor cores, then y <- (y - P) R~^{-1} in FP64.
cudaError_t launch_ozcproj(const RowSweep &a, const uint16_t *Qd, int64_t ldc, int64_t plane, const int *Qe,
                           uint16_t *Bd, int *fexp, int grid, cudaStream_t s);
size_t ozcproj_scratch_bytes();
int ozcproj_grid(int64_t m);
constexpr int kOzCacheProjMaxQ = 256;
constexpr int kOzCacheMaxP = 16;
// bf16 FLOPs the tensor-core solve issues per row at width n (digit pairs x
// the k-blocks its upper-triangular T does not skip).
double ozgemm_tc_flops_per_row(int n, bool tc05 = true);
// Q = Y T (T = D R~^{-1}, a.Tinv and a.Tscale from launch_tinv) on the
// tensor cores for 128 < n <= CQR_MAX_N: the contraction in blocks of 64,
// one 64-column block of Q per CTA; three launches (T's digits, the row
// exponents, the product) through `scratch` (wide_solve_scratch_bytes).
cudaError_t launch_wide_solve(const RowSweep &a, void *scratch, cudaStream_t s);
size_t wide_solve_scratch_bytes(int64_t m, int n);
constexpr int kOzGemmMaxN = 128;
// Cross Gramian of the update, C = [Q_in Y]^T Y, on the tensor cores (exact
// digit products, p <= 64): partials of `groups` row groups, each (q + p) x p.
cudaError_t launch_ozxgram(const RowSweep &a, int groups, cudaStream_t s);
int ozxgram_grid(int64_t m, int q, int p);
int ozxgram_tile_rows();
cudaError_t launch_reduce_dense(const double *partials, int G, int64_t E, double *C, const DevState *st,
                                cudaStream_t s);
// The Gramian X = Y^T Y (ld ldx, both triangles) of a block wider than the
// digit Gramian (128 < p <= CQR_MAX_N) by 64 x 64 block pairs on the tensor
// cores (csrc/ozgemm.cu), through `partials` (wide_gram_partial_elems
// doubles); adds its kernel launches to *launches.
cudaError_t launch_wide_gram(const double *Y, int64_t ldy, int64_t m, int p, double *partials, double *X,
                             int64_t ldx, const DevState *st, cudaStream_t s, int *launches);
int64_t wide_gram_partial_elems(int64_t m, int p);
// Appends of at least kOzUpdMinP columns to bases of at least kOzUpdMinRows
// rows take the tensor-core cross Gramian.  Narrower blocks keep the fused
// FP64 sweep (its projection and Gramian share one read, and their FP64 work
// is small); shorter bases keep it too (the serving runtime's batched appends
// use it, so a batched append and a direct one agree bitwise).
constexpr int64_t kOzUpdMinRows = 262144;
constexpr int kOzUpdMinP = 32;
// From this width on the solve is the digit product (padded to 32, 64 or 128
// columns); at n <= 16 the FP64 substitution's n^2 / 2 FMAs per row stay.
constexpr int kOzGemmMinN = 17;
int ozgram_tile_rows();
// The digit Gramian on tcgen05 (csrc/tcgram.cu) for kTcGramMinN <= p <= 64,
// q = 0, no fused solve, Y 16-byte aligned with an even leading dimension;
// launch_ozgram dispatches to it when tcgram_usable(a).
constexpr int kTcGramMinN = 17;
// RowSweep::tc05 bits
constexpr int32_t kTc05Gram = 1, kTc05Solve = 2;
// Widths whose Gramian runs on the tcgen05 kernel under CQR_EMU_AUTO (below
// 33 columns the mma.sync kernel's narrower tile is faster than the tcgen05
// kernel's 64 padded columns)
constexpr int kTcGramAutoMinN = 33;
// Does the factorisation's (and cholqr_gram's) Gramian use the tcgen05
// kernel at this width and emulation mode?  The solve does under
// CQR_EMU_TCGEN05 only.
inline bool tc05_gram_mode(int emulation, int n) {
  return n <= 64 && ((emulation == CQR_EMU_TCGEN05 && n >= kTcGramMinN) ||
                     (emulation == CQR_EMU_AUTO && n >= kTcGramAutoMinN));
}
bool tcgram_usable(const RowSweep &a);
int tcgram_grid(int64_t m);
cudaError_t launch_tcgram(const RowSweep &a, int grid, cudaStream_t s);
// The digit solve Q = Y T on tcgen05 (csrc/tcgemm.cu) for kTcGemmMinN <= p
// <= 64 in 128-row tiles; launch_ozgemm dispatches to it when
// tcgemm_usable(a).
constexpr int kTcGemmMinN = 17;
bool tcgemm_usable(const RowSweep &a);
int tcgemm_tile_rows();
int tcgemm_grid(int64_t m);
double tcgemm_tc_flops_per_row();
cudaError_t launch_tcgemm(const RowSweep &a, int grid, cudaStream_t s);
constexpr int kOzMaxN = 128;
// FP64 row solve Q = Y R~^{-1} alone for n <= 16 (one thread per row,
// registers); shares SMs with ozgram_kernel when the two run on different
// streams.
cudaError_t launch_trsm_rows(const RowSweep &a, int grid, cudaStream_t s);
int trsm_rows_grid(int64_t m);

// Row-sharded factorisation: C[e] = sum over ranks r = 0, 1, ... (in that
// order) of recv[r * count + e].
cudaError_t launch_sum_ranks(const double *recv, int world, int64_t count, double *C, cudaStream_t s);

// Geometry of a row sweep for the given widths: tile rows, shared stride and
// bytes of dynamic shared memory.
void rowsweep_geometry(int q, int p, int *tile_rows, int *lds, size_t *smem);
int rowsweep_grid(int64_t m, int tile_rows);
int num_sms();

}  // namespace cqr
