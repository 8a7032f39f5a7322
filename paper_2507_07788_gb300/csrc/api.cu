// C ABI of libcholqr: argument checking, scratch management and the launch
// sequence of a factorisation (Alg. 1 with the sCholQR3 first-pass shift) and
// of a basis update (Alg. 2).
//
// Launch sequence of one call (all on the caller's stream, no host round
// trip until the end):
//   init                      R = I (and B = 0), device state cleared
//   sweep (Gram)              partial sums of [Q_in Y]^T Y, Y = A or A_in
//   reduce, ctrl              X, stop test, shift, Cholesky, R~, R <- R~ R
//   repeat: sweep (solve+Gram), reduce, ctrl
// The row sweeps and reductions return immediately once the control kernel
// has marked the call done, so launching a few passes ahead is harmless.  The
// host reads the 72-byte device state once after `kPrelaunch` passes and
// only launches further passes (one at a time) when the tolerance has not
// been met yet.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <deque>
#include <mutex>
#include <vector>

#include "cqr_internal.cuh"

using namespace cqr;

namespace {

constexpr int kPrelaunch = 3;

// ---- instrumentation (cqr_timing_*)
std::mutex g_timing_mu;
cqr_timing g_timing = {};
std::atomic<int> g_timing_on{0};
std::atomic<int64_t> g_launches{0};

enum { MARK_SWEEP = 0, MARK_SOLVE = 1, MARK_GRAM = 2, MARK_TSOLVE = 3 };

struct SweepMark {
  cudaEvent_t a, b;
  int pass;    // 0 = first Gramian sweep, k >= 1 = k-th solve + Gramian sweep
  int kind;    // MARK_*
  double flops, bytes;
  double tc_flops;  // MARK_TSOLVE: digit-product FLOPs on the tensor pipe
};

// Per host thread: an auxiliary stream and events for the chunked pass
// pipeline (the row solve of chunk c+1 on the caller's stream overlapping
// the tensor-core Gramian of chunk c on the auxiliary stream).
struct AuxCtx {
  cudaStream_t aux = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> ev;
};

constexpr int kMaxDevices = 64;

int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return (dev >= 0 && dev < kMaxDevices) ? dev : 0;
}

// One auxiliary stream per host thread and device (streams and events belong
// to the device that was current when they were created).
AuxCtx *aux_ctx(int nchunks) {
  thread_local AuxCtx per_device[kMaxDevices];
  AuxCtx &c = per_device[current_device()];
  if (c.aux == nullptr) {
    // the highest priority: a whole-pass Gramian launched here takes SMs
    // ahead of the pending blocks of the host copies (default priority)
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
      (void)cudaGetLastError();
      greatest = 0;
    }
    if (cudaStreamCreateWithPriority(&c.aux, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess) {
      (void)cudaGetLastError();
      c.aux = nullptr;
      return nullptr;
    }
  }
  while ((int)c.ev.size() < nchunks) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    c.ev.push_back(e);
  }
  return &c;
}

// Copy stream of the host-staged factorisation, per host thread and device,
// with an event per row chunk for the device->host copy of Q after a pass,
// and a page-locked record of the pass whose Q each chunk last received.
struct CopyCtx {
  cudaStream_t st = nullptr;
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> c;
  int *copied = nullptr;    // host view
  int *copied_d = nullptr;  // device view
};

constexpr int kCopyGrid = 16, kCopyThreads = 1024;

// Q chunk -> host after pass k's solve of that chunk, speculatively: pass k
// is taken to be the last when its input has ||Q^T Q - I||_F < kCopyAheadOrth
// (then cond(Q^T Q) <= (1 + 1/2) / (1 - 1/2) = 3, and one Cholesky QR pass
// of such a Q lands on the roundoff floor).  It copies iff pass k ran (the
// control step sets iters to the index of the pass it admits; iters never
// decreases) and that test holds; the control step after pass k waits for
// these copies, so the state it reads is the one before pass k.  `copied`
// records the pass.
constexpr double kCopyAheadOrth = 0.5;

__global__ void __launch_bounds__(kCopyThreads) copy_out_kernel(const double *src, int64_t lds, int64_t rows,
                                                                int cols, double *dst, int64_t ldd, int k,
                                                                const DevState *st, int *copied) {
  if (st->iters < k || !(st->orth_frob < kCopyAheadOrth)) return;
  const int64_t n = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    dst[i + j * ldd] = src[i + j * lds];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *copied = k;
}

CopyCtx *copy_ctx(int nchunks) {
  thread_local CopyCtx per_device[kMaxDevices];
  CopyCtx &x = per_device[current_device()];
  if (x.st == nullptr) {
    if (cudaStreamCreateWithFlags(&x.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.start, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc((void **)&x.copied, sizeof(int) * 64, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&x.copied_d, x.copied, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      x.st = nullptr;
      return nullptr;
    }
  }
  while ((int)x.c.size() < nchunks) {
    cudaEvent_t b;
    if (cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    x.c.push_back(b);
  }
  return &x;
}

constexpr int kMaxChunks = 8;
constexpr int64_t kMinChunkRows = 78 * 1024;

// Thread-local pool of event pairs for the sweep marks of one call, per
// device.  A deque: a mark taken before a later one is added must keep its
// address.
std::deque<SweepMark> &marks_pool() {
  thread_local std::deque<SweepMark> pool[kMaxDevices];
  return pool[current_device()];
}

cqr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CQR_OK;
  if (e == cudaErrorMemoryAllocation) return CQR_ERR_OOM;
  return CQR_ERR_CUDA;
}

#define CQR_TRY(expr)                                   \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) {                            \
      (void)cudaGetLastError();                         \
      return cuda_status(_e);                           \
    }                                                   \
  } while (0)

bool opts_valid(const cqr_opts &o) {
  return o.tol >= 0.0 && o.max_iter >= 1 && o.max_iter <= 100 && o.min_iter >= 0 &&
         o.update_min_iter >= 0 && o.max_escalations >= 0 && o.max_escalations <= 400 &&
         (o.precision == CQR_PREC_FP64 || o.precision == CQR_PREC_MIXED) &&
         o.shift_policy >= CQR_SHIFT_SCHOLQR3 && o.shift_policy <= CQR_SHIFT_ISCHOLQR &&
         (o.stop_rule == CQR_STOP_FROB_TOL || o.stop_rule == CQR_STOP_U_SQRT_N) &&
         (o.emulation == CQR_EMU_AUTO || o.emulation == CQR_EMU_OFF || o.emulation == CQR_EMU_TCGEN05);
}

// Pinned host mirror of the device state, one per host thread.
DevState *host_state() {
  thread_local DevState *h = nullptr;
  if (h == nullptr) {
    if (cudaMallocHost((void **)&h, sizeof(DevState)) != cudaSuccess) {
      (void)cudaGetLastError();
      h = nullptr;
    }
  }
  return h;
}

void keep_pool_memory() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    (void)cudaGetLastError();
  });
}

// Scratch of one call: device state, reduced C, R~, 1/diag R~, B~, partials.
struct Scratch {
  char *base = nullptr;
  DevState *st;
  double *C, *Rt, *Rdinv, *Bt, *Tinv, *partials;
  int *Tscale;
  uint16_t *Bd;  // digits of the scaled B~ (cached-digit projection)
  int *fexp;
  int *emax;     // column exponents of the reduced-digit first Gramian
  double *cwork; // global working storage of the control step (p > kCtrlSmemMaxP)
  void *xwork;   // working storage of the wide solve (or null)
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

cudaError_t scratch_alloc(Scratch &s, int q, int p, int G, int64_t E, cudaStream_t str, size_t xbytes = 0) {
  const size_t b_st = align256(sizeof(DevState));
  const size_t b_C = align256(sizeof(double) * (size_t)(q + p) * p);
  const size_t b_Rt = align256(sizeof(double) * (size_t)p * p);
  const size_t b_Rd = align256(sizeof(double) * (size_t)p);
  const size_t b_Bt = align256(sizeof(double) * (size_t)std::max(q, 1) * p);
  const size_t b_P = align256(sizeof(double) * (size_t)G * (size_t)E);
  keep_pool_memory();
  const size_t b_Ts = align256(sizeof(int) * (size_t)p);
  const size_t b_Bd = align256(ozcproj_scratch_bytes());
  const size_t b_W = (p > kCtrlSmemMaxP) ? align256(ctrl_work_bytes(p)) : 0;
  const size_t b_X = align256(xbytes);
  cudaError_t e = cudaMallocAsync((void **)&s.base,
                                  b_st + b_C + 2 * b_Rt + b_Rd + b_Bt + 2 * b_Ts + b_Bd + b_W + b_X + b_P, str);
  if (e != cudaSuccess) return e;
  char *p0 = s.base;
  s.st = (DevState *)p0;
  p0 += b_st;
  s.C = (double *)p0;
  p0 += b_C;
  s.Rt = (double *)p0;
  p0 += b_Rt;
  s.Rdinv = (double *)p0;
  p0 += b_Rd;
  s.Bt = (double *)p0;
  p0 += b_Bt;
  s.Tinv = (double *)p0;
  p0 += b_Rt;
  s.Tscale = (int *)p0;
  p0 += b_Ts;
  s.emax = (int *)p0;
  p0 += b_Ts;
  s.Bd = (uint16_t *)p0;
  s.fexp = (int *)(p0 + sizeof(uint16_t) * 7 * 16 * (256 + 8));
  p0 += b_Bd;
  s.cwork = b_W ? (double *)p0 : nullptr;
  p0 += b_W;
  s.xwork = b_X ? (void *)p0 : nullptr;
  p0 += b_X;
  s.partials = (double *)p0;
  return cudaSuccess;
}

// The iteration driver shared by factor (q = 0) and append (q > 0).
struct Problem {
  int64_t m;
  int q, p;
  const double *Qin;
  int64_t ldqin;
  const double *Y0;  // input block (A or A_in)
  int64_t ldy0;
  double *Y;         // output block (Q or the basis columns q .. q+p-1)
  int64_t ldy;
  double *R;         // p x p block, ld ldr
  int64_t ldr;
  double *B;         // q x p block, ld ldb (nullptr when q == 0)
  int64_t ldb;
  int mode;
  int min_iter;
  cqr_opts o;
  // Digit cache of Q_in (appends to a basis that keeps one), or null.
  const uint16_t *Qd = nullptr;
  const int *Qe = nullptr;
  int64_t ldc = 0, cplane = 0;
  // Host staging (cholqr_factor_host): Y0 == Y is the device copy of hA,
  // copied ahead of the first Gramian; hQ (host memory the device can write,
  // or null) receives Q chunk by chunk as the pass expected to be the last
  // solves it, and *hq_written tells the caller whether it holds the final Q.
  const double *hA = nullptr;
  int64_t ldha = 0;
  double *hQ = nullptr;
  int64_t ldhq = 0;
  bool *hq_written = nullptr;
  // Row-sharded factorisation (cholqr_factor_sharded): this rank's rows are
  // P.m of m_total; each reduced Gramian is exchanged through the reducer and
  // summed in rank order before the control step.
  const cqr_reducer *red = nullptr;
  int64_t m_total = 0;
};

cqr_status run(const Problem &P, cqr_info *info, cudaStream_t str) {
  const int q = P.q, p = P.p;
  int tile_rows, lds;
  size_t smem;
  rowsweep_geometry(q, p, &tile_rows, &lds, &smem);
  const int G = rowsweep_grid(P.m, tile_rows);
  const int64_t tiles = (P.m + tile_rows - 1) / tile_rows;
  const int64_t rows_per_cta = ((tiles + G - 1) / G) * tile_rows;
  const int64_t E = (int64_t)q * p + (int64_t)p * (p + 1) / 2;
  const bool split = E > (int64_t)kThreads * 33;  // fused solve+Gram needs one entry group
  // Mixed precision (factor only): the first Gramian from FP32 data, with the
  // first shift sized for that roundoff:
  //   sigma = 11 (n (2 u_in + d u_acc) + n (n + 1) u) ||X||,
  // u_in = 2^-23 (truncation to FP32), u_acc = 2^-24, d = FP32 summation
  // depth of one partial, u = 2^-53 for the FP64 Cholesky.
  const bool mixed = (P.mode == MODE_FACTOR) && (P.o.precision == CQR_PREC_MIXED);
  // With the digit kernels (n <= 128, emulation on, one process) the first
  // Gramian is the reduced-digit one (kOzMixedDigits digits) and its shift
  //   sigma = 11 (m e_row sum_j Ubar_j^2 + n (n + 1 + G + 9) u ||X||)
  // covers its truncation (m rows of at most e_row Ubar_i Ubar_j each, a
  // rank-one bound of norm e_row sum_j Ubar_j^2), the single rounding of the
  // G partials and their fixed-order sum (at most (G + 9) u ||X|| per entry)
  // and the FP64 Cholesky (n (n + 1) u ||X||), in the form of Alg. 1.
  // Otherwise it is the FP32 sweep.  A sharded factorisation keeps the FP32
  // sweep: its shift does not depend on the rank's rows.
  const bool mixed_oz = mixed && (p <= kOzMaxN) && (P.o.emulation != CQR_EMU_OFF) && (P.red == nullptr);
  double mixed_coeff = 0.0, mixed_emax_coeff = 0.0;
  const int Gmix = mixed_oz ? ozgram_grid(P.m, p, false) : 0;  // partials of that Gramian
  if (mixed_oz) {
    mixed_coeff = 11.0 * (double)p * ((double)p + 1.0 + (double)Gmix + 9.0) * kU64;
    mixed_emax_coeff = 11.0 * (double)P.m * kOzMixedRowErr;
  } else if (mixed) {
    const double u_in = 1.1920928955078125e-07, u_acc = 5.9604644775390625e-08;
    mixed_coeff = 11.0 * ((double)p * (2.0 * u_in + kGram32Depth * u_acc) +
                          (double)p * (p + 1.0) * kU64);
  }

  // Tensor-core pass pipeline (digit Gramian, digit or FP64 solve) for
  // factorisations with n <= 128, and for appends to an empty basis above
  // the serving runtime's batched-append rows (q = 0: the row work of Alg. 2
  // is the same solve and Gramian; the control step keeps Alg. 2's shifts
  // and minimum iterations).  Wide appends to tall non-empty bases
  // (m >= kOzUpdMinRows, 32 <= p <= 64) form their cross Gramian
  // [Q_in Y]^T Y on the tensor cores (xoz) and keep the FP64 projection +
  // solve; the others keep the fused FP64 sweep.
  const bool ozu = (P.mode == MODE_UPDATE) && (q == 0) && (P.o.emulation != CQR_EMU_OFF) &&
                   (P.m > kOzUpdMinRows) && (p <= kOzMaxN);
  // Narrow appends (p <= 16) to a basis with a digit cache form the cross
  // Gramian from the cached digits of Q_in instead (cxg), with the same
  // FP64 projection + solve.
  const bool cxg = (P.mode == MODE_UPDATE) && (P.o.emulation != CQR_EMU_OFF) && !ozu && q > 0 &&
                   P.Qd != nullptr && (P.m > kOzUpdMinRows) && (p <= kOzCacheMaxP);
  const bool xoz = (P.mode == MODE_UPDATE) && (P.o.emulation != CQR_EMU_OFF) && !ozu && !cxg &&
                   (P.m >= kOzUpdMinRows) && (p >= kOzUpdMinP) && (p <= 64);
  int Gx = 0;
  int64_t x_rows_per_cta = 0;
  if (xoz || cxg) {
    Gx = xoz ? ozxgram_grid(P.m, q, p) : ozcgram_grid(P.m, q, p);
    const int64_t tr = xoz ? ozxgram_tile_rows() : ozcgram_tile_rows();
    const int64_t tiles = (P.m + tr - 1) / tr;
    x_rows_per_cta = ((tiles + Gx - 1) / Gx) * tr;
  }
  const bool oz = ((P.mode == MODE_FACTOR) || ozu) && (p <= kOzMaxN) && (P.o.emulation != CQR_EMU_OFF);
  // Blocks wider than the digit Gramian (p > 128) in a factorisation or an
  // append to an empty basis: the Gramian by column blocks on the
  // cross-Gramian kernel (wgx), the solve the FP64 row substitution.
  const bool wgx = ((P.mode == MODE_FACTOR) || (P.mode == MODE_UPDATE && q == 0)) && (p > kOzMaxN) &&
                   (P.o.emulation != CQR_EMU_OFF);
  // and their solve Q = Y T on the tensor cores, T = D R~^{-1} formed after
  // each control step (the contraction in blocks of 64)
  const bool wsolve = wgx;
  // tcgen05 kernels: the Gramian under AUTO for 33 <= n <= 64 and under
  // TCGEN05 for 17 <= n <= 64 (tc05_gram_mode); the solve under TCGEN05
  const bool tc05 = P.o.emulation == CQR_EMU_TCGEN05;
  const bool tcg = (P.mode == MODE_FACTOR || ozu) && tc05_gram_mode(P.o.emulation, p);
  const int Goz = oz ? ozgram_grid(P.m, p, tcg) : 0;
  int64_t oz_rows_per_cta = 0;
  if (oz) {
    const int64_t tr = ozgram_tile_rows();
    const int64_t tiles = (P.m + tr - 1) / tr;
    oz_rows_per_cta = ((tiles + Goz - 1) / Goz) * tr;
  }
  // Chunked pipeline of the passes for large m (see AuxCtx); for n > 64 the
  // solve and the Gramian always run as separate kernels (one chunk for small
  // m), with chunks half as tall since each row is twice as wide.
  const int64_t min_chunk = (p > 64) ? kMinChunkRows / 2 : kMinChunkRows;
  // The tcgen05 Gramian occupies whole SMs (216 KB of shared memory and the
  // whole register file), so it cannot share SMs with the solve's chunks: it
  // runs once per pass over all rows, after the solve (gram_whole), in one
  // chunk.  Host staging of Q ahead of the end (host_io) then costs more
  // than it saves: its copy kernels hold SMs the Gramian waits for (measured
  // 10.71 ms with, 10.37 ms without, at 1e6 x 64), so it is kept for the
  // chunked pipeline only.
  const bool gram_whole = tcg;
  const bool host_io = (P.hA != nullptr) && !mixed && !gram_whole;
  const int nchunks = (oz && !gram_whole)
                          ? (int)std::max<int64_t>(1, std::min<int64_t>(kMaxChunks, P.m / min_chunk))
                          : 1;
  const bool pipe = oz;
  // the solve of the pipelined passes: Q = Y T on the tensor cores (T = R~^{-1}
  // formed after the control kernel) for 17 <= n <= 128, FP64 substitution
  // otherwise
  const bool gemm = pipe && p >= kOzGemmMinN && p <= kOzGemmMaxN;
  int64_t chunk_rows = 0, chunk_rpc = 0;
  int Gc = 0;
  if (pipe) {
    const int64_t tr = ozgram_tile_rows();
    chunk_rows = (((P.m + nchunks - 1) / nchunks + tr - 1) / tr) * tr;
    Gc = ozgram_grid(chunk_rows, p, tcg);
    const int64_t tiles = chunk_rows / tr;
    chunk_rpc = ((tiles + Gc - 1) / Gc) * tr;
  }
  AuxCtx *ax = pipe ? aux_ctx(nchunks) : nullptr;
  if (pipe && ax == nullptr) return CQR_ERR_CUDA;  // no auxiliary stream or events
  // host staging pipelined with the passes (the tensor-core pipeline only)
  CopyCtx *cx = (host_io && pipe && ax != nullptr) ? copy_ctx(nchunks) : nullptr;
  const bool stage = cx != nullptr;
  if (P.hq_written != nullptr) *P.hq_written = false;
  const int64_t oz_parts =
      oz ? std::max<int64_t>(std::max<int64_t>((int64_t)Goz, (int64_t)Gc), (int64_t)Gmix) * p * p : 0;
  const int64_t x_parts = (xoz || cxg) ? (int64_t)Gx * (q + p) * p : 0;
  const int64_t w_parts = wgx ? wide_gram_partial_elems(P.m, p) : 0;
  const int64_t part_elems = std::max<int64_t>(E, (std::max(std::max(oz_parts, x_parts), w_parts) + G - 1) / G);
  bool last_x = false;   // the last sweep left dense cross-Gramian partials
  bool last_w = false;   // the last sweep left the reduced wide Gramian in C
  bool last_oz = false;  // which reduction the last sweep needs
  int last_oz_G = Goz;   // and over how many partials

  Scratch s;
  CQR_TRY(scratch_alloc(s, q, p, G, part_elems, str, wsolve ? wide_solve_scratch_bytes(P.m, p) : 0));
  DevState *hs = host_state();
  cqr_status result = CQR_OK;
  const bool timing = g_timing_on.load() != 0;
  std::deque<SweepMark> &pool = marks_pool();
  size_t nmarks = 0;
  int npass = 0;
  // algorithmic work of one sweep (the minimum, whether or not it is split)
  const double m_d = (double)P.m;
  const double gram_flops = 2.0 * m_d * (double)E;
  const double gram_bytes = 8.0 * m_d * (double)(q + p);
  const double solve_flops = 2.0 * m_d * ((double)q * p + (double)p * (p - 1) / 2.0) + m_d * p;
  const double solve_bytes = 8.0 * m_d * (double)p;  // the write of the new block

  // a mark around one kernel launch on stream `on` (timing only)
  auto kmark = [&](int kind, int pass, double flops, double bytes) -> SweepMark * {
    if (!timing) return nullptr;
    if (nmarks == pool.size()) {
      SweepMark nm{};
      cudaEventCreate(&nm.a);
      cudaEventCreate(&nm.b);
      pool.push_back(nm);
    }
    SweepMark *k = &pool[nmarks++];
    k->kind = kind;
    k->pass = pass;
    k->flops = flops;
    k->bytes = bytes;
    return k;
  };
  auto sweep = [&](bool trsm, bool first) -> cudaError_t {
    RowSweep a{};
    a.m = P.m;
    a.q = q;
    a.p = p;
    a.Qin = P.Qin;
    a.ldqin = P.ldqin;
    a.Yin = first ? P.Y0 : P.Y;
    a.ldyin = first ? P.ldy0 : P.ldy;
    a.Yout = P.Y;
    a.ldyout = P.ldy;
    a.Rt = s.Rt;
    a.Rdinv = s.Rdinv;
    a.Bt = s.Bt;
    a.partials = s.partials;
    a.E = E;
    a.rows_per_cta = rows_per_cta;
    a.tile_rows = tile_rows;
    a.lds = lds;
    a.do_trsm = trsm ? 1 : 0;
    a.st = s.st;
    a.tc05 = (tcg ? kTc05Gram : 0) | (tc05 ? kTc05Solve : 0);
    SweepMark *mk = nullptr;
    if (timing) {
      if (nmarks == pool.size()) {
        SweepMark nm{};
        cudaEventCreate(&nm.a);
        cudaEventCreate(&nm.b);
        pool.push_back(nm);
      }
      mk = &pool[nmarks++];
      mk->kind = MARK_SWEEP;
      mk->pass = trsm ? ++npass : 0;
      mk->flops = gram_flops + (trsm ? solve_flops : 0.0);
      mk->bytes = gram_bytes + (trsm ? solve_bytes : 0.0);
      cudaEventRecord(mk->a, str);
    } else if (trsm) {
      ++npass;
    }
    cudaError_t e = cudaSuccess;
    last_oz = false;
    last_x = false;
    last_w = false;
    if (xoz || cxg) {
      // projection + solve on the FP64 sweep (transform only), then the
      // cross Gramian of the new block on the tensor cores
      if (trsm) {
        if (cxg && q <= kOzCacheProjMaxQ) {
          // P = Q_in B~ from the cached digits, then the FP64 row solve
          RowSweep tf = a;
          const int Gp = ozcproj_grid(P.m);
          const int64_t tr = ozcgram_tile_rows();
          tf.rows_per_cta = (((P.m + tr - 1) / tr + Gp - 1) / Gp) * tr;
          e = launch_ozcproj(tf, P.Qd, P.ldc, P.cplane, P.Qe, s.Bd, s.fexp, Gp, str);
          g_launches += 2;
        } else {
          RowSweep tf = a;
          tf.E = 0;
          e = launch_rowsweep(tf, G, str);
          g_launches++;
        }
      }
      RowSweep x = a;
      x.Yin = trsm ? P.Y : a.Yin;
      x.ldyin = trsm ? P.ldy : a.ldyin;
      x.do_trsm = 0;
      x.rows_per_cta = x_rows_per_cta;
      SweepMark *mg = kmark(MARK_GRAM, npass, 2.0 * m_d * (q + p) * p, 8.0 * m_d * (q + p));
      if (mg && e == cudaSuccess) cudaEventRecord(mg->a, str);
      if (e == cudaSuccess)
        e = xoz ? launch_ozxgram(x, Gx, str) : launch_ozcgram(x, P.Qd, P.ldc, P.cplane, P.Qe, Gx, str);
      if (mg && e == cudaSuccess) cudaEventRecord(mg->b, str);
      g_launches++;
      last_x = true;
      if (mk != nullptr) cudaEventRecord(mk->b, str);
      return e;
    }
    if (pipe && trsm && ax != nullptr) {
      // chunked pipeline: solve chunk c on str; its Gramian on the aux stream
      int last_c = -1;  // the last chunk copied to the host
      for (int c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int64_t r0 = (int64_t)c * chunk_rows;
        const int64_t rc = std::min(chunk_rows, P.m - r0);
        if (rc <= 0) break;
        RowSweep tr = a;
        tr.m = rc;
        tr.Yin = a.Yin + r0;
        tr.Yout = a.Yout + r0;
        const double rcd = (double)rc;
        SweepMark *ms = kmark(gemm ? MARK_TSOLVE : MARK_SOLVE, npass, rcd * p * p, 16.0 * rcd * p);
        if (ms) ms->tc_flops = gemm ? rcd * ozgemm_tc_flops_per_row(p, tc05) : 0.0;
        if (ms) cudaEventRecord(ms->a, str);
        if (gemm) {
          const int Gg = ozgemm_grid(rc, p, tc05);
          const int64_t tg = ozgemm_tile_rows(p, tc05);
          tr.rows_per_cta = (((rc + tg - 1) / tg + Gg - 1) / Gg) * tg;
          tr.Tinv = s.Tinv;
          tr.Tscale = s.Tscale;
          e = launch_ozgemm(tr, Gg, str);
        } else {
          e = launch_trsm_rows(tr, trsm_rows_grid(rc), str);
        }
        if (ms) cudaEventRecord(ms->b, str);
        g_launches++;
        if (e == cudaSuccess) e = cudaEventRecord(ax->ev[c], str);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ax->aux, ax->ev[c], 0);
        if (stage && P.hQ != nullptr && e == cudaSuccess) {
          // chunk c of this pass's Q to the host while the next chunks run
          e = cudaStreamWaitEvent(cx->st, ax->ev[c], 0);
          if (e == cudaSuccess) {
            copy_out_kernel<<<kCopyGrid, kCopyThreads, 0, cx->st>>>(tr.Yout, tr.ldyout, rc, p, P.hQ + r0,
                                                                      P.ldhq, npass, s.st, cx->copied_d + c);
            e = cudaGetLastError();
            g_launches++;
          }
          if (e == cudaSuccess) e = cudaEventRecord(cx->c[c], cx->st);
          last_c = c;
        }
        if (gram_whole) continue;  // the Gramian follows all chunks
        RowSweep z = a;
        z.m = rc;
        z.Yin = a.Yout + r0;
        z.ldyin = a.ldyout;
        z.do_trsm = 0;
        z.partials = s.partials;  // chunk c adds into chunk c-1's slots (in order on aux)
        z.accumulate = (c > 0) ? 1 : 0;
        z.rows_per_cta = chunk_rpc;
        z.E = (int64_t)p * p;
        SweepMark *mg = kmark(MARK_GRAM, npass, rcd * p * (p + 1.0), 8.0 * rcd * p);
        if (mg && e == cudaSuccess) cudaEventRecord(mg->a, ax->aux);
        if (e == cudaSuccess) e = launch_ozgram(z, Gc, ax->aux);
        if (mg && e == cudaSuccess) cudaEventRecord(mg->b, ax->aux);
        g_launches++;
      }
      if (gram_whole) {
        // one Gramian of the solved block over all rows, after the last
        // chunk, on the high-priority auxiliary stream (host copies of the
        // chunks may still be running on the copy stream)
        RowSweep z = a;
        z.Yin = a.Yout;
        z.ldyin = a.ldyout;
        z.do_trsm = 0;
        z.accumulate = 0;
        z.rows_per_cta = oz_rows_per_cta;
        z.E = (int64_t)p * p;
        if (e == cudaSuccess) e = cudaEventRecord(ax->ev[0], str);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ax->aux, ax->ev[0], 0);
        SweepMark *mg = kmark(MARK_GRAM, npass, m_d * p * (p + 1.0), 8.0 * m_d * p);
        if (mg && e == cudaSuccess) cudaEventRecord(mg->a, ax->aux);
        if (e == cudaSuccess) e = launch_ozgram(z, Goz, ax->aux);
        if (mg && e == cudaSuccess) cudaEventRecord(mg->b, ax->aux);
        g_launches++;
        if (e == cudaSuccess) e = cudaEventRecord(ax->done, ax->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(str, ax->done, 0);
      } else {
        // chunks past the end of m (none with the sizing above) would leave
        // stale partials; all nchunks * Gc partials are written when rc > 0
        if (e == cudaSuccess) e = cudaEventRecord(ax->done, ax->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(str, ax->done, 0);
      }
      // the control step reads the state the copies test, and the next pass
      // overwrites the chunks they read
      if (stage && P.hQ != nullptr && e == cudaSuccess && last_c >= 0)
        e = cudaStreamWaitEvent(str, cx->c[last_c], 0);
      last_oz = true;
      last_oz_G = gram_whole ? Goz : Gc;
      if (mk != nullptr) cudaEventRecord(mk->b, str);
      return e;
    }
    if (oz && !(first && !trsm && mixed && !mixed_oz)) {
      RowSweep z = a;
      z.rows_per_cta = oz_rows_per_cta;
      z.E = (int64_t)p * p;
      if (first && !trsm && mixed_oz) {
        // the reduced-digit Gramian on the mma.sync kernel, which records
        // the column exponents for the shift
        const int64_t tiles = (P.m + ozgram_tile_rows() - 1) / ozgram_tile_rows();
        z.rows_per_cta = ((tiles + Gmix - 1) / Gmix) * ozgram_tile_rows();
        z.digits = kOzMixedDigits;
        z.emax = s.emax;
        z.tc05 = 0;
        e = cudaMemsetAsync(s.emax, 0, sizeof(int) * p, str);
        if (e == cudaSuccess) e = launch_ozgram(z, Gmix, str);
        g_launches++;
        last_oz = true;
        last_oz_G = Gmix;
        if (mk != nullptr) cudaEventRecord(mk->b, str);
        return e;
      }
      SweepMark *mg = trsm ? nullptr : kmark(MARK_GRAM, 0, m_d * p * (p + 1.0), 8.0 * m_d * p);
      if (mg) cudaEventRecord(mg->a, str);
      e = launch_ozgram(z, Goz, str);
      if (mg) cudaEventRecord(mg->b, str);
      g_launches++;
      last_oz = true;
      last_oz_G = Goz;
      if (mk != nullptr) cudaEventRecord(mk->b, str);
      return e;
    }
    if (!trsm && first && mixed) {
      RowSweep g = a;
      int tr32, lds32;
      size_t smem32;
      gram32_geometry(q, p, &tr32, &lds32, &smem32);
      g.tile_rows = tr32;
      g.lds = lds32;
      e = launch_gram32(g, G, str);
      g_launches++;
      if (mk != nullptr) cudaEventRecord(mk->b, str);
      return e;
    }
    if (wgx && !(first && !trsm && mixed)) {
      // the FP64 solve (transform only), then the Gramian of the result by
      // column blocks, reduced into C
      if (trsm && wsolve) {
        RowSweep t = a;
        t.Tinv = s.Tinv;
        t.Tscale = s.Tscale;
        e = launch_wide_solve(t, s.xwork, str);
        g_launches += 3;
      } else if (trsm) {
        RowSweep t = a;
        t.E = 0;
        e = launch_rowsweep(t, G, str);
        g_launches++;
      }
      int nl = 0;
      const double *Yg = trsm ? P.Y : a.Yin;
      const int64_t ldg = trsm ? P.ldy : a.ldyin;
      if (e == cudaSuccess) e = launch_wide_gram(Yg, ldg, P.m, p, s.partials, s.C, p, s.st, str, &nl);
      g_launches += nl;
      last_w = true;
      if (mk != nullptr) cudaEventRecord(mk->b, str);
      return e;
    }
    if (trsm && split) {
      // transform only, then a separate Gram sweep over the result
      RowSweep t = a;
      t.E = 0;
      e = launch_rowsweep(t, G, str);
      g_launches++;
      a.do_trsm = 0;
      a.Yin = P.Y;
      a.ldyin = P.ldy;
    }
    if (e == cudaSuccess) {
      e = launch_rowsweep(a, G, str);
      g_launches++;
    }
    if (mk != nullptr) cudaEventRecord(mk->b, str);
    return e;
  };
  bool red_failed = false;  // a reducer call of a sharded factorisation failed
  auto reduce_local = [&]() -> cudaError_t {
    if (last_w) return cudaSuccess;  // reduced block by block after each launch
    g_launches++;
    if (last_x) return launch_reduce_dense(s.partials, Gx, (int64_t)(q + p) * p, s.C, s.st, str);
    if (last_oz) return launch_reduce_oz(s.partials, last_oz_G, p, s.C, s.st, str);
    Reduce r{s.partials, G, E, q, p, s.C, s.st};
    return launch_reduce(r, str);
  };
  auto reduce = [&]() -> cudaError_t {
    cudaError_t e = reduce_local();
    if (e != cudaSuccess || P.red == nullptr) return e;
    // this rank's Gramian -> send; gather all ranks' blocks; sum in rank order
    const int64_t count = (int64_t)(q + p) * p;
    e = cudaMemcpyAsync(P.red->send, s.C, sizeof(double) * count, cudaMemcpyDeviceToDevice, str);
    if (e != cudaSuccess) return e;
    if (P.red->allgather(P.red->ctx, count, (void *)str) != 0) {
      red_failed = true;
      return cudaErrorUnknown;
    }
    g_launches++;
    return launch_sum_ranks(P.red->recv, P.red->world, count, s.C, str);
  };
  auto ctrl = [&]() -> cudaError_t {
    Ctrl c{};
    c.m = (P.red != nullptr) ? P.m_total : P.m;
    c.q = q;
    c.p = p;
    c.mode = P.mode;
    c.shift_policy = P.o.shift_policy;
    c.max_iter = P.o.max_iter;
    c.min_iter = P.min_iter;
    c.max_escalations = P.o.max_escalations;
    c.stop_rule = P.o.stop_rule;
    c.tol = P.o.tol;
    c.first_shift_coeff = mixed_coeff;
    c.emax = mixed_oz ? s.emax : nullptr;
    c.emax_coeff = mixed_emax_coeff;
    c.work = s.cwork;
    c.C = s.C;
    c.Rt = s.Rt;
    c.Rdinv = s.Rdinv;
    c.Bt = s.Bt;
    c.R = P.R;
    c.ldr = P.ldr;
    c.B = P.B;
    c.ldb = P.ldb;
    c.st = s.st;
    c.r_external = (P.mode == MODE_FACTOR || q == 0) ? 1 : 0;
    g_launches++;
    cudaError_t e = launch_ctrl(c, str);
    if (e == cudaSuccess && c.r_external) {
      g_launches++;
      e = launch_rupdate(s.Rt, p, P.R, P.ldr, s.st, str);
    }
    // T = D R~^{-1} for the next pass's tensor-core solve
    if (e == cudaSuccess && (gemm || wsolve)) {
      g_launches++;
      e = launch_tinv(s.Rt, s.Rdinv, s.C, q + p, q, p, s.Tinv, s.Tscale, s.st, str);
    }
    return e;
  };
  auto pass = [&](bool first) -> cudaError_t {
    cudaError_t e = sweep(true, first);
    if (e == cudaSuccess) e = reduce();
    if (e == cudaSuccess) e = ctrl();
    return e;
  };

  cudaError_t e = cudaSuccess;
  if (P.hA != nullptr) {
    // host input: one copy ahead of everything, so the first Gramian (and
    // with it the whole factorisation) is formed exactly as from device data
    e = cudaMemcpy2DAsync(const_cast<double *>(P.Y0), sizeof(double) * P.ldy0, P.hA,
                          sizeof(double) * P.ldha, sizeof(double) * P.m, p, cudaMemcpyHostToDevice, str);
  }
  if (stage) {
    for (int c = 0; c < nchunks; ++c) cx->copied[c] = -1;
    // the copy stream starts after the caller's stream has reached this point
    if (e == cudaSuccess) e = cudaEventRecord(cx->start, str);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cx->st, cx->start, 0);
  }
  if (e == cudaSuccess) e = launch_init(P.R, P.ldr, p, P.B, P.ldb, q, s.st, str);
  g_launches++;
  if (e == cudaSuccess) e = sweep(false, true);
  if (e == cudaSuccess) e = reduce();
  if (e == cudaSuccess) e = ctrl();
  int launched = 0;
  for (; e == cudaSuccess && launched < std::min(kPrelaunch, P.o.max_iter); ++launched)
    e = pass(launched == 0);
  while (e == cudaSuccess) {
    e = cudaMemcpyAsync(hs, s.st, sizeof(DevState), cudaMemcpyDeviceToHost, str);
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
    if (e != cudaSuccess || hs->done || launched >= P.o.max_iter) break;
    e = pass(launched == 0);
    ++launched;
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (stage) (void)cudaStreamSynchronize(cx->st);
    cudaFreeAsync(s.base, str);
    if (red_failed) {
      // queued work may still read the reducer's buffers: drain it first
      (void)cudaStreamSynchronize(str);
      (void)cudaGetLastError();
      return CQR_ERR_REDUCE;
    }
    return cuda_status(e);
  }
  if (!hs->done) {
    result = CQR_ERR_CUDA;  // the control kernel never concluded (cannot happen)
  } else {
    result = (cqr_status)hs->status;
    if (hs->iters == 0 && P.Y != P.Y0) {
      // loop not entered (X = I): Q = A (Alg. 1 / Alg. 2)
      e = cudaMemcpy2DAsync(P.Y, sizeof(double) * P.ldy, P.Y0, sizeof(double) * P.ldy0,
                            sizeof(double) * P.m, p, cudaMemcpyDeviceToDevice, str);
    }
  }
  if (info != nullptr) {
    info->iters = hs->iters;
    info->chol_attempts = hs->chol_attempts;
    info->shifts = hs->shifts;
    info->escalations = hs->escalations;
    info->sigma_first = hs->sigma_first;
    info->sigma_last = hs->sigma_last;
    info->orth_frob = hs->orth_frob;
    info->proj_frob = hs->proj_frob;
  }
  if (stage) {
    // the copies read the device state and Q: finish them before the
    // scratch (and the caller's buffers) can go
    cudaError_t ec = cudaStreamSynchronize(cx->st);
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess && P.hQ != nullptr && hs->done) {
      // chunks whose last copy is not of the final pass (or none ran: Q = A)
      for (int c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int64_t r0 = (int64_t)c * chunk_rows;
        const int64_t rc = std::min(chunk_rows, P.m - r0);
        if (rc <= 0 || cx->copied[c] == hs->iters) continue;
        e = cudaMemcpy2DAsync(P.hQ + r0, sizeof(double) * P.ldhq, P.Y + r0, sizeof(double) * P.ldy,
                              sizeof(double) * rc, p, cudaMemcpyDefault, str);
      }
      if (e == cudaSuccess && P.hq_written != nullptr) *P.hq_written = true;
    }
  }
  cudaError_t ef = cudaFreeAsync(s.base, str);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  if (timing && hs->done) {
    // sweeps that did work: the first Gramian sweep and passes 1 .. iters
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (size_t i = 0; i < nmarks; ++i) {
      const SweepMark &mk = pool[i];
      if (mk.pass > hs->iters) continue;
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, mk.a, mk.b) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      if (mk.kind == MARK_SOLVE) {
        g_timing.solve_launches++;
        g_timing.solve_ms += ms;
        g_timing.solve_flops += mk.flops;
        g_timing.solve_bytes += mk.bytes;
        continue;
      }
      if (mk.kind == MARK_TSOLVE) {
        g_timing.tsolve_launches++;
        g_timing.tsolve_ms += ms;
        g_timing.tsolve_flops += mk.flops;
        g_timing.tsolve_bytes += mk.bytes;
        g_timing.tsolve_tc_flops += mk.tc_flops;
        continue;
      }
      if (mk.kind == MARK_GRAM) {
        g_timing.gram_launches++;
        g_timing.gram_ms += ms;
        g_timing.gram_flops += mk.flops;
        g_timing.gram_bytes += mk.bytes;
        continue;
      }
      g_timing.sweep_launches++;
      g_timing.sweep_ms += ms;
      g_timing.sweep_flops += mk.flops;
      g_timing.sweep_bytes += mk.bytes;
      if (mk.pass > 0) {
        g_timing.fused_launches++;
        g_timing.fused_ms += ms;
        g_timing.fused_flops += mk.flops;
        g_timing.fused_bytes += mk.bytes;
      }
    }
  }
  return result;
}

}  // namespace

extern "C" {

void cqr_default_opts(cqr_opts *o) {
  if (o == nullptr) return;
  o->tol = 1e-13;
  o->max_iter = 10;
  o->min_iter = 0;
  o->update_min_iter = 2;
  o->precision = CQR_PREC_FP64;
  o->shift_policy = CQR_SHIFT_SCHOLQR3;
  o->stop_rule = CQR_STOP_FROB_TOL;
  o->max_escalations = 40;
  o->emulation = CQR_EMU_AUTO;
}

const char *cqr_status_string(int status) {
  switch (status) {
    case CQR_OK: return "ok";
    case CQR_NOT_CONVERGED: return "not converged within max_iter";
    case CQR_ERR_INVALID: return "invalid argument";
    case CQR_ERR_BREAKDOWN: return "Cholesky breakdown after all permitted shifts";
    case CQR_ERR_OOM: return "device out of memory";
    case CQR_ERR_CAPACITY: return "basis capacity exceeded";
    case CQR_ERR_CUDA: return "CUDA error";
    case CQR_ERR_TIMEOUT: return "timeout";
    case CQR_ERR_REDUCE: return "reducer failure (sharded factorisation)";
    default: return "unknown status";
  }
}

cqr_status cholqr_factor(const cqr_opts *opts, int64_t m, int64_t n, const double *A,
                         int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr,
                         cqr_info *info, void *stream) {
  cqr_opts o;
  cqr_default_opts(&o);
  if (opts != nullptr) o = *opts;
  if (!opts_valid(o)) return CQR_ERR_INVALID;
  if (n < 1 || n > CQR_MAX_N || m < n || lda < m || ldq < m || ldr < n) return CQR_ERR_INVALID;
  if (A == nullptr || Q == nullptr || R == nullptr) return CQR_ERR_INVALID;
  if (A == Q && lda != ldq) return CQR_ERR_INVALID;
  if (A != Q) {
    const char *a0 = (const char *)A, *a1 = (const char *)(A + lda * (n - 1) + m);
    const char *q0 = (const char *)Q, *q1 = (const char *)(Q + ldq * (n - 1) + m);
    if (a0 < q1 && q0 < a1) return CQR_ERR_INVALID;
  }
  if (host_state() == nullptr) return CQR_ERR_CUDA;
  Problem P{};
  P.m = m;
  P.q = 0;
  P.p = (int)n;
  P.Qin = nullptr;
  P.ldqin = 1;
  P.Y0 = A;
  P.ldy0 = lda;
  P.Y = Q;
  P.ldy = ldq;
  P.R = R;
  P.ldr = ldr;
  P.B = nullptr;
  P.ldb = 1;
  P.mode = MODE_FACTOR;
  P.min_iter = o.min_iter;
  P.o = o;
  return run(P, info, (cudaStream_t)stream);
}

cqr_status cholqr_factor_sharded(const cqr_opts *opts, int64_t m_local, int64_t m_total, int64_t n,
                                 const double *A, int64_t lda, double *Q, int64_t ldq, double *R,
                                 int64_t ldr, const cqr_reducer *red, cqr_info *info, void *stream) {
  cqr_opts o;
  cqr_default_opts(&o);
  if (opts != nullptr) o = *opts;
  if (!opts_valid(o)) return CQR_ERR_INVALID;
  if (red == nullptr || red->world < 1 || red->rank < 0 || red->rank >= red->world ||
      red->allgather == nullptr || red->send == nullptr || red->recv == nullptr)
    return CQR_ERR_INVALID;
  if (n < 1 || n > CQR_MAX_N || m_local < 1 || m_total < n || m_local > m_total || lda < m_local ||
      ldq < m_local || ldr < n || red->capacity < n * n)
    return CQR_ERR_INVALID;
  if (A == nullptr || Q == nullptr || R == nullptr) return CQR_ERR_INVALID;
  if (A == Q && lda != ldq) return CQR_ERR_INVALID;
  if (A != Q) {
    const char *a0 = (const char *)A, *a1 = (const char *)(A + lda * (n - 1) + m_local);
    const char *q0 = (const char *)Q, *q1 = (const char *)(Q + ldq * (n - 1) + m_local);
    if (a0 < q1 && q0 < a1) return CQR_ERR_INVALID;
  }
  if (host_state() == nullptr) return CQR_ERR_CUDA;
  Problem P{};
  P.m = m_local;
  P.q = 0;
  P.p = (int)n;
  P.Qin = nullptr;
  P.ldqin = 1;
  P.Y0 = A;
  P.ldy0 = lda;
  P.Y = Q;
  P.ldy = ldq;
  P.R = R;
  P.ldr = ldr;
  P.B = nullptr;
  P.ldb = 1;
  P.mode = MODE_FACTOR;
  P.min_iter = o.min_iter;
  P.o = o;
  P.red = red;
  P.m_total = m_total;
  return run(P, info, (cudaStream_t)stream);
}

cqr_status cholqr_gram(const cqr_opts *opts, int64_t m, int64_t n, const double *A, int64_t lda,
                       double *X, int64_t ldx, void *stream) {
  cqr_opts o;
  cqr_default_opts(&o);
  if (opts != nullptr) o = *opts;
  if (!opts_valid(o)) return CQR_ERR_INVALID;
  if (n < 1 || n > CQR_MAX_N || m < 1 || lda < m || ldx < n) return CQR_ERR_INVALID;
  if (A == nullptr || X == nullptr) return CQR_ERR_INVALID;
  cudaStream_t str = (cudaStream_t)stream;
  const int p = (int)n;
  const bool oz = (p <= kOzMaxN) && (o.emulation != CQR_EMU_OFF);
  int tile_rows, lds;
  size_t smem;
  rowsweep_geometry(0, p, &tile_rows, &lds, &smem);
  // CQR_PREC_MIXED: the Gramian of the mixed factorisation's first pass
  // (reduced-digit on the tensor cores, or FP32 with emulation off)
  const bool mixed = o.precision == CQR_PREC_MIXED;
  const bool tc05 = tc05_gram_mode(o.emulation, p) && !mixed;
  // wider than the digit Gramian: by column blocks, as the factorisation
  const bool wide = (p > kOzMaxN) && (o.emulation != CQR_EMU_OFF) && !mixed;
  const int G = oz ? ozgram_grid(m, p, tc05) : rowsweep_grid(m, tile_rows);
  const int64_t tr = oz ? ozgram_tile_rows() : tile_rows;
  const int64_t tiles = (m + tr - 1) / tr;
  const int64_t rows_per_cta = ((tiles + G - 1) / G) * tr;
  const int64_t E0 = oz ? (int64_t)p * p : (int64_t)p * (p + 1) / 2;
  const int64_t E = wide ? std::max<int64_t>(E0, (wide_gram_partial_elems(m, p) + G - 1) / G) : E0;
  Scratch s;
  CQR_TRY(scratch_alloc(s, 0, p, G, E, str));
  RowSweep a{};
  a.m = m;
  a.q = 0;
  a.p = p;
  a.Yin = A;
  a.ldyin = lda;
  a.partials = s.partials;
  a.E = E;
  a.rows_per_cta = rows_per_cta;
  a.tile_rows = tile_rows;
  a.lds = lds;
  a.do_trsm = 0;
  a.st = nullptr;
  a.tc05 = tc05 ? kTc05Gram : 0;
  cudaError_t e = cudaSuccess;
  if (oz) {
    if (mixed) {
      a.digits = kOzMixedDigits;
      a.emax = s.emax;
      e = cudaMemsetAsync(s.emax, 0, sizeof(int) * p, str);
    }
    if (e == cudaSuccess) e = launch_ozgram(a, G, str);
  } else if (wide) {
    int nl = 0;
    e = launch_wide_gram(A, lda, m, p, s.partials, s.C, p, nullptr, str, &nl);
    g_launches += nl - 1;
  } else if (mixed) {
    size_t smem32;
    gram32_geometry(0, p, &a.tile_rows, &a.lds, &smem32);
    e = launch_gram32(a, G, str);
  } else {
    e = launch_rowsweep(a, G, str);
  }
  g_launches++;
  if (e == cudaSuccess && !wide) {
    if (oz) {
      e = launch_reduce_oz(s.partials, G, p, s.C, nullptr, str);
    } else {
      Reduce r{s.partials, G, E, 0, p, s.C, nullptr};
      e = launch_reduce(r, str);
    }
    g_launches++;
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(X, sizeof(double) * ldx, s.C, sizeof(double) * p, sizeof(double) * p, p,
                          cudaMemcpyDeviceToDevice, str);
  cudaError_t ef = cudaFreeAsync(s.base, str);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  return CQR_OK;
}

cqr_status cholqr_factor_host(const cqr_opts *opts, int64_t m, int64_t n, const double *A,
                              int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr,
                              cqr_info *info, void *stream) {
  cqr_opts o;
  cqr_default_opts(&o);
  if (opts != nullptr) o = *opts;
  if (!opts_valid(o)) return CQR_ERR_INVALID;
  if (n < 1 || n > CQR_MAX_N || m < n || lda < m || ldq < m || ldr < n) return CQR_ERR_INVALID;
  if (A == nullptr || Q == nullptr || R == nullptr) return CQR_ERR_INVALID;
  {
    // Q is written while A may still be read (the copy-out of the last pass)
    const char *a0 = (const char *)A, *a1 = (const char *)(A + lda * (n - 1) + m);
    const char *q0 = (const char *)Q, *q1 = (const char *)(Q + ldq * (n - 1) + m);
    if (a0 < q1 && q0 < a1) return CQR_ERR_INVALID;
  }
  if (host_state() == nullptr) return CQR_ERR_CUDA;
  cudaStream_t str = (cudaStream_t)stream;
  keep_pool_memory();
  // Q written by the device as each pass ends needs page-locked host memory
  // the device can address
  double *dQh = nullptr;
  {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, Q) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr)
      dQh = (double *)at.devicePointer;
    (void)cudaGetLastError();
  }
  double *dA = nullptr, *dR = nullptr;
  const int64_t ldd = m;
  CQR_TRY(cudaMallocAsync((void **)&dA, sizeof(double) * (size_t)m * n, str));
  cudaError_t e = cudaMallocAsync((void **)&dR, sizeof(double) * (size_t)n * n, str);
  if (e != cudaSuccess) {
    cudaFreeAsync(dA, str);
    return cuda_status(e);
  }
  bool q_written = false;
  Problem P{};
  P.m = m;
  P.q = 0;
  P.p = (int)n;
  P.Qin = nullptr;
  P.ldqin = 1;
  P.Y0 = dA;
  P.ldy0 = ldd;
  P.Y = dA;
  P.ldy = ldd;
  P.R = dR;
  P.ldr = n;
  P.B = nullptr;
  P.ldb = 1;
  P.mode = MODE_FACTOR;
  P.min_iter = o.min_iter;
  P.o = o;
  P.hA = A;
  P.ldha = lda;
  P.hQ = dQh;
  P.ldhq = ldq;
  P.hq_written = &q_written;
  cqr_status st = run(P, info, str);
  if (st >= 0) {
    e = cudaSuccess;
    if (!q_written)
      e = cudaMemcpy2DAsync(Q, sizeof(double) * ldq, dA, sizeof(double) * ldd, sizeof(double) * m, n,
                            cudaMemcpyDeviceToHost, str);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(R, sizeof(double) * ldr, dR, sizeof(double) * n, sizeof(double) * n, n,
                            cudaMemcpyDeviceToHost, str);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  cudaFreeAsync(dA, str);
  cudaFreeAsync(dR, str);
  e = cudaStreamSynchronize(str);
  if (e != cudaSuccess && st >= 0) st = cuda_status(e);
  (void)cudaGetLastError();
  return st;
}

cqr_status basis_create(int64_t m, int64_t n_max, const cqr_opts *opts, void *stream,
                        cqr_basis **out) {
  if (out == nullptr) return CQR_ERR_INVALID;
  *out = nullptr;
  cqr_opts o;
  cqr_default_opts(&o);
  if (opts != nullptr) o = *opts;
  if (!opts_valid(o)) return CQR_ERR_INVALID;
  if (m < 1 || n_max < 1 || n_max > CQR_MAX_BASIS) return CQR_ERR_INVALID;
  cqr_basis *b = (cqr_basis *)calloc(1, sizeof(cqr_basis));
  if (b == nullptr) return CQR_ERR_OOM;
  cudaGetDevice(&b->device);
  b->m = m;
  b->n_max = n_max;
  b->q = 0;
  b->ldq = (m + 1) & ~(int64_t)1;
  b->ldr = n_max;
  b->opts = o;
  cudaError_t e = cudaMalloc((void **)&b->Q, sizeof(double) * (size_t)b->ldq * n_max);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->R, sizeof(double) * (size_t)n_max * n_max);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->R, 0, sizeof(double) * (size_t)n_max * n_max, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (b->Q) cudaFree(b->Q);
    if (b->R) cudaFree(b->R);
    free(b);
    return cuda_status(e);
  }
  *out = b;
  return CQR_OK;
}

cqr_status basis_append(cqr_basis *b, int64_t p, const double *A_in, int64_t lda,
                        cqr_info *info, void *stream) {
  if (b == nullptr || A_in == nullptr) return CQR_ERR_INVALID;
  if (p < 1 || p > CQR_MAX_N || lda < b->m) return CQR_ERR_INVALID;
  if (b->q + p > b->n_max) return CQR_ERR_CAPACITY;
  {
    const char *a0 = (const char *)A_in, *a1 = (const char *)(A_in + lda * (p - 1) + b->m);
    const char *q0 = (const char *)b->Q, *q1 = (const char *)(b->Q + b->ldq * b->n_max);
    if (a0 < q1 && q0 < a1) return CQR_ERR_INVALID;
  }
  if (host_state() == nullptr) return CQR_ERR_CUDA;
  const int64_t q = b->q;
  Problem P{};
  P.m = b->m;
  P.q = (int)q;
  P.p = (int)p;
  P.Qin = b->Q;
  P.ldqin = b->ldq;
  P.Y0 = A_in;
  P.ldy0 = lda;
  P.Y = b->Q + q * b->ldq;
  P.ldy = b->ldq;
  P.R = b->R + q + q * b->ldr;
  P.ldr = b->ldr;
  P.B = (q > 0) ? b->R + q * b->ldr : nullptr;
  P.ldb = b->ldr;
  P.mode = MODE_UPDATE;
  P.min_iter = b->opts.update_min_iter;
  P.o = b->opts;
  if (b->Qd != nullptr) {
    P.Qd = b->Qd;
    P.Qe = b->Qe;
    P.ldc = b->ldc;
    P.cplane = b->ldc * b->n_max;
  }
  cqr_status st = run(P, info, (cudaStream_t)stream);
  if (st == CQR_OK || st == CQR_NOT_CONVERGED) {
    if (b->Qd != nullptr) {
      // the new columns join the digit cache before anything can read them
      cudaError_t e = launch_cache_fill(b->Q, b->ldq, b->m, (int)q, (int)p, b->Qe, b->Qd, b->ldc,
                                        b->ldc * b->n_max, (cudaStream_t)stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return cuda_status(e);  // the basis keeps its previous q columns
      }
    }
    b->q = q + p;
  }
  return st;
}

cqr_status basis_enable_digit_cache(cqr_basis *b, void *stream) {
  if (b == nullptr) return CQR_ERR_INVALID;
  if (b->Qd != nullptr) return CQR_OK;
  const int64_t ldc = (b->m + 63) & ~(int64_t)63;
  uint16_t *Qd = nullptr;
  int *Qe = nullptr;
  cudaError_t e = cudaMalloc((void **)&Qd, sizeof(uint16_t) * 7 * (size_t)ldc * b->n_max);
  if (e == cudaSuccess) e = cudaMalloc((void **)&Qe, sizeof(int) * (size_t)b->n_max);
  if (e == cudaSuccess && b->q > 0)
    e = launch_cache_fill(b->Q, b->ldq, b->m, 0, (int)b->q, Qe, Qd, ldc, ldc * b->n_max, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (Qd) cudaFree(Qd);
    if (Qe) cudaFree(Qe);
    return cuda_status(e);
  }
  b->Qd = Qd;
  b->Qe = Qe;
  b->ldc = ldc;
  return CQR_OK;
}

cqr_status cholqr_pn(const cqr_opts *opts, int64_t m, int64_t n, int64_t r, const double *A,
                     int64_t lda, double *Q, int64_t ldq, double *R, int64_t ldr, cqr_info *info,
                     void *stream) {
  cqr_opts o;
  cqr_default_opts(&o);
  if (opts != nullptr) o = *opts;
  if (!opts_valid(o)) return CQR_ERR_INVALID;
  if (n < 1 || n > CQR_MAX_BASIS || r < 1 || r > n || m < n) return CQR_ERR_INVALID;
  if ((n + r - 1) / r > CQR_MAX_N) return CQR_ERR_INVALID;
  if (lda < m || ldq < m || ldr < n) return CQR_ERR_INVALID;
  if (A == nullptr || Q == nullptr || R == nullptr) return CQR_ERR_INVALID;
  {
    const char *a0 = (const char *)A, *a1 = (const char *)(A + lda * (n - 1) + m);
    const char *q0 = (const char *)Q, *q1 = (const char *)(Q + ldq * (n - 1) + m);
    if (a0 < q1 && q0 < a1) return CQR_ERR_INVALID;
  }
  if (host_state() == nullptr) return CQR_ERR_CUDA;
  cudaStream_t str = (cudaStream_t)stream;
  cudaError_t e = cudaMemset2DAsync(R, sizeof(double) * ldr, 0, sizeof(double) * n, n, str);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  // Panels of <= 16 columns on a tall block keep a transient digit cache of
  // the columns already factored (as a basis with basis_enable_digit_cache):
  // their cross Gramian and projection then run on the tensor cores.
  const int64_t pmax = (n + r - 1) / r;
  uint16_t *Qd = nullptr;
  int *Qe = nullptr;
  const int64_t ldc = (m + 63) & ~(int64_t)63;
  if (r > 1 && pmax <= kOzCacheMaxP && m > kOzUpdMinRows && o.emulation != CQR_EMU_OFF) {
    if (cudaMallocAsync((void **)&Qd, sizeof(uint16_t) * 7 * (size_t)ldc * n, str) != cudaSuccess ||
        cudaMallocAsync((void **)&Qe, sizeof(int) * (size_t)n, str) != cudaSuccess) {
      (void)cudaGetLastError();  // no cache: the panels keep the FP64 path
      if (Qd) cudaFreeAsync(Qd, str);
      Qd = nullptr;
      Qe = nullptr;
    }
  }
  cqr_info tot{};
  cqr_status status = CQR_OK;
  int64_t q = 0;
  for (int64_t k = 0; k < r; ++k) {
    const int64_t p = n / r + (k < n % r ? 1 : 0);
    // panel k = columns q .. q+p-1 of A, appended to Q's first q columns
    Problem P{};
    P.m = m;
    P.q = (int)q;
    P.p = (int)p;
    P.Qin = Q;
    P.ldqin = ldq;
    P.Y0 = A + q * lda;
    P.ldy0 = lda;
    P.Y = Q + q * ldq;
    P.ldy = ldq;
    P.R = R + q + q * ldr;
    P.ldr = ldr;
    P.B = (q > 0) ? R + q * ldr : nullptr;
    P.ldb = ldr;
    P.mode = MODE_UPDATE;
    P.min_iter = o.update_min_iter;
    P.o = o;
    if (Qd != nullptr) {
      P.Qd = Qd;
      P.Qe = Qe;
      P.ldc = ldc;
      P.cplane = ldc * n;
    }
    cqr_info pi{};
    const cqr_status st = run(P, &pi, str);
    tot.iters += pi.iters;
    tot.chol_attempts += pi.chol_attempts;
    tot.shifts += pi.shifts;
    tot.escalations += pi.escalations;
    if (tot.sigma_first == 0.0) tot.sigma_first = pi.sigma_first;
    if (pi.sigma_last != 0.0) tot.sigma_last = pi.sigma_last;
    tot.orth_frob = pi.orth_frob;
    tot.proj_frob = pi.proj_frob;
    if (st < 0) {
      status = st;
      break;
    }
    if (st == CQR_NOT_CONVERGED) status = CQR_NOT_CONVERGED;
    if (Qd != nullptr && k + 1 < r) {
      // the panel's columns join the cache before the next panel reads it
      cudaError_t e = launch_cache_fill(Q, ldq, m, (int)q, (int)p, Qe, Qd, ldc, ldc * n, str);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        status = cuda_status(e);
        break;
      }
    }
    q += p;
  }
  if (Qd != nullptr) {
    cudaFreeAsync(Qd, str);
    cudaFreeAsync(Qe, str);
    if (cudaStreamSynchronize(str) != cudaSuccess && status >= 0) status = CQR_ERR_CUDA;
    (void)cudaGetLastError();
  }
  if (info != nullptr) *info = tot;
  return status;
}

cqr_status basis_free(cqr_basis *b) {
  if (b == nullptr) return CQR_OK;
  if (b->Qd != nullptr) cudaFree(b->Qd);
  if (b->Qe != nullptr) cudaFree(b->Qe);
  cudaError_t e1 = cudaFree(b->Q);
  cudaError_t e2 = cudaFree(b->R);
  free(b);
  if (e1 != cudaSuccess) return cuda_status(e1);
  return cuda_status(e2);
}

cqr_status cqr_timing_enable(int enable) {
  g_timing_on.store(enable ? 1 : 0);
  return CQR_OK;
}

cqr_status cqr_timing_read(cqr_timing *out) {
  if (out == nullptr) return CQR_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  *out = g_timing;
  out->kernel_launches = g_launches.load();
  return CQR_OK;
}

void cqr_timing_reset(void) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timing = cqr_timing{};
  g_launches.store(0);
}

int64_t basis_cols(const cqr_basis *b) { return b ? b->q : -1; }
int64_t basis_rows(const cqr_basis *b) { return b ? b->m : -1; }
int64_t basis_capacity(const cqr_basis *b) { return b ? b->n_max : -1; }

cqr_status basis_q(const cqr_basis *b, const double **Q, int64_t *ldq) {
  if (b == nullptr || Q == nullptr || ldq == nullptr) return CQR_ERR_INVALID;
  *Q = b->Q;
  *ldq = b->ldq;
  return CQR_OK;
}

cqr_status basis_r(const cqr_basis *b, const double **R, int64_t *ldr) {
  if (b == nullptr || R == nullptr || ldr == nullptr) return CQR_ERR_INVALID;
  *R = b->R;
  *ldr = b->ldr;
  return CQR_OK;
}

}  // extern "C"
