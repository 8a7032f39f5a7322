// cholqr_factor_noalloc: the sCholQR3 factorisation with every byte of its
// device scratch taken from one fixed array compiled into this library,
// for callers that cannot allocate device memory.
//
// Who cannot allocate: processes that have already handed all device memory
// to their own allocator (a framework caching allocator, or a serving loop
// that admits work against a fixed HBM budget), where a library-side
// cudaMalloc could fail or fragment their pool; and latency-critical loops
// that must never pay for, or risk the failure of, an allocation inside a
// call.  This entry point calls no cudaMalloc, cudaMallocAsync, cudaFree,
// cudaMallocHost or any other allocating routine.
//
// What it runs: the FP64 CUDA-core path of cholqr_factor (the path that
// cholqr_factor takes with opts->emulation = CQR_EMU_OFF): the fused row
// sweep (triangular solve + Gramian), its fixed-order reduction and the
// control kernel, with the same launch geometry, so its Q and R are bitwise
// those of cholqr_factor with CQR_EMU_OFF.  The tensor-core pipeline needs
// per-chunk partials and an auxiliary stream that do not fit this scheme;
// opts->emulation is therefore ignored (both values run the FP64 path) and
// opts->precision = CQR_PREC_MIXED is rejected with CQR_ERR_INVALID.
//
// The scratch array below (kNoAllocScratchBytes, 8 MiB) is part of the
// library's device image: every GPU that loads the library holds it until
// the process exits.  It holds the device state, the reduced Gramian, R~,
// 1/diag(R~) and the per-CTA partial sums of the row sweeps, which limits
// this entry point to n <= 64 (larger n returns CQR_ERR_CAPACITY).
//
// Its device address is looked up with cudaGetSymbolAddress on every call,
// with the current device (which must hold A, Q and R) current: the lookup
// allocates nothing, and a cached address could go stale after the module
// is reloaded (a device reset).
//
// All calls share the one array and it keeps the last call's contents.  Each
// call starts with the init kernel, which clears the device state; the
// partial sums, the reduced Gramian and R~ are fully rewritten before they
// are read, so no other clearing is needed.  Calls whose work overlaps on
// the GPU (for example on two streams at once) race on the array: the caller
// must serialise them.
#include <string.h>

#include <algorithm>

#include "cqr_internal.cuh"

using namespace cqr;

namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr int kNoAllocMaxN = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory; the device address comes from cudaGetSymbolAddress with the
// device that runs the call current.
cudaError_t scratch_address(void **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (p == nullptr) return cudaErrorInvalidSymbol;
  *out = p;
  return cudaSuccess;
}

// True when ptr is device (or managed) memory that the current device `dev`
// can use as this call's operand: memory of another device is rejected, as
// is host memory.
bool on_device(const void *ptr, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

cqr_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return CQR_OK;
  if (e == cudaErrorMemoryAllocation) return CQR_ERR_OOM;
  return CQR_ERR_CUDA;
}

}  // namespace

extern "C" cqr_status cholqr_factor_noalloc(const cqr_opts *opts, int64_t m, int64_t n,
                                            const double *A, int64_t lda, double *Q, int64_t ldq,
                                            double *R, int64_t ldr, cqr_info *info,
                                            void *stream) {
  cqr_opts o;
  cqr_default_opts(&o);
  if (opts != nullptr) o = *opts;
  const bool opts_ok =
      o.tol >= 0.0 && o.max_iter >= 1 && o.max_iter <= 100 && o.min_iter >= 0 &&
      o.max_escalations >= 0 && o.max_escalations <= 400 &&
      o.precision == CQR_PREC_FP64 &&
      o.shift_policy >= CQR_SHIFT_SCHOLQR3 && o.shift_policy <= CQR_SHIFT_ISCHOLQR &&
      (o.stop_rule == CQR_STOP_FROB_TOL || o.stop_rule == CQR_STOP_U_SQRT_N) &&
      (o.emulation == CQR_EMU_AUTO || o.emulation == CQR_EMU_OFF || o.emulation == CQR_EMU_TCGEN05);
  if (!opts_ok) return CQR_ERR_INVALID;
  if (n < 1 || m < n || lda < m || ldq < m || ldr < n) return CQR_ERR_INVALID;
  if (A == nullptr || Q == nullptr || R == nullptr) return CQR_ERR_INVALID;
  if (A == Q && lda != ldq) return CQR_ERR_INVALID;
  if (A != Q) {
    const char *a0 = (const char *)A, *a1 = (const char *)(A + lda * (n - 1) + m);
    const char *q0 = (const char *)Q, *q1 = (const char *)(Q + ldq * (n - 1) + m);
    if (a0 < q1 && q0 < a1) return CQR_ERR_INVALID;
  }
  if (n > kNoAllocMaxN) return CQR_ERR_CAPACITY;

  const int p = (int)n;
  int tile_rows, lds;
  size_t smem;
  rowsweep_geometry(0, p, &tile_rows, &lds, &smem);
  const int G = rowsweep_grid(m, tile_rows);
  const int64_t tiles = (m + tile_rows - 1) / tile_rows;
  const int64_t rows_per_cta = ((tiles + G - 1) / G) * tile_rows;
  const int64_t E = (int64_t)p * (p + 1) / 2;

  const size_t b_st = a256(sizeof(DevState));
  const size_t b_C = a256(sizeof(double) * (size_t)p * p);
  const size_t b_Rt = a256(sizeof(double) * (size_t)p * p);
  const size_t b_Rd = a256(sizeof(double) * (size_t)p);
  const size_t b_Bt = a256(sizeof(double) * (size_t)p);
  const size_t b_P = a256(sizeof(double) * (size_t)G * (size_t)E);
  if (b_st + b_C + b_Rt + b_Rd + b_Bt + b_P > kNoAllocScratchBytes) return CQR_ERR_CAPACITY;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return to_status(e);
  }
  if (!on_device(A, dev) || !on_device(Q, dev) || !on_device(R, dev)) return CQR_ERR_INVALID;
  void *base = nullptr;
  e = scratch_address(&base);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return to_status(e);
  }
  char *c0 = (char *)base;
  DevState *st = (DevState *)c0;
  c0 += b_st;
  double *Cm = (double *)c0;
  c0 += b_C;
  double *Rt = (double *)c0;
  c0 += b_Rt;
  double *Rdinv = (double *)c0;
  c0 += b_Rd;
  double *Bt = (double *)c0;
  c0 += b_Bt;
  double *partials = (double *)c0;

  cudaStream_t str = (cudaStream_t)stream;
  auto sweep = [&](bool trsm, bool first) -> cudaError_t {
    RowSweep a{};
    a.m = m;
    a.q = 0;
    a.p = p;
    a.Qin = nullptr;
    a.ldqin = 1;
    a.Yin = first ? A : Q;
    a.ldyin = first ? lda : ldq;
    a.Yout = Q;
    a.ldyout = ldq;
    a.Rt = Rt;
    a.Rdinv = Rdinv;
    a.Bt = Bt;
    a.partials = partials;
    a.E = E;
    a.rows_per_cta = rows_per_cta;
    a.tile_rows = tile_rows;
    a.lds = lds;
    a.do_trsm = trsm ? 1 : 0;
    a.st = st;
    return launch_rowsweep(a, G, str);
  };
  auto reduce = [&]() -> cudaError_t {
    Reduce r{partials, G, E, 0, p, Cm, st};
    return launch_reduce(r, str);
  };
  auto ctrl = [&]() -> cudaError_t {
    Ctrl c{};
    c.m = m;
    c.q = 0;
    c.p = p;
    c.mode = MODE_FACTOR;
    c.shift_policy = o.shift_policy;
    c.max_iter = o.max_iter;
    c.min_iter = o.min_iter;
    c.max_escalations = o.max_escalations;
    c.stop_rule = o.stop_rule;
    c.tol = o.tol;
    c.C = Cm;
    c.Rt = Rt;
    c.Rdinv = Rdinv;
    c.Bt = Bt;
    c.R = R;
    c.ldr = ldr;
    c.B = nullptr;
    c.ldb = 1;
    c.st = st;
    return launch_ctrl(c, str);
  };

  e = launch_init(R, ldr, p, nullptr, 1, 0, st, str);
  if (e == cudaSuccess) e = sweep(false, true);
  if (e == cudaSuccess) e = reduce();
  if (e == cudaSuccess) e = ctrl();
  DevState hs;
  memset(&hs, 0, sizeof(hs));
  int launched = 0;
  for (; e == cudaSuccess && launched < std::min(3, o.max_iter); ++launched) {
    e = sweep(true, launched == 0);
    if (e == cudaSuccess) e = reduce();
    if (e == cudaSuccess) e = ctrl();
  }
  while (e == cudaSuccess) {
    // pageable host destination: a plain copy, no pinned buffer is allocated
    e = cudaMemcpyAsync(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost, str);
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
    if (e != cudaSuccess || hs.done || launched >= o.max_iter) break;
    e = sweep(true, launched == 0);
    if (e == cudaSuccess) e = reduce();
    if (e == cudaSuccess) e = ctrl();
    ++launched;
  }
  if (e == cudaSuccess && hs.done && hs.iters == 0 && Q != A) {
    e = cudaMemcpy2DAsync(Q, sizeof(double) * ldq, A, sizeof(double) * lda, sizeof(double) * m,
                          n, cudaMemcpyDeviceToDevice, str);
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return to_status(e);
  }
  if (info != nullptr) {
    info->iters = hs.iters;
    info->chol_attempts = hs.chol_attempts;
    info->shifts = hs.shifts;
    info->escalations = hs.escalations;
    info->sigma_first = hs.sigma_first;
    info->sigma_last = hs.sigma_last;
    info->orth_frob = hs.orth_frob;
    info->proj_frob = hs.proj_frob;
  }
  if (!hs.done) return CQR_ERR_CUDA;
  return (cqr_status)hs.status;
}
