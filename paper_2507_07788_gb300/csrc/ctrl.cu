// Single-CTA control kernel: the small n x n (or p x p) steps of one pass.
//
// Reads the reduced Gramian C = [Q_in Y]^T Y and performs, for one pass of
// Alg. 1 (MODE_FACTOR) or one outer iteration of Alg. 2 (MODE_UPDATE):
//   X = Y^T Y - B~^T B~             (Alg. 2; B~ empty for Alg. 1)
//   stop test ||X - I||_F < tol     (Alg. 1, Alg. 2, Sec. 4.1)
//   shift and Cholesky with breakdown detection and retry
//                                   (Alg. 1, Alg. 2)
//   R~ and 1/diag(R~) for the row sweep, B <- B + B~ R, R <- R~ R
//                                   (Alg. 1, Alg. 2)
// Every loop is bounded (max_iter passes, max_escalations shift retries,
// kPowerMaxIter power iterations), so the kernel always terminates; a failure is
// recorded in the device state and stops all later kernels of the call.
#include <math.h>

#include <atomic>
#include <mutex>

#include "cqr_internal.cuh"

namespace cqr {

constexpr int kCqrMaxN = CQR_MAX_N;
constexpr int kTinvMaxN = 128;  // widths of the tensor-core solve, whose T the tinv kernel forms
constexpr int kPowerMaxIter = 300;  // power iterations of the norm estimate

__device__ __forceinline__ int pk(int i, int j) { return i + j * (j + 1) / 2; }  // i <= j

// Sum over the block, fixed butterfly + fixed warp order: deterministic.
__device__ double block_sum(double v, double *red) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < nw; ++k) s += red[k];
  __syncthreads();
  return s;
}

__device__ float block_sumf(float v, float *red) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float s = 0.0f;
  for (int k = 0; k < nw; ++k) s += red[k];
  __syncthreads();
  return s;
}

// FP64 -> FP32 by truncation of the bit pattern (integer pipe only; the
// GB300 FP64 unit is slow and the norm estimate needs ~1e-3 accuracy).
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
  if (e < -126) return __int_as_float((int)sign);
  if (e > 127) return __int_as_float((int)(sign | 0x7F800000u));
  const unsigned mant = (unsigned)((b >> 29) & 0x7FFFFFull);
  return __int_as_float((int)(sign | ((unsigned)(e + 127) << 23) | mant));
}

// Estimate of ||X||_2 for symmetric X (the norm in the shifts of Alg. 1 and
// Alg. 2, which the paper computes with a Lanczos solver at tolerance 1e-2
// starting from the all-ones vector).  Power iteration in FP32 from the
// all-ones vector, stopped when the part of the Rayleigh quotient still
// missing, extrapolated from the ratio of its last two increments, is below
// 1e-3 relative, or an increment is at FP32 resolution (at most
// kPowerMaxIter steps); the result is never below max_i |X_ii|.
// X enters the FP32 iteration scaled by 2^-e, e the exponent of max_i |X_ii|
// (exact, so the iteration is the same as on X itself wherever X fits FP32),
// which keeps Gramians of norm beyond the FP32 range (||A|| > 2^64) or
// below its normal range finite and accurate.
__device__ double norm_estimate(const double *X, int p, float *Xf, float *v, float *w,
                                float *fred, double *red) {
  const int t = threadIdx.x, NT = blockDim.x;
  __syncthreads();  // Xf may alias storage read just before the call
  if (t < 32) {
    double mv = 0.0;
    for (int i = t; i < p; i += 32) mv = fmax(mv, fabs(X[i + i * p]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
    if (t == 0) red[31] = mv;
  }
  __syncthreads();
  const double dmax = red[31];
  // 2^-e and 2^e for a finite, non-zero diagonal maximum (else 1)
  int ex = 0;
  if (dmax > 0.0 && dmax <= 1.7976931348623157e308)
    ex = (int)((__double_as_longlong(dmax) >> 52) & 0x7FF) - 1023;
  const double down = ldexp(1.0, -ex), up = ldexp(1.0, ex);
  for (int e = t; e < p * p; e += NT) Xf[e] = d2f_trunc(X[e] * down);
  __syncthreads();
  const float inv = rsqrtf((float)p);
  for (int i = t; i < p; i += NT) v[i] = inv;
  __syncthreads();
  float lam = 0.0f, lam_prev = 0.0f, dprev = 0.0f;
  for (int it = 0; it < kPowerMaxIter; ++it) {
    float part_l = 0.0f, part_n = 0.0f;
    for (int i = t; i < p; i += NT) {
      float s = 0.0f;
      for (int j = 0; j < p; ++j) s = fmaf(Xf[i + j * p], v[j], s);
      w[i] = s;
      part_l += v[i] * s;
      part_n += s * s;
    }
    lam = block_sumf(part_l, fred);
    const float nrm = sqrtf(block_sumf(part_n, fred));
    if (!(nrm > 0.0f) || !isfinite(nrm)) break;
    const float rn = 1.0f / nrm;
    for (int i = t; i < p; i += NT) v[i] = w[i] * rn;
    __syncthreads();
    if (it > 0) {
      // the increments of the Rayleigh quotient shrink geometrically (ratio
      // rho, the squared ratio of the two largest eigenvalues): the part
      // still missing is about d rho / (1 - rho), which a close second
      // eigenvalue makes far larger than the last increment d
      const float d = fabsf(lam - lam_prev);
      if (d <= 1e-6f * fabsf(lam)) break;  // at FP32 resolution
      if (it > 1 && d < dprev && d * (d / dprev) <= 1e-3f * (1.0f - d / dprev) * fabsf(lam)) break;
      dprev = d;
    }
    lam_prev = lam;
  }
  double l = (double)lam * up;
  if (!(l == l)) l = INFINITY;
  return fmax(l, dmax);
}

// Cholesky R^T R = X + sigma I into packed upper storage Rk, right-looking:
// Rk starts as the upper triangle of X + sigma I; step j takes the pivot
// d_j = the updated (j, j) entry, scales row j by 1 / sqrt(d_j) and
// subtracts R_ji R_jk from the trailing entries (i, k), j < i <= k.  Each
// entry thus receives X_ik - R_0i R_0k - R_1i R_1k - ... in increasing j.
// Breakdown: d_j not strictly positive or not finite.  Returns 0 or j + 1 of
// the failing pivot.  All of the block's threads share the trailing update
// (8 lanes per column), so a step costs one FP64 instruction per entry.
__device__ int cholesky(const double *X, int p, double sigma, double *Rk, double *s_inv,
                        int *s_fail) {
  const int t = threadIdx.x, NT = blockDim.x;
  __syncthreads();  // every thread has read the previous call's *s_fail
  for (int e = t; e < p * p; e += NT) {
    const int i = e % p, j = e / p;
    if (i <= j) Rk[pk(i, j)] = X[i + j * p] + (i == j ? sigma : 0.0);
  }
  if (t == 0) *s_fail = 0;
  __syncthreads();
  const int cl = t >> 3, rl = t & 7, cstep = NT >> 3;
  for (int j = 0; j < p; ++j) {
    if (t == 0) {
      const double d = Rk[pk(j, j)];
      if (!(d > 0.0) || !isfinite(d)) {
        *s_fail = j + 1;
      } else {
        const double r = sqrt(d);
        Rk[pk(j, j)] = r;
        *s_inv = 1.0 / r;
      }
    }
    __syncthreads();
    if (*s_fail) return *s_fail;
    const double inv = *s_inv;
    for (int k = j + 1 + t; k < p; k += NT) Rk[pk(j, k)] *= inv;
    __syncthreads();
    // trailing update of column k (rows j < i <= k) by its 8 lanes
    for (int k = j + 1 + cl; k < p; k += cstep) {
      const double rjk = Rk[pk(j, k)];
      for (int i = j + 1 + rl; i <= k; i += 8) Rk[pk(i, k)] -= Rk[pk(j, i)] * rjk;
    }
    __syncthreads();
  }
  return 0;
}

__device__ __forceinline__ double shift_alg1(int64_t m, int n, double normX) {
  const double c = 11.0 * ((double)m * (double)n + (double)n * ((double)n + 1.0));
  return fmax(c * kU64 * normX, 2.0 * kU64);
}

__device__ __forceinline__ double shift_alg2_first(int64_t m, int q, int p, double normX) {
  if (q == 0) return shift_alg1(m, p, normX);
  const double c = 11.0 * ((double)m * (double)q + (double)q * ((double)q + 1.0));
  return c * kU64 * normX;
}

// The Cholesky of the control step on the calling CTA alone.
struct LocalChol {
  __device__ int operator()(const double *X, int p, double sigma, double *Rk, double *s_inv, int *s_fail) const {
    return cholesky(X, p, sigma, Rk, s_inv, s_fail);
  }
};

// One control step of one problem; shared by the single, batched and
// cooperative kernels.  sm: the working storage (X, packed R~, two
// vectors), or with gX set, X in gX and the rest in sm.  chol(X, p, sigma,
// Rk, s_inv, s_fail) factors X + sigma I into the packed Rk (0, or j + 1 of
// the failing pivot).
template <class Chol>
__device__ void ctrl_body_t(const Ctrl &c, double *sm, double *gX, const Chol &chol) {
  DevState *st = c.st;
  if (st->done) return;
  __shared__ double red[32];
  __shared__ float fred[32];
  __shared__ int s_fail;
  __shared__ double s_inv;
  const int p = c.p, q = c.q, t = threadIdx.x, NT = blockDim.x;
  const int ldc = q + p;
  double *X = gX ? gX : sm;             // p x p, full
  double *Rk = gX ? sm : X + p * p;     // packed upper, p (p + 1) / 2
  float *vecs = (float *)(Rk + p * (p + 1) / 2 + 1);
  float *v = vecs, *w = vecs + p;

  // X = Y^T Y - B~^T B~
  for (int e = t; e < p * p; e += NT) {
    const int i = e % p, j = e / p;
    double s = c.C[(q + i) + (int64_t)j * ldc];
    if (q > 0) {
      double b = 0.0;
      for (int k = 0; k < q; ++k) b += c.C[k + (int64_t)i * ldc] * c.C[k + (int64_t)j * ldc];
      s -= b;
    }
    X[e] = s;
  }
  double part = 0.0, partb = 0.0;
  __syncthreads();
  for (int e = t; e < p * p; e += NT) {
    const int i = e % p, j = e / p;
    const double d = X[e] - (i == j ? 1.0 : 0.0);
    part = fma(d, d, part);
  }
  for (int e = t; e < q * p; e += NT) {
    const double b = c.C[(e % q) + (int64_t)(e / q) * ldc];
    partb = fma(b, b, partb);
  }
  const double orth = sqrt(block_sum(part, red));
  const double projf = sqrt(block_sum(partb, red));

  const int it = st->iters;
  if (!isfinite(orth)) {
    // NaN/Inf in the Gramian: the stop test is undefined and no shift can
    // make X factorable; report a breakdown.
    if (t == 0) {
      st->done = 1;
      st->status = CQR_ERR_BREAKDOWN;
      st->orth_frob = orth;
      st->proj_frob = projf;
      st->active = 0;
    }
    return;
  }
  const double tol = (c.stop_rule == CQR_STOP_U_SQRT_N) ? kU64 * sqrt((double)p) : c.tol;
  const bool cont = (orth >= tol || it < c.min_iter) && it < c.max_iter;
  if (!cont) {
    if (t == 0) {
      st->done = 1;
      st->status = (orth < tol) ? CQR_OK : CQR_NOT_CONVERGED;
      st->orth_frob = orth;
      st->proj_frob = projf;
      st->active = 0;
    }
    return;
  }

  // ---- shift loop
  double sigma = 0.0;
  int attempts = 0, shifts = 0, escal = 0, rc = 0;
  double s_first = 0.0;
  bool fatal = false;
  if (c.mode == MODE_FACTOR) {
    const bool mixed_first = (it == 0) && (c.first_shift_coeff > 0.0);
    const bool shifted_first =
        mixed_first || ((it == 0) && (c.shift_policy == CQR_SHIFT_SCHOLQR3 ||
                                      c.shift_policy == CQR_SHIFT_SCHOLQR3_STRICT));
    const double sigma_once = st->sigma_once;  // read before thread 0 may set it
    if (shifted_first) {
      const double lam = norm_estimate(X, p, (float *)Rk, v, w, fred, red);
      if (mixed_first) {
        // the reduced-digit Gramian's bound: emax_coeff sum_j Ubar_j^2
        // (largest eigenvalue of the rank-one bound Ubar Ubar^T), summed in
        // column order
        double ub = 0.0;
        if (c.emax != nullptr)
          for (int j = 0; j < p; ++j) ub += ldexp(1.0, 2 * (c.emax[j] - 1022));
        sigma = fmax(c.first_shift_coeff * lam + c.emax_coeff * ub, 2.0 * kU64);
      } else {
        sigma = shift_alg1(c.m, p, lam);
      }
      ++shifts;
      s_first = sigma;
    }
    rc = chol(X, p, sigma, Rk, &s_inv, &s_fail);
    ++attempts;
    if (rc != 0 && !shifted_first) {
      if (c.shift_policy == CQR_SHIFT_NONE || c.shift_policy == CQR_SHIFT_SCHOLQR3_STRICT) {
        fatal = true;
      } else {
        if (c.shift_policy == CQR_SHIFT_ISCHOLQR && sigma_once > 0.0) {
          sigma = sigma_once;
        } else {
          const double lam = norm_estimate(X, p, (float *)Rk, v, w, fred, red);
          sigma = shift_alg1(c.m, p, lam);
          if (c.shift_policy == CQR_SHIFT_ISCHOLQR && t == 0) st->sigma_once = sigma;
        }
        ++shifts;
        s_first = sigma;
        rc = chol(X, p, sigma, Rk, &s_inv, &s_fail);
        ++attempts;
      }
    }
    int esc = 0;
    while (!fatal && rc != 0 && esc < c.max_escalations) {
      sigma *= 10.0;
      ++escal;
      ++esc;
      rc = chol(X, p, sigma, Rk, &s_inv, &s_fail);
      ++attempts;
    }
  } else {
    rc = chol(X, p, 0.0, Rk, &s_inv, &s_fail);
    ++attempts;
    int esc = 0;
    while (rc != 0 && esc < c.max_escalations) {
      if (sigma == 0.0) {
        const double lam = norm_estimate(X, p, (float *)Rk, v, w, fred, red);
        sigma = shift_alg2_first(c.m, q, p, lam);
        ++shifts;
        s_first = fmax(sigma, 2.0 * kU64);
      } else {
        sigma *= 10.0;
        ++escal;
      }
      sigma = fmax(sigma, 2.0 * kU64);
      ++esc;
      rc = chol(X, p, sigma, Rk, &s_inv, &s_fail);
      ++attempts;
    }
  }
  if (fatal || rc != 0) {
    if (t == 0) {
      st->chol_attempts += attempts;
      st->shifts += shifts;
      st->escalations += escal;
      st->done = 1;
      st->status = CQR_ERR_BREAKDOWN;
      st->orth_frob = orth;
      st->proj_frob = projf;
      st->active = 0;
    }
    return;
  }

  // ---- outputs of the pass
  for (int e = t; e < p * p; e += NT) {
    const int i = e % p, j = e / p;
    c.Rt[e] = (i <= j) ? Rk[pk(i, j)] : 0.0;
  }
  for (int j = t; j < p; j += NT) c.Rdinv[j] = 1.0 / Rk[pk(j, j)];
  __syncthreads();
  // R_old into the (no longer needed) X region
  double *Rold = X;
  for (int e = t; e < p * p; e += NT) {
    const int i = e % p, j = e / p;
    Rold[e] = c.R[i + (int64_t)j * c.ldr];
  }
  __syncthreads();
  if (c.mode == MODE_UPDATE && q > 0) {
    // B~ for the row sweep; B <- B + B~ R_old  (Alg. 2)
    for (int e = t; e < q * p; e += NT) {
      const int i = e % q, j = e / q;
      c.Bt[e] = c.C[i + (int64_t)j * ldc];
      double s = 0.0;
      for (int k = 0; k <= j; ++k) s += c.C[i + (int64_t)k * ldc] * Rold[k + j * p];
      c.B[i + (int64_t)j * c.ldb] = c.B[i + (int64_t)j * c.ldb] + s;
    }
  }
  // R <- R~ R_old  (Alg. 1, Alg. 2); with r_external the
  // factorisation leaves it to rupdate_kernel, which spreads the columns of
  // R over SMs
  for (int e = t; e < (c.r_external ? 0 : p * p); e += NT) {
    const int i = e % p, j = e / p;
    double s = 0.0;
    if (i <= j)
      for (int k = i; k <= j; ++k) s += Rk[pk(i, k)] * Rold[k + j * p];
    c.R[i + (int64_t)j * c.ldr] = s;
  }
  if (t == 0) {
    if (st->shifts == 0 && shifts > 0) st->sigma_first = s_first;
    if (sigma > 0.0) st->sigma_last = sigma;
    st->chol_attempts += attempts;
    st->shifts += shifts;
    st->escalations += escal;
    st->iters = it + 1;
    st->orth_frob = orth;
    st->proj_frob = projf;
    st->active = 1;
  }
}

__device__ __forceinline__ void ctrl_body(const Ctrl &c, double *sm, double *gX = nullptr) {
  ctrl_body_t(c, sm, gX, LocalChol{});
}

__global__ void __launch_bounds__(kCtrlThreads) ctrl_kernel(Ctrl c) {
  extern __shared__ double sm[];
  ctrl_body(c, sm);
}

// The same control step for widths above kCtrlSmemMaxP, whose n x n Gramian
// does not fit in shared memory: X in global memory (c.work) and the packed
// R~ with the vectors in shared memory (the Cholesky works there), or, when
// even R~ does not fit (ctrl_split_smem_bytes above 200 KB), everything in
// global memory (through L1 and L2).
__global__ void __launch_bounds__(kCtrlThreads) ctrl_split_kernel(Ctrl c) {
  extern __shared__ double sm[];
  ctrl_body(c, sm, c.work);
}
__global__ void __launch_bounds__(kCtrlThreads) ctrl_global_kernel(Ctrl c) { ctrl_body(c, c.work); }

// ---- Cooperative control step for wide blocks (p > kCtrlSmemMaxP)
//
// The Cholesky is the one O(n^3) part of the step, and on one SM it runs at
// ~2 FP64 FMAs per clock.  Here CTA 0 runs the control step above (stop
// test, norm estimate and shifts, retries, outputs) with its working storage
// in global memory, and every Cholesky it starts is shared by all CTAs of
// the cooperative launch, which wait for it in between.  The factorisation
// is right-looking by panels of 64 columns [j0, j1):
//   (a) every CTA copies the panel's diagonal block to shared memory and
//       factors it (the same arithmetic in each; CTA 0 writes it back);
//   (b) the row panel R_12 = R_11^{-T} A_12, one column per warp across the
//       grid, by the same scale-then-update steps as the unblocked routine;
//   (c) the trailing update A_22 -= R_12^T R_12 in 32 x 32 tiles across the
//       grid, each entry subtracting the panel's products in increasing row
//       order,
// so every entry of R~ takes the operations of `cholesky` in the same order.
// Grid barriers separate (b) and (c) and the panels; a Cholesky starts
// with a barrier (the previous one may have ended early at a failing pivot
// in some CTAs) and ends with one.  Every wait is bounded in wall time: one
// that runs out sets `timeout`, after which no CTA waits again and the step
// ends with CQR_ERR_TIMEOUT.
struct CoopCtl {
  unsigned job;        // number of Choleskys CTA 0 has posted
  unsigned quit;       // CTA 0 has finished the control step
  unsigned bar_count;  // grid barrier: arrivals of the current phase
  unsigned bar_gen;    // grid barrier: completed phases
  int timeout;         // a wait gave up
  int pad;
  double sigma;        // shift of the posted Cholesky
};

namespace {

constexpr int kCoopPanel = 64;
constexpr int kCoopTile = 32;
constexpr uint64_t kCoopWaitNs = 5000000000ull;  // 5 s
// shared memory of a cooperative CTA: the diagonal block (64 x 64), its
// inverse pivots, two 64 x 32 slices of the row panel
constexpr size_t kCoopSmem = sizeof(double) * ((size_t)kCoopPanel * kCoopPanel + kCoopPanel +
                                               2 * (size_t)kCoopPanel * kCoopTile);

__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// All CTAs of the grid reach this point (sense by generation count); false
// when the wait ran out (then `timeout` is set for everyone).
__device__ bool coop_sync(CoopCtl *cc) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = &cc->bar_gen;
    volatile int *to = &cc->timeout;
    int ok = (*to == 0);
    if (ok) {
      const unsigned g = *gen;
      __threadfence();
      if (atomicAdd(&cc->bar_count, 1u) == gridDim.x - 1) {
        cc->bar_count = 0;
        __threadfence();
        atomicAdd(&cc->bar_gen, 1u);
      } else {
        const uint64_t t0 = gtimer_ns();
        while (*gen == g) {
          if (*to != 0 || gtimer_ns() - t0 > kCoopWaitNs) {
            atomicExch(&cc->timeout, 1);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Unblocked right-looking factorisation of the diagonal block in shared
// memory (D, ld kCoopPanel, upper triangle), the steps of `cholesky`;
// inv[j] = 1 / R_jj.  Returns 0 or j0 + j + 1 of the failing pivot.
__device__ int coop_diag(double *D, double *inv, int nb, int j0) {
  __shared__ int s_fail;
  const int t = threadIdx.x, NT = blockDim.x;
  if (t == 0) s_fail = 0;
  __syncthreads();
  const int cl = t >> 3, rl = t & 7, cstep = NT >> 3;
  for (int j = 0; j < nb; ++j) {
    if (t == 0) {
      const double d = D[j + j * kCoopPanel];
      if (!(d > 0.0) || !isfinite(d)) {
        s_fail = j0 + j + 1;
      } else {
        const double r = sqrt(d);
        D[j + j * kCoopPanel] = r;
        inv[j] = 1.0 / r;
      }
    }
    __syncthreads();
    if (s_fail) return s_fail;
    const double iv = inv[j];
    for (int k = j + 1 + t; k < nb; k += NT) D[j + k * kCoopPanel] *= iv;
    __syncthreads();
    for (int k = j + 1 + cl; k < nb; k += cstep) {
      const double rjk = D[j + k * kCoopPanel];
      for (int i = j + 1 + rl; i <= k; i += 8) D[i + k * kCoopPanel] -= D[j + i * kCoopPanel] * rjk;
    }
    __syncthreads();
  }
  return 0;
}

// R~^T R~ = X + sigma I into the packed Rk (global), by all CTAs of the
// grid.  Returns 0, j + 1 of the failing pivot, or -1 after a timeout.
__device__ int coop_cholesky(const double *X, int p, double sigma, double *Rk, CoopCtl *cc, double *csm) {
  double *D = csm, *inv = D + kCoopPanel * kCoopPanel, *Pi = inv + kCoopPanel, *Pk = Pi + kCoopPanel * kCoopTile;
  const int t = threadIdx.x, NT = blockDim.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  if (!coop_sync(cc)) return -1;  // every CTA has left the previous Cholesky
  for (int64_t e = (int64_t)b * NT + t; e < (int64_t)p * p; e += (int64_t)G * NT) {
    const int i = (int)(e % p), j = (int)(e / p);
    if (i <= j) Rk[pk(i, j)] = X[e] + (i == j ? sigma : 0.0);
  }
  if (!coop_sync(cc)) return -1;
  for (int j0 = 0; j0 < p; j0 += kCoopPanel) {
    const int nb = min(kCoopPanel, p - j0), j1 = j0 + nb;
    // (a) the diagonal block
    for (int e = t; e < nb * nb; e += NT) {
      const int i = e % nb, j = e / nb;
      D[i + j * kCoopPanel] = (i <= j) ? Rk[pk(j0 + i, j0 + j)] : 0.0;
    }
    __syncthreads();
    const int rc = coop_diag(D, inv, nb, j0);
    if (rc != 0) return rc;  // the same pivot fails in every CTA
    if (b == 0)
      for (int e = t; e < nb * nb; e += NT) {
        const int i = e % nb, j = e / nb;
        if (i <= j) Rk[pk(j0 + i, j0 + j)] = D[i + j * kCoopPanel];
      }
    // (b) row panel: column k of A_12 by one warp; lane l holds rows l, l + 32
    const int nw = NT >> 5;
    for (int k = j1 + b * nw + warp; k < p; k += G * nw) {
      double a0 = (lane < nb) ? Rk[pk(j0 + lane, k)] : 0.0;
      double a1 = (lane + 32 < nb) ? Rk[pk(j0 + lane + 32, k)] : 0.0;
      for (int j = 0; j < nb; ++j) {
        // scale row j, then subtract its product from the rows below
        const bool mine0 = (j < 32) && (lane == j), mine1 = (j >= 32) && (lane == j - 32);
        if (mine0) a0 *= inv[j];
        if (mine1) a1 *= inv[j];
        const double x = __shfl_sync(0xffffffffu, j < 32 ? a0 : a1, j & 31);
        if (lane > j && lane < nb) a0 -= D[j + lane * kCoopPanel] * x;
        if (lane + 32 > j && lane + 32 < nb) a1 -= D[j + (lane + 32) * kCoopPanel] * x;
      }
      if (lane < nb) Rk[pk(j0 + lane, k)] = a0;
      if (lane + 32 < nb) Rk[pk(j0 + lane + 32, k)] = a1;
    }
    if (!coop_sync(cc)) return -1;
    // (c) trailing update of the upper triangle of [j1, p)^2 in tiles
    const int nt = (p - j1 + kCoopTile - 1) / kCoopTile;
    const int ntiles = nt * (nt + 1) / 2;
    for (int w = b; w < ntiles; w += G) {
      int K = 0;
      while ((K + 1) * (K + 2) / 2 <= w) ++K;
      const int I = w - K * (K + 1) / 2;  // tile (I, K), I <= K
      const int i0 = j1 + kCoopTile * I, k0 = j1 + kCoopTile * K;
      __syncthreads();  // the previous tile's readers are done
      for (int e = t; e < nb * kCoopTile; e += NT) {
        const int j = e % nb, c = e / nb;
        Pi[j + c * kCoopPanel] = (i0 + c < p) ? Rk[pk(j0 + j, i0 + c)] : 0.0;
        Pk[j + c * kCoopPanel] = (k0 + c < p) ? Rk[pk(j0 + j, k0 + c)] : 0.0;
      }
      __syncthreads();
      for (int e = t; e < kCoopTile * kCoopTile; e += NT) {
        const int il = e % kCoopTile, kl = e / kCoopTile, i = i0 + il, k = k0 + kl;
        if (i > k || k >= p) continue;
        double a = Rk[pk(i, k)];
        for (int j = 0; j < nb; ++j) a -= Pi[j + il * kCoopPanel] * Pk[j + kl * kCoopPanel];
        Rk[pk(i, k)] = a;
      }
    }
    if (!coop_sync(cc)) return -1;
  }
  return 0;
}

// CTA 0's Cholesky: post the shift, then take part like the others.
struct CoopChol {
  CoopCtl *cc;
  double *csm;
  __device__ int operator()(const double *X, int p, double sigma, double *Rk, double *, int *) const {
    __shared__ int s_to;
    __syncthreads();
    if (threadIdx.x == 0) {
      s_to = *(volatile int *)&cc->timeout;
      if (!s_to) {
        *(volatile double *)&cc->sigma = sigma;
        __threadfence();
        atomicAdd(&cc->job, 1u);
      }
    }
    __syncthreads();
    if (s_to) return -1;
    return coop_cholesky(X, p, sigma, Rk, cc, csm);
  }
};

}  // namespace

__global__ void __launch_bounds__(kCtrlThreads, 1) ctrl_coop_kernel(Ctrl c, CoopCtl *cc) {
  extern __shared__ double csm[];
  const int p = c.p;
  double *X = c.work, *Rk = X + (size_t)p * p;
  if (blockIdx.x == 0) {
    ctrl_body_t(c, c.work, nullptr, CoopChol{cc, csm});
    __syncthreads();
    if (threadIdx.x == 0) {
      if (*(volatile int *)&cc->timeout) {
        c.st->done = 1;
        c.st->status = CQR_ERR_TIMEOUT;
        c.st->active = 0;
      }
      __threadfence();
      atomicExch(&cc->quit, 1u);
    }
    return;
  }
  __shared__ int s_go;
  __shared__ double s_sigma;
  unsigned seen = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      volatile unsigned *job = &cc->job, *quit = &cc->quit;
      const uint64_t t0 = gtimer_ns();
      int go = 0;
      for (;;) {
        const unsigned jb = *job;
        if (jb != seen) {
          seen = jb;
          go = 1;
          break;
        }
        if (*quit || *(volatile int *)&cc->timeout) break;
        if (gtimer_ns() - t0 > kCoopWaitNs) {
          atomicExch(&cc->timeout, 1);
          break;
        }
        __nanosleep(128);
      }
      __threadfence();
      s_go = go;
      s_sigma = *(volatile double *)&cc->sigma;
    }
    __syncthreads();
    if (!s_go) return;
    (void)coop_cholesky(X, p, s_sigma, Rk, cc, csm);
    __syncthreads();
  }
}

// Cooperative grid of the wide control step (0: not available).
static int ctrl_coop_grid() {
  static std::atomic<int> cache[64];
  int dev = 0;
  cudaGetDevice(&dev);
  const bool cached = dev >= 0 && dev < 64;
  int g = cached ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (g != 0) return g > 0 ? g : 0;
  int coop = 0, per_sm = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (coop && cudaFuncSetAttribute(ctrl_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kCoopSmem) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ctrl_coop_kernel, kCtrlThreads, kCoopSmem) ==
          cudaSuccess &&
      per_sm > 0)
    g = num_sms();  // one CTA per SM
  else
    g = -1;
  (void)cudaGetLastError();
  if (cached) cache[dev].store(g, std::memory_order_relaxed);
  return g > 0 ? g : 0;
}

// The stream on which every cooperative control step of the current device
// runs (created once per device, with the two events that join it to the
// caller's stream), or null when it cannot be created: the single-CTA
// kernels then take the step.  Two cooperative grids running at once could
// each hold SMs that the other's barriers wait for.
struct CoopLane {
  std::mutex mu;
  cudaStream_t st = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
  int state = 0;  // 0 not tried, 1 ready, -1 failed
};
static CoopLane *coop_lane() {
  static CoopLane lanes[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  CoopLane &L = lanes[dev];
  std::lock_guard<std::mutex> lock(L.mu);
  if (L.state == 0) {
    const bool ok = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&L.in, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&L.out, cudaEventDisableTiming) == cudaSuccess;
    (void)cudaGetLastError();
    L.state = ok ? 1 : -1;
  }
  return L.state == 1 ? &L : nullptr;
}

// Bytes of the global working storage of a wide control step: X, packed R~,
// two vectors (ctrl_smem_bytes) and the cooperative launch's control words.
size_t ctrl_work_bytes(int p) { return ((ctrl_smem_bytes(p) + 255) & ~(size_t)255) + sizeof(CoopCtl); }

// Batched control: CTA b handles problems b, b + grid, ...
__global__ void __launch_bounds__(kCtrlThreads) ctrl_batched_kernel(const Ctrl *reqs, const int *nreq) {
  extern __shared__ double sm[];
  const int n = *nreq;
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const Ctrl c = reqs[r];
    ctrl_body(c, sm);
    __syncthreads();
  }
}

cudaError_t launch_ctrl_batched(const Ctrl *reqs, const int *nreq, int grid, size_t smem,
                                cudaStream_t s) {
  static KernelAttr attr;
  set_smem_attr(attr, ctrl_batched_kernel, 200 * 1024, false);
  ctrl_batched_kernel<<<grid, kCtrlThreads, smem, s>>>(reqs, nreq);
  return cudaGetLastError();
}

// X (p x p), packed R~, two float vectors.
// bytes of the packed R~ and the two vectors (the split layout's shared part)
static size_t ctrl_split_smem_bytes(int p) {
  return (size_t)(p * (p + 1) / 2 + 1) * sizeof(double) + (size_t)2 * p * sizeof(float) + 64;
}

size_t ctrl_smem_bytes(int p) {
  return (size_t)p * p * sizeof(double) + (size_t)(p * (p + 1) / 2 + 1) * sizeof(double) +
         (size_t)2 * p * sizeof(float) + 64;
}

// T = D R~^{-1} for the tensor-core solve (the explicit inverse of App. A),
// one single-warp CTA per row: row i of T solves t R~ = e_i^T by forward
// substitution, T_ii = 1 / R~_ii and T_ij = -(sum_{i<=k<j} T_ik R~_kj) / R~_jj
// in increasing j (each sum split over the 32 lanes, combined in a fixed
// butterfly), so T R~ - I stays at working accuracy.  The row is then scaled
// by 2^c_i, c_i = floor(log2 sqrt(X_ii)): the product Q = Y T is formed as
// (Y D^-1)(D T), D = diag(2^c), which balances the columns of Y and the rows
// of T (exact: powers of two).  Rows are independent, so they run on
// separate SMs.  Up to kTinvMaxN columns R~ is copied to shared memory;
// above (GLOBAL_R) the sums read its columns from global memory (L2), 32
// consecutive entries per step.
template <bool GLOBAL_R>
__global__ void __launch_bounds__(128) tinv_kernel(const double *Rt, const double *Rdinv, const double *C,
                                                   int ldc, int q, int p, double *Tinv, int *Tscale,
                                                   const DevState *st) {
  if (st != nullptr && st->done) return;
  extern __shared__ double sh[];  // [R~ (p x p, ld p)], 1 / diag, then row i of T
  const double *Rs = GLOBAL_R ? Rt : sh;
  double *rd = GLOBAL_R ? sh : sh + (size_t)p * p, *tr = rd + p;
  const int i = blockIdx.x, t = threadIdx.x, lane = t & 31;
  if (i >= p) return;
  // the dependent steps below read only shared memory; the copy issues 8
  // loads before it stores (the loads are then in flight together)
  for (int e0 = 0; !GLOBAL_R && e0 < p * p; e0 += 8 * 128) {
    double v[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int e = e0 + h * 128 + t;
      v[h] = (e < p * p) ? Rt[e] : 0.0;
    }
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int e = e0 + h * 128 + t;
      if (e < p * p) sh[e] = v[h];
    }
  }
  for (int j = t; j < p; j += blockDim.x) {
    rd[j] = Rdinv[j];
    tr[j] = 0.0;
  }
  __syncthreads();
  if (t >= 32) return;
  if (lane == 0) tr[i] = rd[i];
  __syncwarp();
  for (int j = i + 1; j < p; ++j) {
    double s = 0.0;
    for (int k = i + lane; k < j; k += 32) s = fma(tr[k], Rs[k + (int64_t)j * p], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) tr[j] = -s * rd[j];
    __syncwarp();
  }
  const double xii = C[(q + i) + (int64_t)i * ldc];
  const int ci = (xii > 0.0 && isfinite(xii)) ? (ilogb(xii) >> 1) : 0;
  if (lane == 0) Tscale[i] = ci;
  // times 2^c_i: one multiplication by an exact power of two when 2^c_i is
  // a normal number, ldexp otherwise
  const bool normal = (ci >= -1022 && ci <= 1023);
  const double sc = normal ? __longlong_as_double((long long)(1023 + ci) << 52) : 1.0;
  for (int j = lane; j < p; j += 32) {
    const double v = tr[j];
    Tinv[i + (int64_t)j * p] = (j < i) ? 0.0 : (normal ? v * sc : ldexp(v, ci));
  }
}

// R <- R~ R for a factorisation pass that continues: column j of the new R
// is R~ times column j of the old one (rows i <= j, the sum over k = i..j in
// increasing k), so each CTA updates its own column in place.
__global__ void __launch_bounds__(128) rupdate_kernel(const double *Rt, int p, double *R, int64_t ldr,
                                                      const DevState *st) {
  if (st != nullptr && st->done) return;  // the pass stopped: R is final
  __shared__ double col[kCqrMaxN];
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= p) return;
  for (int k = t; k <= j; k += blockDim.x) col[k] = R[k + (int64_t)j * ldr];
  __syncthreads();
  for (int i = t; i <= j; i += blockDim.x) {
    double s = 0.0;
    for (int k = i; k <= j; ++k) s += Rt[i + (int64_t)k * p] * col[k];
    R[i + (int64_t)j * ldr] = s;
  }
}

cudaError_t launch_rupdate(const double *Rt, int p, double *R, int64_t ldr, const DevState *st,
                           cudaStream_t s) {
  if (p > kCqrMaxN) return cudaErrorInvalidValue;
  rupdate_kernel<<<p, 128, 0, s>>>(Rt, p, R, ldr, st);
  return cudaGetLastError();
}

cudaError_t launch_tinv(const double *Rt, const double *Rdinv, const double *C, int ldc, int q, int p,
                        double *Tinv, int *Tscale, const DevState *st, cudaStream_t s) {
  if (p > kCqrMaxN) return cudaErrorInvalidValue;
  if (p > kTinvMaxN) {  // R~ read from global memory; 1 / diag and a row of T in shared memory
    tinv_kernel<true><<<p, 128, sizeof(double) * 2 * (size_t)p, s>>>(Rt, Rdinv, C, ldc, q, p, Tinv, Tscale, st);
    return cudaGetLastError();
  }
  static KernelAttr attr;  // R~ and a row of T in shared memory (133 KB at 128)
  const size_t smem = sizeof(double) * ((size_t)kTinvMaxN * kTinvMaxN + 2 * kTinvMaxN);
  set_smem_attr(attr, tinv_kernel<false>, (int)smem, false);
  tinv_kernel<false><<<p, 128, sizeof(double) * ((size_t)p * p + 2 * p), s>>>(Rt, Rdinv, C, ldc, q, p, Tinv,
                                                                             Tscale, st);
  return cudaGetLastError();
}

cudaError_t launch_ctrl(const Ctrl &a, cudaStream_t s) {
  if (a.p > kCtrlSmemMaxP) {
    if (a.work == nullptr) return cudaErrorInvalidValue;
    const int G = ctrl_coop_grid();
    CoopLane *L = G > 0 ? coop_lane() : nullptr;
    if (L != nullptr) {
      // on the device's cooperative stream, between two events on the
      // caller's stream: cooperative steps of concurrent calls run one
      // after another, so none holds SMs that another's barriers wait for
      std::lock_guard<std::mutex> lock(L->mu);
      CoopCtl *cc = (CoopCtl *)((char *)a.work + ((ctrl_smem_bytes(a.p) + 255) & ~(size_t)255));
      cudaError_t e = cudaMemsetAsync(cc, 0, sizeof(CoopCtl), s);
      if (e == cudaSuccess) e = cudaEventRecord(L->in, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(L->st, L->in, 0);
      if (e != cudaSuccess) return e;
      Ctrl c = a;
      void *args[] = {(void *)&c, (void *)&cc};
      e = cudaLaunchCooperativeKernel((const void *)ctrl_coop_kernel, dim3(G), dim3(kCtrlThreads), args,
                                      kCoopSmem, L->st);
      if (e == cudaSuccess) e = cudaEventRecord(L->out, L->st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, L->out, 0);
      return e;
    }
    const size_t sm = ctrl_split_smem_bytes(a.p);
    if (sm <= 200 * 1024) {
      static KernelAttr sattr;
      set_smem_attr(sattr, ctrl_split_kernel, 200 * 1024, false);
      ctrl_split_kernel<<<1, kCtrlThreads, sm, s>>>(a);
    } else {
      ctrl_global_kernel<<<1, kCtrlThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
  }
  static KernelAttr attr;
  set_smem_attr(attr, ctrl_kernel, 200 * 1024, false);
  ctrl_kernel<<<1, kCtrlThreads, ctrl_smem_bytes(a.p), s>>>(a);
  return cudaGetLastError();
}

}  // namespace cqr
