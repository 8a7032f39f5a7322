// Row-wise triangular solve Q = Y R~^{-1} in FP64 (Alg. 1 line 9), one thread
// per row with the row held in registers.
//
// The solve is forward substitution on R~^T q^T = y^T, done right-looking:
// for j = 0..n-1, q_j <- q_j / R~_jj (a multiplication by the precomputed
// 1 / R~_jj), then q_k <- q_k - q_j R~_jk for every k > j.  Each q_k thus
// accumulates y_k - sum_{j<k} q_j R~_jk in increasing j, the plain recursive
// summation of the textbook substitution.  Per row that is exactly
// n (n-1) / 2 fused multiply-adds and n multiplications, the fewest FP64
// instructions a substitution can issue (a left-looking form with split
// partial sums spends a fifth more on combining them), and every step j
// offers n - j - 1 independent FMAs, so a few warps per SM keep GB300's
// narrow FP64 pipe busy.  Row j of R~ (k > j) is stored contiguously in
// shared memory and every thread of a warp reads the same entry (broadcast).
#include <algorithm>

#include "cqr_internal.cuh"

namespace cqr {

constexpr int kTrsmThreads = 64;

template <int NT>
__global__ void __launch_bounds__(kTrsmThreads) trsm_rows_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  // Rs[j * NT + k] = R~_jk for j < k < n (zero elsewhere), then 1 / R~_jj
  extern __shared__ double Rs[];
  const int n = a.p, t = threadIdx.x;
  for (int e = t; e < NT * NT; e += kTrsmThreads) {
    const int j = e / NT, k = e % NT;
    Rs[e] = (k > j && k < n) ? a.Rt[j + (int64_t)k * n] : 0.0;
  }
  for (int j = t; j < NT; j += kTrsmThreads) Rs[NT * NT + j] = (j < n) ? a.Rdinv[j] : 0.0;
  __syncthreads();
  const double *Rd = Rs + NT * NT;
  for (int64_t row = (int64_t)blockIdx.x * kTrsmThreads + t; row < a.m;
       row += (int64_t)gridDim.x * kTrsmThreads) {
    double q[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) q[j] = (j < n) ? a.Yin[row + (int64_t)j * a.ldyin] : 0.0;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      if (j < n) {
        q[j] *= Rd[j];
        const double nq = -q[j];
        const double *Rj = Rs + j * NT;
#pragma unroll
        for (int k = j + 1; k < NT; ++k) q[k] = fma(nq, Rj[k], q[k]);
      }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j < n) a.Yout[row + (int64_t)j * a.ldyout] = q[j];
  }
}

// n in (64, 128]: a row no longer fits one thread's registers, so a group of
// four adjacent lanes shares it, lane g of the group owning the columns
// k = 4i + g (32 doubles each).  At step j the owner of column j scales q_j
// and the group reads it with one shuffle; every lane then updates its own
// columns k > j.  The FP64 work per row is the same n(n-1)/2 FMAs and n
// multiplications.  R~ is split by column residue in shared memory (132 KB),
// one CTA of 8 warps per SM (248 registers per thread).
constexpr int kTrsm4Threads = 256;
constexpr int kTrsm4NT = 128;

__global__ void __launch_bounds__(kTrsm4Threads, 1) trsm_rows4_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  constexpr int NT = kTrsm4NT, H = NT / 4;
  // Rs[(g * NT + j) * H + i] = R~_{j, 4i+g} for j < 4i+g < n (zero elsewhere),
  // then 1 / R~_jj
  extern __shared__ double Rs[];
  const int n = a.p, t = threadIdx.x;
  for (int e = t; e < 4 * NT * H; e += kTrsm4Threads) {
    const int g = e / (NT * H), j = (e / H) % NT, k = 4 * (e % H) + g;
    Rs[e] = (k > j && k < n) ? a.Rt[j + (int64_t)k * n] : 0.0;
  }
  for (int j = t; j < NT; j += kTrsm4Threads) Rs[4 * NT * H + j] = (j < n) ? a.Rdinv[j] : 0.0;
  __syncthreads();
  const double *Rd = Rs + 4 * NT * H;
  const int g = t & 3, lane = t & 31;
  const double *Rg = Rs + g * NT * H;
  const int64_t rows_per_iter = (int64_t)gridDim.x * (kTrsm4Threads / 4);
  // every lane of a warp runs the same number of iterations (the shuffles
  // stay convergent); rows past m are computed on zeros and not stored
  const int64_t iters = (a.m + rows_per_iter - 1) / rows_per_iter;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t row = it * rows_per_iter + (int64_t)blockIdx.x * (kTrsm4Threads / 4) + (t >> 2);
    const bool live = row < a.m;
    double q[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const int k = 4 * i + g;
      q[i] = (live && k < n) ? a.Yin[row + (int64_t)k * a.ldyin] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      if (j < n) {
        if ((j & 3) == g) q[j >> 2] *= Rd[j];
        const double qj = __shfl_sync(0xffffffffu, q[j >> 2], (lane & ~3) | (j & 3));
        const double nq = -qj;
        const double *Rj = Rg + j * H;
#pragma unroll
        for (int i = (j + 1) >> 2; i < H; ++i) {
          // column 4i+g; entries with 4i+g <= j are zero in shared memory,
          // so only i = floor((j+1)/4)'s lanes below j see a no-op update
          if (4 * i + g > j) q[i] = fma(nq, Rj[i], q[i]);
        }
      }
    }
    if (live) {
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const int k = 4 * i + g;
        if (k < n) a.Yout[row + (int64_t)k * a.ldyout] = q[i];
      }
    }
  }
}

template <int NT>
static cudaError_t launch_tr(const RowSweep &a, int grid, cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)NT * NT + NT);
  static KernelAttr attr;
  set_smem_attr(attr, trsm_rows_kernel<NT>, 64 * 1024, false);
  trsm_rows_kernel<NT><<<grid, kTrsmThreads, smem, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_tr4(const RowSweep &a, cudaStream_t s) {
  constexpr int NT = kTrsm4NT;
  const size_t smem = sizeof(double) * ((size_t)NT * NT + NT);
  static KernelAttr attr;
  set_smem_attr(attr, trsm_rows4_kernel, (int)smem, false);
  const int64_t rows_per_cta = kTrsm4Threads / 4;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((a.m + rows_per_cta - 1) / rows_per_cta, (int64_t)num_sms()));
  trsm_rows4_kernel<<<grid, kTrsm4Threads, smem, s>>>(a);
  return cudaGetLastError();
}

// Up to four CTAs per SM (two warps each): on a 125,000-row chunk at n = 64
// one CTA per SM reaches half the rate of four.
int trsm_rows_grid(int64_t m) {
  const int64_t blocks = (m + kTrsmThreads - 1) / kTrsmThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, 4 * (int64_t)num_sms()));
}

// n <= 64: `grid` CTAs of the one-thread-per-row kernel; 64 < n <= 128: the
// four-lanes-per-row kernel with one CTA per SM (grid is ignored).
cudaError_t launch_trsm_rows(const RowSweep &a, int grid, cudaStream_t s) {
  if (a.p <= 16) return launch_tr<16>(a, grid, s);
  if (a.p <= 32) return launch_tr<32>(a, grid, s);
  if (a.p <= 64) return launch_tr<64>(a, grid, s);
  if (a.p <= kTrsm4NT) return launch_tr4(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace cqr
