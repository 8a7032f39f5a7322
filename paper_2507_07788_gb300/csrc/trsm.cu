// Row-wise triangular solve Q = Y R~^{-1} in FP64 (Alg. 1), one thread
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

template <int NT>
static cudaError_t launch_tr(const RowSweep &a, int grid, cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)NT * NT + NT);
  static KernelAttr attr;
  set_smem_attr(attr, trsm_rows_kernel<NT>, 64 * 1024, false);
  trsm_rows_kernel<NT><<<grid, kTrsmThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Up to four CTAs per SM (two warps each): on a 125,000-row chunk at n = 64
// one CTA per SM reaches half the rate of four.
int trsm_rows_grid(int64_t m) {
  const int64_t blocks = (m + kTrsmThreads - 1) / kTrsmThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, 4 * (int64_t)num_sms()));
}

// n <= 16 (wider blocks take the tensor-core product): `grid` CTAs of the
// one-thread-per-row kernel.
cudaError_t launch_trsm_rows(const RowSweep &a, int grid, cudaStream_t s) {
  if (a.p <= 16) return launch_tr<16>(a, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace cqr
