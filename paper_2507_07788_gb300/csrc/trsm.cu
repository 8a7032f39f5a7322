// Row-wise triangular solve Q = Y R~^{-1} in FP64 (Alg. 1 line 9), one thread
// per row with the row held in registers.
//
// The solve is forward substitution on R~^T q^T = y^T: q_j = (y_j -
// sum_{k<j} q_k R~_kj) / R~_jj, with the sum split into eight interleaved
// partial sums (k mod 8) added pairwise, for instruction-level parallelism on
// GB300's narrow FP64 pipe, and the division done as a
// multiplication by the precomputed 1 / R~_jj.  R~ and its inverse diagonal
// sit in shared memory and every thread of a warp reads the same entry
// (broadcast).  CTAs are small (64 threads, ~33 KB shared memory) so that
// they share SMs with the tensor-core Gramian kernel of the same pass, which
// runs on another stream on the previous chunk of rows.
#include <algorithm>

#include "cqr_internal.cuh"

namespace cqr {

constexpr int kTrsmThreads = 64;

template <int NT>
__global__ void __launch_bounds__(kTrsmThreads) trsm_rows_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  extern __shared__ double Rs[];  // R~ (n x n, ld n) then 1 / diag
  const int n = a.p, t = threadIdx.x;
  for (int e = t; e < n * n; e += kTrsmThreads) Rs[e] = a.Rt[e];
  for (int j = t; j < n; j += kTrsmThreads) Rs[n * n + j] = a.Rdinv[j];
  __syncthreads();
  const double *Rd = Rs + n * n;
  for (int64_t row = (int64_t)blockIdx.x * kTrsmThreads + t; row < a.m;
       row += (int64_t)gridDim.x * kTrsmThreads) {
    double q[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) q[j] = (j < n) ? a.Yin[row + (int64_t)j * a.ldyin] : 0.0;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      if (j < n) {
        const double *Rj = Rs + j * n;
        double sp[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sp[u] = 0.0;
#pragma unroll
        for (int k = 0; k < j; ++k) sp[k & 7] = fma(q[k], Rj[k], sp[k & 7]);
        const double s = ((sp[0] + sp[1]) + (sp[2] + sp[3])) + ((sp[4] + sp[5]) + (sp[6] + sp[7]));
        q[j] = (q[j] - s) * Rd[j];
      }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j < n) a.Yout[row + (int64_t)j * a.ldyout] = q[j];
  }
}

template <int NT>
static cudaError_t launch_tr(const RowSweep &a, int grid, cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)a.p * a.p + a.p);
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(trsm_rows_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    attr_done = true;
  }
  trsm_rows_kernel<NT><<<grid, kTrsmThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Up to four CTAs per SM: the FP64 pipe needs several warps with
// independent chains to stay busy.
int trsm_rows_grid(int64_t m) {
  const int64_t blocks = (m + kTrsmThreads - 1) / kTrsmThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, 4 * (int64_t)num_sms()));
}

cudaError_t launch_trsm_rows(const RowSweep &a, int grid, cudaStream_t s) {
  if (a.p <= 16) return launch_tr<16>(a, grid, s);
  if (a.p <= 32) return launch_tr<32>(a, grid, s);
  if (a.p <= 64) return launch_tr<64>(a, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace cqr
