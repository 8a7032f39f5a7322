// Rank-ordered sum of the gathered Gramian partials of a row-sharded
// factorisation (communication-avoiding Cholesky QR, Sec. 1): every rank
// holds the gathered blocks of all ranks, recv[r * count + e], and forms
// C[e] = (((recv_0[e] + recv_1[e]) + recv_2[e]) + ...) in rank order, so the
// Gramian, and with it every shift, breakdown and stop decision, is bitwise
// the same on every rank.
#include <algorithm>

#include "cqr_internal.cuh"

namespace cqr {

__global__ void __launch_bounds__(256) sum_ranks_kernel(const double *recv, int world, int64_t count,
                                                        double *C) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = recv[e];
    for (int r = 1; r < world; ++r) s += recv[(int64_t)r * count + e];
    C[e] = s;
  }
}

cudaError_t launch_sum_ranks(const double *recv, int world, int64_t count, double *C, cudaStream_t s) {
  if (world < 1 || count < 1) return cudaErrorInvalidValue;
  const int grid = (int)std::min<int64_t>(64, (count + 255) / 256);
  sum_ranks_kernel<<<grid, 256, 0, s>>>(recv, world, count, C);
  return cudaGetLastError();
}

}  // namespace cqr
