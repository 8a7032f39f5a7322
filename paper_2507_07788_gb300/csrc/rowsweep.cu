// Row sweeps over the tall dimension m (FP64 CUDA-core version).
//
// One kernel covers the three bandwidth-bound steps of the method:
//   * the Gramian X = A^T A of the first pass (Alg. 1),
//   * the row-wise triangular solve Q = Q R~^{-1} of a pass fused with the
//     Gramian of the result for the next pass (Alg. 1),
//   * for the update, the projection y <- (y - q_in B~) R~^{-1} fused with
//     the next B~ = Q_in^T Q and Q^T Q (Alg. 2; its initial B~ and
//     Gramian are the first sweep, without the solve).
// Each CTA owns a contiguous range of rows, walks it in tiles staged in
// shared memory, and accumulates its share of C = [Q_in Y]^T Y in registers
// in ascending row order.  The per-CTA partials are summed afterwards in a
// fixed order (reduce_kernel), so results do not depend on scheduling.
#include <algorithm>

#include "cqr_internal.cuh"

namespace cqr {

// Map entry e of C = [Q_in Y]^T Y to shared-memory column indices (ca, cb):
// e < q p: B~ entry (i, j) = (e mod q, e div q), columns (i, q + j);
// else the upper triangle of Y^T Y in column-major packed order,
// columns (q + i, q + j) with i <= j.
__device__ __forceinline__ void entry_columns(int64_t e, int q, int p, int &ca, int &cb) {
  const int64_t qp = (int64_t)q * p;
  if (e < qp) {
    ca = (int)(e % q);
    cb = q + (int)(e / q);
  } else {
    int64_t f = e - qp;
    // j = largest with j (j + 1) / 2 <= f
    int j = (int)((sqrt(8.0 * (double)f + 1.0) - 1.0) * 0.5);
    while ((int64_t)(j + 1) * (j + 2) / 2 <= f) ++j;
    while ((int64_t)j * (j + 1) / 2 > f) --j;
    int i = (int)(f - (int64_t)j * (j + 1) / 2);
    ca = q + i;
    cb = q + j;
  }
}

// The work of CTA (bx, by) of one sweep.  Shared by the single-problem
// kernel and the batched persistent kernel, so that a problem computes the
// same partial sums in the same order whether it runs alone or in a batch.
template <int EPT>
__device__ __forceinline__ void rowsweep_body(const RowSweep &a, int bx, int by, double *tile) {
  if (a.st != nullptr && a.st->done) return;
  const int t = threadIdx.x;
  const int q = a.q, p = a.p, W = q + p, lds = a.lds, TR = a.tile_rows;
  const int64_t row0 = (int64_t)bx * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);

  uint32_t idx[EPT];
  double acc[EPT];
  const int64_t ebase = (int64_t)by * (kThreads * EPT);
  // slots of this thread that hold entries (entry ebase + t + k kThreads,
  // k < kact): the batched kernel is compiled for the largest E, and warps
  // past the last entry skip the products
  const int64_t left = a.E - ebase - t;
  const int kact = left <= 0 ? 0 : (int)min((int64_t)EPT, (left + kThreads - 1) / kThreads);
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = ebase + t + (int64_t)k * kThreads;
    int ca = 0, cb = 0;
    if (e < a.E) entry_columns(e, q, p, ca, cb);
    idx[k] = (uint32_t)ca | ((uint32_t)cb << 16);
    acc[k] = 0.0;
  }

  for (int64_t r0 = row0; r0 < row1; r0 += TR) {
    const int nr = (int)min((int64_t)TR, row1 - r0);
    // Stage rows r0 .. r0 + TR - 1 of [Q_in Y] (zero beyond nr).  Consecutive
    // threads read consecutive rows of one column: coalesced.
    for (int e = t; e < TR * W; e += kThreads) {
      const int i = e % TR, c = e / TR;
      double v = 0.0;
      if (i < nr)
        v = (c < q) ? a.Qin[(r0 + i) + (int64_t)c * a.ldqin]
                    : a.Yin[(r0 + i) + (int64_t)(c - q) * a.ldyin];
      tile[i * lds + c] = v;
    }
    __syncthreads();
    if (a.do_trsm) {
      if (t < nr) {
        double *row = tile + t * lds;
        // y <- y - q_in B~  (Alg. 2, first factor)
        if (q > 0) {
          for (int j = 0; j < p; ++j) {
            double s = row[q + j];
            for (int i = 0; i < q; ++i) s -= row[i] * a.Bt[i + (int64_t)j * q];
            row[q + j] = s;
          }
        }
        // y <- y R~^{-1} by forward substitution on R~^T y^T = y^T
        for (int j = 0; j < p; ++j) {
          double s = row[q + j];
          for (int k = 0; k < j; ++k) s -= row[q + k] * a.Rt[k + (int64_t)j * p];
          row[q + j] = s * a.Rdinv[j];
        }
      }
      __syncthreads();
      for (int e = t; e < nr * p; e += kThreads) {
        const int i = e % nr, j = e / nr;
        a.Yout[(r0 + i) + (int64_t)j * a.ldyout] = tile[i * lds + q + j];
      }
    }
    for (int i = 0; i < nr; ++i) {
      const double *row = tile + i * lds;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        if (k >= kact) break;
        acc[k] = fma(row[idx[k] & 0xFFFFu], row[idx[k] >> 16], acc[k]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = ebase + t + (int64_t)k * kThreads;
    if (e < a.E) a.partials[(int64_t)bx * a.E + e] = acc[k];
  }
}

template <int EPT>
__global__ void __launch_bounds__(kThreads) rowsweep_kernel(RowSweep a) {
  extern __shared__ double tile[];
  rowsweep_body<EPT>(a, blockIdx.x, blockIdx.y, tile);
}

// Batched persistent sweep: work item w is CTA item_cta[w] of problem
// item_req[w]; a fixed grid loops over the *nitems items.
template <int EPT>
__global__ void __launch_bounds__(kThreads)
    rowsweep_batched_kernel(const RowSweep *reqs, const int *item_req, const int *item_cta,
                            const int *nitems) {
  extern __shared__ double tile[];
  const int n = *nitems;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const RowSweep a = reqs[item_req[w]];
    rowsweep_body<EPT>(a, item_cta[w], 0, tile);
    __syncthreads();
  }
}

// Fixed-order sum of the per-CTA partials: C(e) = sum_{g=0}^{G-1} P[g][e];
// the Y^T Y part is written to both triangles.
__device__ __forceinline__ void reduce_body(const Reduce &a, int64_t e) {
  if (a.st != nullptr && a.st->done) return;
  if (e >= a.E) return;
  double s = 0.0;
  for (int g = 0; g < a.G; ++g) s += a.partials[(int64_t)g * a.E + e];
  const int q = a.q, p = a.p, ldc = q + p;
  const int64_t qp = (int64_t)q * p;
  if (e < qp) {
    a.C[(e % q) + (e / q) * ldc] = s;
  } else {
    int64_t f = e - qp;
    int j = (int)((sqrt(8.0 * (double)f + 1.0) - 1.0) * 0.5);
    while ((int64_t)(j + 1) * (j + 2) / 2 <= f) ++j;
    while ((int64_t)j * (j + 1) / 2 > f) --j;
    int i = (int)(f - (int64_t)j * (j + 1) / 2);
    a.C[(q + i) + (int64_t)j * ldc] = s;
    a.C[(q + j) + (int64_t)i * ldc] = s;
  }
}

__global__ void reduce_kernel(Reduce a) {
  reduce_body(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Batched reduction: work item w covers entries [64 chunk, 64 chunk + 64) of
// problem item_req[w] (chunk = item_chunk[w]).
__global__ void reduce_batched_kernel(const Reduce *reqs, const int *item_req, const int *item_chunk,
                                      const int *nitems) {
  const int n = *nitems;
  for (int w = blockIdx.x; w < n; w += gridDim.x)
    reduce_body(reqs[item_req[w]], (int64_t)item_chunk[w] * blockDim.x + threadIdx.x);
}

__device__ __forceinline__ void init_body(double *R, int64_t ldr, int p, double *B, int64_t ldb,
                                          int q, DevState *st, int t, int nt) {
  for (int e = t; e < p * p; e += nt) {
    const int i = e % p, j = e / p;
    R[i + (int64_t)j * ldr] = (i == j) ? 1.0 : 0.0;
  }
  if (B != nullptr)
    for (int e = t; e < q * p; e += nt) B[(e % q) + (int64_t)(e / q) * ldb] = 0.0;
  if (t == 0) {
    DevState z = {};
    *st = z;
  }
}

__global__ void init_kernel(double *R, int64_t ldr, int p, double *B, int64_t ldb, int q,
                            DevState *st) {
  init_body(R, ldr, p, B, ldb, q, st, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Batched init: CTA r (grid-stride) initialises problem r from its control
// descriptor (R block = I, B block = 0, state cleared).
__global__ void init_batched_kernel(const Ctrl *reqs, const int *nreq) {
  const int n = *nreq;
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const Ctrl c = reqs[r];
    init_body(c.R, c.ldr, c.p, c.B, c.ldb, c.q, c.st, threadIdx.x, blockDim.x);
  }
}

// SM count of the current device (cached per device).
int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  cudaGetDevice(&dev);
  const bool cached = dev >= 0 && dev < 64;
  int sms = cached ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (sms == 0) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    if (cached) cache[dev].store(sms, std::memory_order_relaxed);
  }
  return sms;
}

void rowsweep_geometry(int q, int p, int *tile_rows, int *lds, size_t *smem) {
  const int W = q + p;
  int s = W | 1;  // odd stride in doubles
  int tr = (int)(196608 / (8 * (size_t)s));
  tr = std::min(tr, 64);
  tr = std::max(8, tr & ~7);
  *tile_rows = tr;
  *lds = s;
  *smem = (size_t)tr * s * sizeof(double);
}

int rowsweep_grid(int64_t m, int tile_rows) {
  const int64_t tiles = (m + tile_rows - 1) / tile_rows;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 2));
}

template <int EPT>
static cudaError_t launch_ept(const RowSweep &a, dim3 grid, size_t smem, cudaStream_t s) {
  static KernelAttr attr;
  set_smem_attr(attr, rowsweep_kernel<EPT>, 200 * 1024, false);
  rowsweep_kernel<EPT><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rowsweep(const RowSweep &a, int grid, cudaStream_t s) {
  const size_t smem = (size_t)a.tile_rows * a.lds * sizeof(double);
  const int64_t per = (a.E + kThreads - 1) / kThreads;
  int ept;
  if (per <= 1) ept = 1;
  else if (per <= 2) ept = 2;
  else if (per <= 4) ept = 4;
  else if (per <= 8) ept = 8;
  else if (per <= 16) ept = 16;
  else ept = 33;
  const int64_t gy = std::max<int64_t>(1, (a.E + (int64_t)kThreads * ept - 1) / ((int64_t)kThreads * ept));
  if (a.do_trsm && gy != 1) return cudaErrorInvalidValue;  // caller splits the sweep
  dim3 g(grid, (unsigned)gy);
  switch (ept) {
    case 1: return launch_ept<1>(a, g, smem, s);
    case 2: return launch_ept<2>(a, g, smem, s);
    case 4: return launch_ept<4>(a, g, smem, s);
    case 8: return launch_ept<8>(a, g, smem, s);
    case 16: return launch_ept<16>(a, g, smem, s);
    default: return launch_ept<33>(a, g, smem, s);
  }
}

cudaError_t launch_rowsweep_batched(const RowSweep *reqs, const int *item_req, const int *item_cta,
                                    const int *nitems, int grid, size_t smem, cudaStream_t s) {
  static KernelAttr attr;
  set_smem_attr(attr, rowsweep_batched_kernel<kBatchEPT>, 200 * 1024, false);
  rowsweep_batched_kernel<kBatchEPT><<<grid, kThreads, smem, s>>>(reqs, item_req, item_cta, nitems);
  return cudaGetLastError();
}

cudaError_t launch_reduce_batched(const Reduce *reqs, const int *item_req, const int *item_chunk,
                                  const int *nitems, int grid, cudaStream_t s) {
  reduce_batched_kernel<<<grid, 64, 0, s>>>(reqs, item_req, item_chunk, nitems);
  return cudaGetLastError();
}

cudaError_t launch_init_batched(const Ctrl *reqs, const int *nreq, int grid, cudaStream_t s) {
  init_batched_kernel<<<grid, 256, 0, s>>>(reqs, nreq);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const Reduce &a, cudaStream_t s) {
  const int bs = 64;
  const int64_t blocks = (a.E + bs - 1) / bs;
  reduce_kernel<<<(unsigned)blocks, bs, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_init(double *R, int64_t ldr, int p, double *B, int64_t ldb, int q,
                        DevState *st, cudaStream_t s) {
  init_kernel<<<8, 256, 0, s>>>(R, ldr, p, B, ldb, q, st);
  return cudaGetLastError();
}

}  // namespace cqr
