// FP32 Gramian sweep for the mixed-precision first pass.
//
// The first (shifted) pass of sCholQR3 only needs its Gramian to the accuracy
// its shift covers (the role of the shift in Alg. 1): with a shift
// sized for FP32 roundoff the Gramian can be formed from FP32 data.  On GB300
// an FP32 FMA is ~67x cheaper than an FP64 one, so this sweep runs at memory
// speed where the FP64 sweep is bound by the FP64 pipe.  Everything after the
// Gramian (norm estimate, shifted Cholesky, the triangular solve and all
// later passes) stays FP64.
//
// Arithmetic, per CTA (fixed order, deterministic):
//   * inputs are truncated to FP32 from their bit patterns on the integer
//     pipe (relative error < 2^-23), values below 2^-126 flush to zero;
//   * each tile of 64 rows is summed in FP32 FMAs, row order ascending;
//   * tile sums are combined with Kahan compensated summation, so the error
//     of a CTA partial is that of a 64 + 2 deep sum;
//   * the partial (sum - compensation) is written as FP64 and the existing
//     fixed-order FP64 reduction adds the CTA partials.
#include <algorithm>

#include "cqr_internal.cuh"

namespace cqr {

// FP64 -> FP32 by truncation of the bit pattern (no FP64 instruction).
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
  if (e < -126) return __int_as_float((int)sign);
  if (e > 127) {
    // Inf stays Inf, NaN stays NaN, finite overflow becomes Inf
    const bool nan = (e == 1024) && ((b & 0xFFFFFFFFFFFFFull) != 0);
    return __int_as_float((int)(sign | (nan ? 0x7FC00000u : 0x7F800000u)));
  }
  const unsigned mant = (unsigned)((b >> 29) & 0x7FFFFFull);
  return __int_as_float((int)(sign | ((unsigned)(e + 127) << 23) | mant));
}

// FP32 -> FP64, exact, from the bit pattern (normal numbers, zero, Inf, NaN).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long mant = (unsigned long long)(u & 0x7FFFFFu) << 29;
  unsigned long long bits;
  if (e == 0) bits = sign;  // zero (FP32 subnormals flushed)
  else if (e == 0xFF) bits = sign | (0x7FFull << 52) | mant;
  else bits = sign | ((unsigned long long)(e + 896) << 52) | mant;
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void entry_columns32(int64_t e, int q, int p, int &ca, int &cb) {
  const int64_t qp = (int64_t)q * p;
  if (e < qp) {
    ca = (int)(e % q);
    cb = q + (int)(e / q);
  } else {
    const int64_t f = e - qp;
    int j = (int)((sqrtf(8.0f * (float)f + 1.0f) - 1.0f) * 0.5f);
    while ((int64_t)(j + 1) * (j + 2) / 2 <= f) ++j;
    while ((int64_t)j * (j + 1) / 2 > f) --j;
    ca = q + (int)(f - (int64_t)j * (j + 1) / 2);
    cb = q + j;
  }
}

template <int EPT>
__global__ void __launch_bounds__(kThreads) gram32_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  extern __shared__ float tilef[];
  const int t = threadIdx.x;
  const int q = a.q, p = a.p, W = q + p, lds = a.lds, TR = a.tile_rows;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);

  uint32_t idx[EPT];
  float hi[EPT], cc[EPT];
  const int64_t ebase = (int64_t)blockIdx.y * (kThreads * EPT);
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = ebase + t + (int64_t)k * kThreads;
    int ca = 0, cb = 0;
    if (e < a.E) entry_columns32(e, q, p, ca, cb);
    idx[k] = (uint32_t)ca | ((uint32_t)cb << 16);
    hi[k] = 0.0f;
    cc[k] = 0.0f;
  }
  for (int64_t r0 = row0; r0 < row1; r0 += TR) {
    const int nr = (int)min((int64_t)TR, row1 - r0);
    for (int e = t; e < TR * W; e += kThreads) {
      const int i = e % TR, c = e / TR;
      float v = 0.0f;
      if (i < nr)
        v = f64_to_f32_trunc((c < q) ? a.Qin[(r0 + i) + (int64_t)c * a.ldqin]
                                     : a.Yin[(r0 + i) + (int64_t)(c - q) * a.ldyin]);
      tilef[i * lds + c] = v;
    }
    __syncthreads();
    float ts[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) ts[k] = 0.0f;
    for (int i = 0; i < nr; ++i) {
      const float *row = tilef + i * lds;
#pragma unroll
      for (int k = 0; k < EPT; ++k) ts[k] = fmaf(row[idx[k] & 0xFFFFu], row[idx[k] >> 16], ts[k]);
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      // Kahan: hi + (-cc) tracks the exact sum of the tile sums
      const float y = ts[k] - cc[k];
      const float s = hi[k] + y;
      cc[k] = (s - hi[k]) - y;
      hi[k] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = ebase + t + (int64_t)k * kThreads;
    if (e < a.E) a.partials[(int64_t)blockIdx.x * a.E + e] = f32_to_f64_bits(hi[k]) - f32_to_f64_bits(cc[k]);
  }
}

void gram32_geometry(int q, int p, int *tile_rows, int *lds, size_t *smem) {
  const int W = q + p;
  const int s = W | 1;
  int tr = (int)(196608 / (4 * (size_t)s));
  tr = std::min(tr, 64);
  tr = std::max(8, tr & ~7);
  *tile_rows = tr;
  *lds = s;
  *smem = (size_t)tr * s * sizeof(float);
}

template <int EPT>
static cudaError_t launch32_ept(const RowSweep &a, dim3 grid, size_t smem, cudaStream_t s) {
  static KernelAttr attr;
  set_smem_attr(attr, gram32_kernel<EPT>, 200 * 1024, false);
  gram32_kernel<EPT><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gram32(const RowSweep &a, int grid, cudaStream_t s) {
  const size_t smem = (size_t)a.tile_rows * a.lds * sizeof(float);
  const int64_t per = (a.E + kThreads - 1) / kThreads;
  int ept;
  if (per <= 1) ept = 1;
  else if (per <= 2) ept = 2;
  else if (per <= 4) ept = 4;
  else if (per <= 8) ept = 8;
  else if (per <= 16) ept = 16;
  else ept = 33;
  const int64_t gy = std::max<int64_t>(1, (a.E + (int64_t)kThreads * ept - 1) / ((int64_t)kThreads * ept));
  dim3 g(grid, (unsigned)gy);
  switch (ept) {
    case 1: return launch32_ept<1>(a, g, smem, s);
    case 2: return launch32_ept<2>(a, g, smem, s);
    case 4: return launch32_ept<4>(a, g, smem, s);
    case 8: return launch32_ept<8>(a, g, smem, s);
    case 16: return launch32_ept<16>(a, g, smem, s);
    default: return launch32_ept<33>(a, g, smem, s);
  }
}

}  // namespace cqr
