// Digit cache of a basis and the cross Gramian of narrow appends that reads
// it (Alg. 2: B~ = Q_in^T Y and Y^T Y in one sweep).
//
// Why: an append of p <= 16 columns to a basis of q columns does about 2 q p
// FP64 FMAs per row and pass; splitting Q_in's rows into digits on every
// pass would cost more issue slots than those FMAs.  The columns of Q_in do
// not change once appended, so their digits are formed once and kept.
//
// Cache (per basis, opt-in): column k of Q_in with E_k = the largest biased
// exponent of the column (zeros and subnormals count as 1) is written as
//   q_rk = sign * V * 2^(E_k - 1078),  V < 2^56 (56 bits below the column
//   maximum, truncated),
// V in 7 balanced base-256 digits, V = sum_{i=0..6} D_i 2^(8 (6 - i)), D_0 in
// [0, 256], D_i in [-128, 127] (128 added to the six low bytes, read back
// minus 128), each with the element's sign: exact in bf16.  Planes
// [7][n_max][ldc] of bf16 (ldc = m rounded up to 64, padding rows zero):
// 14 bytes per entry.
//
// Cross Gramian: Z = [Q_in Y] against Y (p <= 16, padded to 16).  Cached
// columns keep their fixed E_k; Y's columns keep a running maximum exponent
// per CTA and are split per 64-row tile in the same representation.
// Products z_c y_j = 2^(E_c + E_j - 2156) sum_{s,t} D_s(z) D_t(y)
//   2^(8 (12 - s - t)); the 28 ordered digit pairs of order s + t <= 6 are
//   kept (the rest lie below 2^-53 of the leading term).
// Exactness: an order's tile sum is at most 64 (2 * 2^15 + 5 * 2^14) =
//   9 * 2^20 < 2^24 (the top digit pairs with at most 2^8 * 2^7), exact in
//   one FP32 accumulator; orders (0,1), (2,3), (4,5) are combined in int32
//   and added into two int64 words (orders 0..3 and 4..6), rescaled by exact
//   shifts when a column of Y grows its exponent, and each entry of a CTA's
//   partial is rounded to FP64 once.
// Work split: CTA (g, b) takes the rows of row group g and the 64 Z columns
//   [64 b, 64 b + 64); warp w owns Z columns 16 (w / 2) .. + 15 against Y
//   columns 8 (w % 2) .. + 7 and forms all orders.  A fixed-order sum of
//   the row groups' partials ((q + p) x p, ld q + p) gives C.
// Non-finite entries of Y make every partial of the CTA NaN (the control
// kernel then reports a breakdown, as the FP64 path does).
#include <algorithm>

#include "cqr_internal.cuh"
#include "ozbalanced.cuh"
#include "ozdigits.cuh"

namespace cqr {

using namespace oz;

namespace {

// Four 8x8 b16 matrices, each stored with its rows as the fragment's
// columns (the transposing form).
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                          uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}

constexpr int kCD = 7;                                // digits
constexpr int kCTR = 64;                              // tile rows
constexpr int kCLD = kCTR + 8;                        // bf16 stride of a plane column
constexpr int kCZ = 64;                               // Z columns per CTA
constexpr int kCY = 16;                               // padded width of Y
constexpr int kCThreads = 256;
constexpr int kCMaxOrder = 6;

constexpr size_t kCSmem = sizeof(double) * (size_t)kCY * kCTR          // FP64 tile of Y
                          + sizeof(uint16_t) * (size_t)kCD * kCZ * kCLD  // Z digit planes
                          + sizeof(uint16_t) * (size_t)kCD * kCY * kCLD  // Y digit planes
                          + sizeof(int) * (size_t)(2 * kCZ + 2 * kCY + 4);

}  // namespace

// ---- cache fill: E_k of columns k0 .. k0 + p - 1.  CTA (x, y) scans rows
// [x rows_per_cta, ...) of column k0 + y with eight independent loads in
// flight per thread and folds its maximum into Qe[k] (cleared to 0 before
// the launch; every CTA contributes at least 1) with atomicMax.
__global__ void __launch_bounds__(256) cache_exp_kernel(const double *Q, int64_t ldq, int64_t m, int k0,
                                                        int64_t rows_per_cta, int *Qe) {
  __shared__ int wm[8];
  const int k = k0 + (int)blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(m, r0 + rows_per_cta);
  const unsigned long long *col = (const unsigned long long *)(Q + (int64_t)k * ldq);
  int mx = 1;
  int64_t r = r0 + threadIdx.x;
  for (; r + 7 * 256 < r1; r += 8 * 256) {
    unsigned long long v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(col + r + u * 256);
#pragma unroll
    for (int u = 0; u < 8; ++u) mx = max(mx, (int)((v[u] >> 52) & 0x7FF));
  }
  for (; r < r1; r += 256) mx = max(mx, (int)((__ldg(col + r) >> 52) & 0x7FF));
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int v = 1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = max(v, wm[w]);
    atomicMax(Qe + k, v);
  }
}

// ---- cache fill: the digits of columns k0 .. k0 + p - 1, two rows per item
__global__ void __launch_bounds__(256) cache_digits_kernel(const double *Q, int64_t ldq, int64_t m, int k0,
                                                           int p, const int *Qe, uint16_t *Qd, int64_t ldc,
                                                           int64_t plane) {
  const int64_t half = ldc / 2, items = (int64_t)p * half;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < items;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = k0 + (int)(e / half);
    const int64_t r = 2 * (e % half);
    const int E = Qe[k];
    unsigned long long W[2];
    float sg[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned long long b =
          (r + h < m) ? (unsigned long long)__double_as_longlong(Q[(r + h) + (int64_t)k * ldq]) : 0ull;
      W[h] = cwords(b, E);
      sg[h] = (b >> 63) ? -1.0f : 1.0f;
    }
#pragma unroll
    for (int d = 0; d < kCD; ++d) {
      const __nv_bfloat162 pr = __floats2bfloat162_rn(cdigit(W[0], d, sg[0]), cdigit(W[1], d, sg[1]));
      *(uint32_t *)(Qd + (int64_t)d * plane + (int64_t)k * ldc + r) = *(const uint32_t *)&pr;
    }
  }
}

cudaError_t launch_cache_fill(const double *Q, int64_t ldq, int64_t m, int k0, int p, int *Qe, uint16_t *Qd,
                              int64_t ldc, int64_t plane, cudaStream_t s) {
  if (p < 1 || (ldc & 63) != 0 || ldc < m) return cudaErrorInvalidValue;
  // about four CTAs per SM over all columns, each slice at least 2048 rows
  const int64_t slices = std::max<int64_t>(
      1, std::min<int64_t>((m + 2047) / 2048, (4 * (int64_t)num_sms() + p - 1) / p));
  const int64_t rpc = (m + slices - 1) / slices;
  cudaError_t e = cudaMemsetAsync(Qe + k0, 0, sizeof(int) * (size_t)p, s);
  if (e != cudaSuccess) return e;
  cache_exp_kernel<<<dim3((unsigned)slices, (unsigned)p), 256, 0, s>>>(Q, ldq, m, k0, rpc, Qe);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t items = (int64_t)p * (ldc / 2);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 4 * (int64_t)num_sms()));
  cache_digits_kernel<<<grid, 256, 0, s>>>(Q, ldq, m, k0, p, Qe, Qd, ldc, plane);
  return cudaGetLastError();
}

// ---- cross Gramian [Q_in Y]^T Y with Q_in's digits from the cache
__global__ void __launch_bounds__(kCThreads, 2) ozcgram_kernel(RowSweep a, const uint16_t *Qd, int64_t ldc,
                                                               int64_t plane, const int *Qe, int nzb) {
  if (a.st != nullptr && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double *ytile = (double *)smem;                                      // [16 cols][64 rows]
  uint16_t *zpl = (uint16_t *)(ytile + (size_t)kCY * kCTR);            // [7][64 cols][kCLD]
  uint16_t *ypl = zpl + (size_t)kCD * kCZ * kCLD;                      // [7][16 cols][kCLD]
  int *Ez = (int *)(ypl + (size_t)kCD * kCY * kCLD);                   // [64] exponent of Z column
  int *Edz = Ez + kCZ;                                                 // [64] growth this tile
  int *Ey = Edz + kCZ;                                                 // [16]
  int *Edy = Ey + kCY;                                                 // [16]
  int *flag = Edy + kCY;                                               // [1]

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int q = a.q, p = a.p, nz = q + p;
  const int zb = (int)(blockIdx.x % nzb);
  const int64_t grp_id = blockIdx.x / nzb;
  const int64_t row0 = grp_id * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  const int z0 = kCZ * zb;                  // first Z column of this CTA
  const int zc_live = min(kCZ, nz - z0);   // Z columns that hold data
  const int zc_cached = max(0, min(kCZ, q - z0));  // of which come from the cache

  for (int j = t; j < kCY; j += kCThreads) {
    Ey[j] = 1;
    Edy[j] = 0;
  }
  for (int c = t; c < kCZ; c += kCThreads) {
    Ez[c] = (c < zc_cached) ? Qe[z0 + c] : 1;
    Edz[c] = 0;
  }
  if (t == 0) *flag = 0;
  // planes and tile columns that never hold data stay zero
  for (int e = t; e < kCD * kCZ * (kCLD / 2); e += kCThreads) {
    const int c = (e / (kCLD / 2)) % kCZ;
    if (c >= zc_live) ((uint32_t *)zpl)[e] = 0u;
  }
  for (int e = t; e < kCD * kCY * (kCLD / 2); e += kCThreads) {
    const int j = (e / (kCLD / 2)) % kCY;
    if (j >= p) ((uint32_t *)ypl)[e] = 0u;
  }
  for (int e = t; e < kCY * kCTR; e += kCThreads)
    if (e / kCTR >= p) ytile[e] = 0.0;

  long long acc_hi[4], acc_lo[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    acc_hi[k] = 0;
    acc_lo[k] = 0;
  }
  const int zs = warp >> 1, yt = warp & 1;
  const int i0 = 16 * zs, j0 = 8 * yt;
  // a row group without rows still writes its (zero) partial: the reduction
  // sums every row group's
  __syncthreads();

  for (int64_t r0 = row0; r0 < row1; r0 += kCTR) {
    const int nr = (int)min((int64_t)kCTR, row1 - r0);
    // ---- stage Y (FP64, zero padded) and the cached Z columns' digits
    for (int e = t; e < p * kCTR; e += kCThreads) {
      const int i = e % kCTR, j = e / kCTR;
      const bool in = i < nr;
      const double *src = in ? a.Yin + (r0 + i) + (int64_t)j * a.ldyin : a.Yin;
      cp_async8(ytile + j * kCTR + i, src, in ? 8 : 0);
    }
    for (int e = t; e < kCD * zc_cached * (kCTR / 8); e += kCThreads) {
      const int ch = e % (kCTR / 8), c = (e / (kCTR / 8)) % zc_cached, d = e / ((kCTR / 8) * zc_cached);
      cp_async16(zpl + ((size_t)d * kCZ + c) * kCLD + 8 * ch,
                 Qd + (int64_t)d * plane + (int64_t)(z0 + c) * ldc + r0 + 8 * ch);
    }
    cp_async_wait_all();
    __syncthreads();
    // ---- running exponents of Y's columns
    for (int j = warp; j < p; j += kCThreads / 32) {
      const uint32_t *hw = (const uint32_t *)(ytile + j * kCTR) + 1;
      int mx = 1;
      for (int i = lane; i < kCTR; i += 32) mx = max(mx, (int)((hw[2 * i] >> 20) & 0x7FF));
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) {
        const int old = Ey[j];
        const int nw = max(old, mx);
        Edy[j] = nw - old;
        Ey[j] = nw;
        if (mx == 0x7FF) *flag = 1;
        const int c = q + j - z0;  // Y column j as a Z column of this CTA
        if (c >= 0 && c < kCZ) {
          Edz[c] = nw - old;
          Ez[c] = nw;
        }
      }
    }
    __syncthreads();
    // ---- split Y into its digit planes (and into Z's, where Z holds Y)
    for (int e = t; e < (kCTR / 2) * p; e += kCThreads) {
      const int i = 2 * (e % (kCTR / 2)), j = e / (kCTR / 2);
      const int E = Ey[j];
      unsigned long long W[2];
      float sg[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(ytile[j * kCTR + i + h]);
        W[h] = cwords(b, E);
        sg[h] = (b >> 63) ? -1.0f : 1.0f;
      }
      const int c = q + j - z0;
      const bool inz = c >= 0 && c < kCZ;
#pragma unroll
      for (int d = 0; d < kCD; ++d) {
        const __nv_bfloat162 pr = __floats2bfloat162_rn(cdigit(W[0], d, sg[0]), cdigit(W[1], d, sg[1]));
        const uint32_t v = *(const uint32_t *)&pr;
        *(uint32_t *)(ypl + ((size_t)d * kCY + j) * kCLD + i) = v;
        if (inz) *(uint32_t *)(zpl + ((size_t)d * kCZ + c) * kCLD + i) = v;
      }
    }
    __syncthreads();
    // ---- rescale where an exponent grew, then every order on the tensor cores
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int zi = i0 + (lane >> 2) + ((r >> 1) << 3);
      const int yj = j0 + 2 * (lane & 3) + (r & 1);
      shift_pair(acc_hi[r], acc_lo[r], Edz[zi] + Edy[yj], 24);
    }
    const int mi = lane >> 3, rr = lane & 7;
    // every order at once: per k-step the warp loads each Y digit and each
    // Z digit once
    float c[kCMaxOrder + 1][4];
#pragma unroll
    for (int o = 0; o <= kCMaxOrder; ++o) c[o][0] = c[o][1] = c[o][2] = c[o][3] = 0.0f;
#pragma unroll 1
    for (int ks = 0; ks < kCTR; ks += 16) {
      uint32_t bf[kCD][2];
#pragma unroll
      for (int tt = 0; tt < kCD; ++tt)
        ldsm_x2(smem_u32(ypl + ((size_t)tt * kCY + j0 + rr) * kCLD + ks + (mi & 1) * 8), bf[tt][0], bf[tt][1]);
#pragma unroll
      for (int sd = 0; sd < kCD; ++sd) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(smem_u32(zpl + ((size_t)sd * kCZ + i0 + (mi & 1) * 8 + rr) * kCLD + ks + (mi >> 1) * 8), a0,
                a1, a2, a3);
#pragma unroll
        for (int tt = 0; tt + sd <= kCMaxOrder; ++tt) mma_bf16(c[sd + tt], a0, a1, a2, a3, bf[tt][0], bf[tt][1]);
      }
    }
    // drain: orders (0,1), (2,3), (4,5) paired in int32, order 6 alone; hi
    // holds orders 0..3 (unit: order 3), lo orders 4..6
#pragma unroll
    for (int o = 1; o <= kCMaxOrder; o += 2) {
      const bool hi = o <= 3;
      const int shl = hi ? 8 * (3 - o) : 8 * (kCMaxOrder - o);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const long long w = (long long)(f2i(c[o - 1][r]) * 256 + f2i(c[o][r]));
        if (hi) acc_hi[r] += w << shl;
        else acc_lo[r] += w << shl;
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) acc_lo[r] += (long long)f2i(c[kCMaxOrder][r]);
    __syncthreads();  // the next tile restages the planes
  }

  // ---- C_cj = (hi 2^24 + lo) 2^(E_c + E_j - 2108), one rounding per entry
  const bool bad = *flag != 0;
  double *P = a.partials + grp_id * (int64_t)nz * p;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int zi = i0 + (lane >> 2) + ((r >> 1) << 3);
    const int yj = j0 + 2 * (lane & 3) + (r & 1);
    if (zi >= zc_live || yj >= p) continue;
    const double v = bad ? __longlong_as_double(0x7FF8000000000000ll)
                         : fixed_to_double(acc_hi[r], acc_lo[r], 24, Ez[zi] + Ey[yj] - 2108);
    P[(z0 + zi) + (int64_t)yj * nz] = v;
  }
}

// ---- projection P = Q_in B~ from the cached digits, then y <- (y - P) R~^{-1}
// (Alg. 2) in FP64, for p <= 16 and q <= 256.
//
// B~ is scaled by rows, B'_kj = B~_kj 2^(E_k - Emax) (exact powers of two,
// Emax = max_k E_k), so that every cached digit of q_rk meets B' in one unit:
//   P_rj = 2^(Emax + f_j - 2108) sum_{s,t} sum_k D_s(q_rk) D_t(B'_kj)
//   2^(8 (6 - s - t)),
// with B' in 7 balanced digits against f_j, its column's largest exponent.
// The 28 ordered digit pairs of order <= 6 are kept; an order's sum over 64 k
// stays below 9 * 2^20 (exact in FP32) and is drained into two int64 words
// per entry every 64 k; each P_rj is rounded to FP64 once.  Then each row
// runs the FP64 substitution of the row sweep: y_j - P_rj, minus the
// earlier solved entries times R~, times 1 / R~_jj.
constexpr int kCPK = 256 + 8;  // bf16 stride of B''s digit columns (q <= 256)
constexpr int kCProjMaxQ = 256;

// B' digits: planes [7][16][kCPK] (zero outside q x p), f_j, Emax.  One CTA.
__global__ void __launch_bounds__(256) cproj_prep_kernel(const double *Bt, int q, int p, const int *Qe,
                                                         uint16_t *Bd, int *fexp) {
  __shared__ int s_emax;
  __shared__ int s_f[kCY];
  const int t = threadIdx.x;
  if (t < 32) {
    int mx = 1;
    for (int k = t; k < q; k += 32) mx = max(mx, Qe[k]);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (t == 0) s_emax = mx;
  }
  if (t < kCY) s_f[t] = 1;
  __syncthreads();
  const int emax = s_emax;
  // column maxima of B' (one warp per column)
  for (int j = t >> 5; j < p; j += 8) {
    int mx = 1;
    for (int k = t & 31; k < q; k += 32) {
      const double v = ldexp(Bt[k + (int64_t)j * q], Qe[k] - emax);
      const unsigned long long b = (unsigned long long)__double_as_longlong(v);
      mx = max(mx, (int)((b >> 52) & 0x7FF));
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((t & 31) == 0) s_f[j] = mx;
  }
  __syncthreads();
  // digits, two k per item
  for (int e = t; e < kCY * (kCPK / 2); e += 256) {
    const int j = e / (kCPK / 2), k = 2 * (e % (kCPK / 2));
    unsigned long long W[2];
    float sg[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool in = j < p && k + h < q;
      const double v = in ? ldexp(Bt[(k + h) + (int64_t)j * q], Qe[k + h] - emax) : 0.0;
      const unsigned long long b = (unsigned long long)__double_as_longlong(v);
      W[h] = cwords(b, s_f[j]);
      sg[h] = (b >> 63) ? -1.0f : 1.0f;
    }
#pragma unroll
    for (int d = 0; d < kCD; ++d) {
      const __nv_bfloat162 pr = __floats2bfloat162_rn(cdigit(W[0], d, sg[0]), cdigit(W[1], d, sg[1]));
      *(uint32_t *)(Bd + ((size_t)d * kCY + j) * kCPK + k) = *(const uint32_t *)&pr;
    }
  }
  if (t < kCY) fexp[t] = s_f[t];
  if (t == 0) fexp[kCY] = emax;
}

constexpr size_t kCPSmem = sizeof(uint16_t) * (size_t)kCD * kCY * kCPK          // B' digits
                           + 2 * sizeof(uint16_t) * (size_t)kCD * kCZ * kCLD     // Q digit chunks (x2)
                           + sizeof(double) * (size_t)kCTR * (kCY + 1)           // P tile
                           + sizeof(double) * (size_t)(kCY * kCY + kCY)          // R~, 1 / diag
                           + sizeof(int) * (size_t)(kCY + 4);

__global__ void __launch_bounds__(kCThreads, 1) ozcproj_kernel(RowSweep a, const uint16_t *Qd, int64_t ldc,
                                                               int64_t plane, const uint16_t *Bd,
                                                               const int *fexp) {
  if (a.st != nullptr && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t *bpl = (uint16_t *)smem;                                   // [7][16][kCPK]
  uint16_t *zbuf = bpl + (size_t)kCD * kCY * kCPK;                    // [2][7][64 k][kCLD]
  double *Pt = (double *)(zbuf + 2 * (size_t)kCD * kCZ * kCLD);       // [64 rows][17]
  double *Rs = Pt + (size_t)kCTR * (kCY + 1);                         // [16 x 16], then [16]
  double *Rd = Rs + kCY * kCY;
  int *fj = (int *)(Rd + kCY);                                        // [16], then Emax

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int q = a.q, p = a.p;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  if (row0 >= row1) return;  // nothing to write for an empty row range

  for (int e = t; e < kCD * kCY * (kCPK / 8); e += kCThreads)
    cp_async16(bpl + 8 * e, Bd + 8 * e);
  for (int e = t; e < p * p; e += kCThreads) Rs[(e % p) * kCY + e / p] = a.Rt[e];  // Rs[k * 16 + j] = R~_kj
  for (int j = t; j < p; j += kCThreads) Rd[j] = a.Rdinv[j];
  if (t <= kCY) fj[t] = fexp[t];

  const int nch = (q + kCZ - 1) / kCZ;  // 64-k chunks of Q_in
  const int64_t ntiles = (row1 - row0 + kCTR - 1) / kCTR;
  const int64_t nsteps = ntiles * nch;
  // chunk loads: digit d of columns k0 .. k0 + 63 (zero past q), rows of the tile
  auto issue = [&](int64_t step) {
    if (step >= nsteps) return;
    const int64_t r0 = row0 + (step / nch) * kCTR;
    const int k0 = (int)(step % nch) * kCZ;
    uint16_t *dst = zbuf + (size_t)(step & 1) * kCD * kCZ * kCLD;
    const int kc = min(kCZ, q - k0);
    for (int e = t; e < kCD * kCZ * (kCTR / 8); e += kCThreads) {
      const int ch = e % (kCTR / 8), c = (e / (kCTR / 8)) % kCZ, d = e / ((kCTR / 8) * kCZ);
      uint16_t *dd = dst + ((size_t)d * kCZ + c) * kCLD + 8 * ch;
      if (c < kc) cp_async16(dd, Qd + (int64_t)d * plane + (int64_t)(k0 + c) * ldc + r0 + 8 * ch);
      else *(uint4 *)dd = make_uint4(0u, 0u, 0u, 0u);
    }
  };
  issue(0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");

  // warp -> 16 rows (rs) and one 8-column tile of P (ct)
  const int rs = warp >> 1, ct = warp & 1;
  const int i0 = 16 * rs, j0 = 8 * ct;
  const int mi = lane >> 3, rr = lane & 7;
  long long acc_hi[4] = {0, 0, 0, 0}, acc_lo[4] = {0, 0, 0, 0};

  for (int64_t step = 0; step < nsteps; ++step) {
    issue(step + 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    const uint16_t *zp = zbuf + (size_t)(step & 1) * kCD * kCZ * kCLD;
    const int k0 = (int)(step % nch) * kCZ;
    // every order at once: per k-step each Q digit and each B' digit once
    float c[kCMaxOrder + 1][4];
#pragma unroll
    for (int o = 0; o <= kCMaxOrder; ++o) c[o][0] = c[o][1] = c[o][2] = c[o][3] = 0.0f;
#pragma unroll 1
    for (int ks = 0; ks < kCZ; ks += 16) {
      uint32_t bf[kCD][2];
#pragma unroll
      for (int td = 0; td < kCD; ++td)
        ldsm_x2(smem_u32(bpl + ((size_t)td * kCY + j0 + rr) * kCPK + k0 + ks + (mi & 1) * 8), bf[td][0],
                bf[td][1]);
#pragma unroll
      for (int sd = 0; sd < kCD; ++sd) {
        uint32_t a0, a1, a2, a3;
        // [k][row] storage, transposed loads: block (mi & 1) rows +8, (mi >> 1) k +8
        ldsm_x4_t(smem_u32(zp + ((size_t)sd * kCZ + ks + (mi >> 1) * 8 + rr) * kCLD + i0 + (mi & 1) * 8), a0,
                  a1, a2, a3);
#pragma unroll
        for (int td = 0; td + sd <= kCMaxOrder; ++td) mma_bf16(c[sd + td], a0, a1, a2, a3, bf[td][0], bf[td][1]);
      }
    }
#pragma unroll
    for (int o = 1; o <= kCMaxOrder; o += 2) {
      const bool hi = o <= 3;
      const int shl = hi ? 8 * (3 - o) : 8 * (kCMaxOrder - o);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const long long w = (long long)(f2i(c[o - 1][r]) * 256 + f2i(c[o][r]));
        if (hi) acc_hi[r] += w << shl;
        else acc_lo[r] += w << shl;
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) acc_lo[r] += (long long)f2i(c[kCMaxOrder][r]);
    if (step % nch == nch - 1) {
      // ---- the tile's P, rounded once, then the FP64 row solve
      const int64_t r0 = row0 + (step / nch) * kCTR;
      const int nr = (int)min((int64_t)kCTR, row1 - r0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int ri = i0 + (lane >> 2) + ((r >> 1) << 3);
        const int cj = j0 + 2 * (lane & 3) + (r & 1);
        Pt[ri * (kCY + 1) + cj] = (cj < p) ? fixed_to_double(acc_hi[r], acc_lo[r], 24, fj[kCY] + fj[cj] - 2108)
                                           : 0.0;
        acc_hi[r] = 0;
        acc_lo[r] = 0;
      }
      __syncthreads();
      if (t < nr) {
        const int64_t row = r0 + t;
        double y[kCY];
#pragma unroll
        for (int j = 0; j < kCY; ++j) y[j] = (j < p) ? a.Yin[row + (int64_t)j * a.ldyin] : 0.0;
#pragma unroll
        for (int j = 0; j < kCY; ++j) {
          if (j < p) {
            double s = y[j] - Pt[t * (kCY + 1) + j];
            for (int k = 0; k < j; ++k) s -= y[k] * Rs[k * kCY + j];
            y[j] = s * Rd[j];
            a.Yout[row + (int64_t)j * a.ldyout] = y[j];
          }
        }
      }
    }
    __syncthreads();  // the buffer of this step is refilled two steps on; P is reused
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// P = Q_in B~ and y <- (y - P) R~^{-1} for p <= 16, q <= 256 (a.m, a.q, a.p,
// a.Yin, a.Yout, a.Bt, a.Rt, a.Rdinv, a.rows_per_cta, a.st); Bd (7 x 16 x
// kCPK bf16) and fexp (17 ints) are scratch for B''s digits.
cudaError_t launch_ozcproj(const RowSweep &a, const uint16_t *Qd, int64_t ldc, int64_t plane, const int *Qe,
                           uint16_t *Bd, int *fexp, int grid, cudaStream_t s) {
  if (a.p < 1 || a.p > kCY || a.q < 1 || a.q > kCProjMaxQ || Qd == nullptr || Qe == nullptr) return cudaErrorInvalidValue;
  if ((ldc & 63) != 0 || ldc < a.m || (a.rows_per_cta % kCTR) != 0) return cudaErrorInvalidValue;
  cproj_prep_kernel<<<1, 256, 0, s>>>(a.Bt, a.q, a.p, Qe, Bd, fexp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static KernelAttr attr;
  set_smem_attr(attr, ozcproj_kernel, (int)kCPSmem, true);
  ozcproj_kernel<<<grid, kCThreads, kCPSmem, s>>>(a, Qd, ldc, plane, Bd, fexp);
  return cudaGetLastError();
}

size_t ozcproj_scratch_bytes() { return sizeof(uint16_t) * (size_t)kCD * kCY * kCPK + 256; }

int ozcproj_grid(int64_t m) {
  const int64_t tiles = (m + kCTR - 1) / kCTR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms()));
}

int ozcgram_zblocks(int q, int p) { return (q + p + kCZ - 1) / kCZ; }

int ozcgram_grid(int64_t m, int q, int p) {
  const int64_t tiles = (m + kCTR - 1) / kCTR;
  const int nzb = ozcgram_zblocks(q, p);
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, std::max<int64_t>(1, 2 * num_sms() / nzb)));
}

int ozcgram_tile_rows() { return kCTR; }

// C partials of [Q_in Y]^T Y for p <= 16 with the cached digits of Q_in's q
// columns (a.m, a.q, a.p, a.Yin, a.ldyin, a.partials, a.rows_per_cta, a.st);
// `groups` row groups.
cudaError_t launch_ozcgram(const RowSweep &a, const uint16_t *Qd, int64_t ldc, int64_t plane, const int *Qe,
                           int groups, cudaStream_t s) {
  if (a.p < 1 || a.p > kCY || a.q < 1 || Qd == nullptr || Qe == nullptr) return cudaErrorInvalidValue;
  if ((ldc & 63) != 0 || ldc < a.m || (a.rows_per_cta % kCTR) != 0) return cudaErrorInvalidValue;
  const int nzb = ozcgram_zblocks(a.q, a.p);
  static KernelAttr attr;
  set_smem_attr(attr, ozcgram_kernel, (int)kCSmem, true);
  ozcgram_kernel<<<groups * nzb, kCThreads, kCSmem, s>>>(a, Qd, ldc, plane, Qe, nzb);
  return cudaGetLastError();
}

}  // namespace cqr
