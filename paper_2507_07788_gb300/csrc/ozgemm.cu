// Q = Y T on the tensor cores, T = R~^{-1}: the triangular solve of Alg. 1
// line 9 in the form the paper's implementation uses (an explicit triangular
// inverse, then a matrix product; App. A), with the product done exactly on
// bf16 digits (the Ozaki splitting scheme).
//
// Why: GB300 retires ~2 FP64 FMAs per SM per clock, so a substitution costs
// n^2 FP64 instructions per row; here a row costs no FP64 instruction at all.
//
// Scaling: the product is formed as (Y D^-1)(D T) with D = diag(2^c_k) and
//   c_k = floor(log2 sqrt(X_kk)) from the pass's Gramian (the control kernel
//   stores D T and c): columns of Y and rows of T of very different scales
//   are balanced first, exactly.
// Representation:
//   row r of the scaled Y tile, with e_r = the largest scaled exponent in the
//   row (biased exponent of y_rk minus c_k, zeros ignored):
//     y_rk 2^-c_k = sign * V * 2^(e_r - 1085),  V = sum_{s=1..9} d_s 2^(63 - 7 s),
//   9 digits d_s in [0, 127] (63 bits below the row maximum, truncated);
//   column j of D T likewise with f_j = the largest exponent in the column.
// Products: Q_rj = 2^(e_r + f_j - 2170) sum_{s,t} sum_k d_s(y_rk) d_t(T_kj)
//   2^(126 - 7(s+t)); all ordered digit pairs with s + t <= 10 are kept.
// Exactness: for an order d the sum over k of its (d - 1) digit pairs is at
//   most 9 * 64 * 127^2 < 2^24: one FP32 mma.sync accumulator holds it
//   exactly.  Orders are combined exactly in int32 pairs and two int64 words
//   (orders 2..6 with unit 2^84, 7..10 with unit 2^56), the two warps that
//   share an output strip (one order group each) are summed exactly, and
//   each entry is rounded to FP64 once.
// Geometry: 32-row tiles, loaded straight from global memory into registers
//   (lanes read consecutive rows), 9 digit planes of the tile and of T in
//   shared memory (T's first 32 columns only keep k < 32: T is upper
//   triangular), 106 KB: two CTAs of 8 warps per SM.
// Error: the dropped digits (beyond 63 bits of the row or column maximum)
//   and the dropped orders (s + t >= 11) change an entry by at most about
//   2^-54 max_k |y_rk| max_k |T_kj|, below the error bound of an FP64 dot
//   product of length n.
// A row with a NaN or Inf entry gives a NaN row of Q.
#include <algorithm>

#include "cqr_internal.cuh"
#include "ozdigits.cuh"

namespace cqr {

using namespace oz;

namespace {

constexpr int kGmTR = 32;              // tile rows
constexpr int kGmDigits = 9;
constexpr int kGmThreads = 256;        // 8 warps, two CTAs per SM
constexpr int kGmNT = 64;              // padded width (33 <= n <= 64)
constexpr int kLdA = 40;               // bf16 stride of T's first 32 columns (k < 32 only)
constexpr int kLdB = 72;               // bf16 stride of T's last 32 columns and of Y's rows

constexpr size_t kGmSmem = sizeof(uint16_t) * (size_t)kGmDigits * 32 * kLdA      // T, columns 0..31
                           + sizeof(uint16_t) * (size_t)kGmDigits * 32 * kLdB    // T, columns 32..63
                           + sizeof(uint16_t) * (size_t)kGmDigits * kGmTR * kLdB  // Y tile digits
                           + sizeof(int) * (size_t)(2 * kGmNT + 2 * kGmTR + 16 * kGmTR);

constexpr int kNoExp = -(1 << 28);  // scaled exponent of a zero (below any real one)

// Scaled alignment exponent of x (bit pattern b) in a column scaled by 2^-c.
__device__ __forceinline__ int scaled_exp(unsigned long long b, int c) {
  if ((b & 0x7FFFFFFFFFFFFFFFull) == 0) return kNoExp;
  return align_exp(b) - c;
}

// Splits x (bit pattern b, column scale 2^-c) against the reference exponent
// eref into 9 digit magnitudes, V = (M << 10) >> (eref - (ev - c)).
__device__ __forceinline__ unsigned long long digits63(unsigned long long b, int eref, int c) {
  const int ef = (int)((b >> 52) & 0x7FF);
  unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  if (ef) M |= 0x10000000000000ull;
  if (ef == 0x7FF || M == 0) return 0ull;
  const int sh = eref - ((ef ? ef : 1) - c);
  return (sh >= 63) ? 0ull : ((M << 10) >> sh);
}

__device__ __forceinline__ uint32_t digit_pair_bf16(unsigned long long V0, unsigned long long V1, int d,
                                                    uint32_t sgnmask) {
  const float f0 = __int_as_float(0x4B000000 | (int)((V0 >> (56 - 7 * d)) & 127u)) - 8388608.0f;
  const float f1 = __int_as_float(0x4B000000 | (int)((V1 >> (56 - 7 * d)) & 127u)) - 8388608.0f;
  const __nv_bfloat162 pr = __floats2bfloat162_rn(f0, f1);
  return *(const uint32_t *)&pr | sgnmask;
}

// The 9 orders d = s + t in {2..10} split over two warps per output strip,
// balanced by their digit pairs (d - 1 each): {3, 4, 9, 10} (22 pairs) and
// {2, 5, 6, 7, 8} (23).  Within a group, (3,4), (9,10), (5,6) and (7,8) are
// combined in int32 as T_d 2^7 + T_(d+1) before the int64 words: hi holds
// orders 2..6 (weight 2^(7 (6 - d))), lo orders 7..10 (2^(7 (10 - d))).
__device__ __forceinline__ bool in_group(int grp, int d) {
  const bool g0 = (d == 3 || d == 4 || d == 9 || d == 10);
  return grp == 0 ? g0 : !g0;
}

}  // namespace

// One CTA: rows [bx * rows_per_cta, ...) of Y in tiles of 32, Q = (Y D^-1)(D T).
__global__ void __launch_bounds__(kGmThreads, 2) ozgemm_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  constexpr int NT = kGmNT;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t *planesT0 = (uint16_t *)smem;                                 // [9][32 cols][kLdA]
  uint16_t *planesT1 = planesT0 + (size_t)kGmDigits * 32 * kLdA;         // [9][32 cols][kLdB]
  uint16_t *planesY = planesT1 + (size_t)kGmDigits * 32 * kLdB;          // [9][32 rows][kLdB]
  int *fcol = (int *)(planesY + (size_t)kGmDigits * kGmTR * kLdB);      // [64]
  int *cs = fcol + NT;                                                   // [64] column scales
  int *erow = cs + NT;                                                   // [32]
  int *bad = erow + kGmTR;                                               // [32]
  int *epart = bad + kGmTR;                                              // [8][32] partial row maxima
  int *bpart = epart + 8 * kGmTR;                                        // [8][32] partial flags

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n = a.p;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  if (row0 >= row1) return;

  // ---- D T (n x n, upper, ld n): column exponents, then 9 digit planes
  // (columns j < 32 only meet rows k < 32 of the triangle)
  for (int k = t; k < NT; k += kGmThreads) cs[k] = (k < n) ? a.Tscale[k] : 0;
  for (int j = warp; j < NT; j += kGmThreads / 32) {
    int mx = 1;
    for (int k = lane; k < n; k += 32)
      if (j < n) mx = max(mx, align_exp((unsigned long long)__double_as_longlong(a.Tinv[k + (int64_t)j * n])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) fcol[j] = mx;
  }
  __syncthreads();
  for (int e = t; e < 32 * 16 + 32 * 32; e += kGmThreads) {
    const bool lo = e < 32 * 16;
    const int ee = lo ? e : e - 32 * 16;
    const int kp = lo ? 16 : 32;  // k pairs of this column half
    const int jl = ee / kp, k = 2 * (ee % kp), j = (lo ? 0 : 32) + jl;
    unsigned long long b[2] = {0ull, 0ull};
    for (int h = 0; h < 2; ++h)
      if (j < n && k + h < n) b[h] = (unsigned long long)__double_as_longlong(a.Tinv[(k + h) + (int64_t)j * n]);
    const unsigned long long V0 = digits63(b[0], fcol[j], 0), V1 = digits63(b[1], fcol[j], 0);
    const uint32_t sg = ((uint32_t)(b[0] >> 63) << 15) | ((uint32_t)(b[1] >> 63) << 31);
    uint16_t *dst = lo ? planesT0 + (size_t)jl * kLdA + k : planesT1 + (size_t)jl * kLdB + k;
    const size_t dstep = lo ? (size_t)32 * kLdA : (size_t)32 * kLdB;
#pragma unroll
    for (int d = 0; d < kGmDigits; ++d) *(uint32_t *)(dst + d * dstep) = digit_pair_bf16(V0, V1, d, sg);
  }

  // warp -> strip (16 rows x 32 columns) and order group
  const int strip = warp >> 1, grp = warp & 1;
  const int ib = strip >> 1, jb = strip & 1;
  const int i0 = ib * 16;
  const uint16_t *Tbase = jb ? planesT1 : planesT0;
  const int ldt = jb ? kLdB : kLdA;
  const int kend = jb ? 64 : 32;  // T is upper triangular
  // loader: thread (r, kc) holds 8 consecutive k of row r (lanes = rows)
  const int lr = t & (kGmTR - 1), kc = t >> 5, k0 = 8 * kc;

  for (int64_t r0 = row0; r0 < row1; r0 += kGmTR) {
    const int nr = (int)min((int64_t)kGmTR, row1 - r0);
    // ---- load 8 entries per thread (coalesced along rows), partial maxima
    unsigned long long bv[8];
    int mx = kNoExp, bd = 0;
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int k = k0 + h;
      bv[h] = (lr < nr && k < n) ? (unsigned long long)__double_as_longlong(a.Yin[(r0 + lr) + (int64_t)k * a.ldyin])
                                 : 0ull;
      bd |= (((bv[h] >> 52) & 0x7FF) == 0x7FF);
      mx = max(mx, scaled_exp(bv[h], cs[k]));
    }
    epart[kc * kGmTR + lr] = mx;
    bpart[kc * kGmTR + lr] = bd;
    __syncthreads();
    // ---- row exponent, then 9 digit planes (row r, k contiguous)
    {
      int er = kNoExp, bb = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        er = max(er, epart[q * kGmTR + lr]);
        bb |= bpart[q * kGmTR + lr];
      }
      if (kc == 0) {
        erow[lr] = er;
        bad[lr] = bb;
      }
      unsigned long long V[8];
      uint32_t sg[4];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        V[h] = digits63(bv[h], er, cs[k0 + h]);
        if (h & 1) sg[h >> 1] |= (uint32_t)(bv[h] >> 63) << 31;
        else sg[h >> 1] = (uint32_t)(bv[h] >> 63) << 15;
      }
#pragma unroll
      for (int d = 0; d < kGmDigits; ++d) {
        uint4 w;
        w.x = digit_pair_bf16(V[0], V[1], d, sg[0]);
        w.y = digit_pair_bf16(V[2], V[3], d, sg[1]);
        w.z = digit_pair_bf16(V[4], V[5], d, sg[2]);
        w.w = digit_pair_bf16(V[6], V[7], d, sg[3]);
        *(uint4 *)(planesY + ((size_t)d * kGmTR + lr) * kLdB + k0) = w;
      }
    }
    __syncthreads();

    // ---- tensor-core products of this warp's order group
    long long acc_hi[16], acc_lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      acc_hi[k] = 0;
      acc_lo[k] = 0;
    }
    int tv[4][4];
#pragma unroll
    for (int d = 2; d <= 10; ++d) {
      if (!in_group(grp, d)) continue;
      float c[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll 1
      for (int s = 1; s < d && s <= kGmDigits; ++s) {
        const int tt = d - s;
        const uint16_t *As = planesY + ((size_t)(s - 1) * kGmTR + i0) * kLdB;
        const uint16_t *Bt = Tbase + (size_t)(tt - 1) * 32 * ldt;
#pragma unroll 2
        for (int ks = 0; ks < kend; ks += 16) {
          uint32_t a0, a1, a2, a3;
          {
            const int mi = lane >> 3, rr = lane & 7;
            const uint16_t *pa = As + ((mi & 1) * 8 + rr) * kLdB + ks + (mi >> 1) * 8;
            ldsm_x4(smem_u32(pa), a0, a1, a2, a3);
          }
#pragma unroll
          for (int nt = 0; nt < 4; nt += 2) {
            uint32_t b0, b1, b2, b3;
            const int mi = lane >> 3, rr = lane & 7;
            const uint16_t *pb = Bt + ((nt + (mi >> 1)) * 8 + rr) * ldt + ks + (mi & 1) * 8;
            ldsm_x4(smem_u32(pb), b0, b1, b2, b3);
            mma_bf16(c[nt], a0, a1, a2, a3, b0, b1);
            mma_bf16(c[nt + 1], a0, a1, a2, a3, b2, b3);
          }
        }
      }
      // drain (see in_group): the first order of a pair waits in tv
      if (d == 3 || d == 5 || d == 7 || d == 9) {
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) tv[nt][r] = f2i(c[nt][r]);
      } else {
        const bool paired = (d != 2);
        const bool hi = d <= 6;
        const int shl = hi ? 7 * (6 - d) : 7 * (10 - d);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int v = f2i(c[nt][r]);
            const long long w = paired ? (long long)(tv[nt][r] * 128 + v) : (long long)v;
            const int k = nt * 4 + r;
            if (hi) acc_hi[k] += w << shl;
            else acc_lo[k] += w << shl;
          }
      }
    }
    // ---- combine the two order groups exactly (reusing the Y planes), round once
    __syncthreads();  // every warp is done reading planesY
    constexpr int kLdO = kGmTR + 1;  // odd stride: the four column lanes of a fragment hit distinct banks
    long long *ohi = (long long *)planesY;  // [64 j][kLdO]
    long long *olo = ohi + (size_t)NT * kLdO;
    for (int g = 0; g < 2; ++g) {
      if (grp == g) {
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int rr = i0 + (lane >> 2) + ((r >> 1) << 3);
            const int jj = jb * 32 + nt * 8 + 2 * (lane & 3) + (r & 1);
            const int k = nt * 4 + r;
            if (g == 0) {
              ohi[rr + jj * kLdO] = acc_hi[k];
              olo[rr + jj * kLdO] = acc_lo[k];
            } else {
              ohi[rr + jj * kLdO] += acc_hi[k];
              olo[rr + jj * kLdO] += acc_lo[k];
            }
          }
      }
      __syncthreads();
    }
    // Q_rj = (hi 2^28 + lo) 2^(e_r + f_j - 2114); one column's rows per warp
    for (int e = t; e < kGmTR * n; e += kGmThreads) {
      const int r = e % kGmTR, j = e / kGmTR;
      if (r >= nr) continue;
      const double v = bad[r] ? __longlong_as_double(0x7FF8000000000000ll)
                              : fixed_to_double(ohi[r + j * kLdO], olo[r + j * kLdO], 28,
                                                erow[r] + fcol[j] - 2114);
      a.Yout[(r0 + r) + (int64_t)j * a.ldyout] = v;
    }
    __syncthreads();  // planesY (ohi/olo), epart and erow are rewritten by the next tile
  }
}

static cudaError_t launch_gm(const RowSweep &a, int grid, cudaStream_t s) {
  static KernelAttr attr;
  set_smem_attr(attr, ozgemm_kernel, (int)kGmSmem, true);
  ozgemm_kernel<<<grid, kGmThreads, kGmSmem, s>>>(a);
  return cudaGetLastError();
}

int ozgemm_grid(int64_t m) {
  const int64_t tiles = (m + kGmTR - 1) / kGmTR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 2 * (int64_t)num_sms()));
}

int ozgemm_tile_rows() { return kGmTR; }

double ozgemm_tc_flops_per_row(int n) {
  (void)n;  // one kernel shape (64 columns) serves 33 <= n <= 64
  const double kcols = 32.0 * 32 + 32.0 * 64;  // column halves x their k extent
  int pairs = 0;
  for (int d = 2; d <= 10; ++d) pairs += std::min(d - 1, kGmDigits) - std::max(1, d - kGmDigits) + 1;
  return 2.0 * pairs * kcols;
}

// Q = Y T for 33 <= n <= 64 (a.Yin, a.Yout, a.Tinv, a.Tscale, a.m, a.p,
// a.rows_per_cta); narrower blocks use the FP64 substitution.
cudaError_t launch_ozgemm(const RowSweep &a, int grid, cudaStream_t s) {
  if (a.Tinv == nullptr || a.Tscale == nullptr) return cudaErrorInvalidValue;
  if (a.p >= kOzGemmMinN && a.p <= kGmNT) return launch_gm(a, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace cqr
