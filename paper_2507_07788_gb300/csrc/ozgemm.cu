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
//   (orders 2..5 with unit 2^91, 6..10 with unit 2^56), then each entry is
//   rounded to FP64 once.
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

constexpr int kGmTR = 64;              // tile rows
constexpr int kGmDigits = 9;
constexpr int kGmThreads = 256;        // 8 warps, one CTA per SM
constexpr int kGmWarps = kGmThreads / 32;

// Work units: strips of 16 tile rows x JB output columns, times groups of
// orders: NT = 64 -> 8 strips x 1 group; NT = 32, 16 -> 4 strips x 2 groups
// (even and odd orders).
template <int NT>
struct GmGeom {
  static constexpr int JB = (NT >= 32) ? 32 : 16;
  static constexpr int NI = kGmTR / 16;
  static constexpr int NJ = NT / JB;
  static constexpr int strips = NI * NJ;
  static constexpr int groups = (strips >= 8) ? 1 : 2;
  static constexpr int LDK = NT + 8;   // bf16 stride of a digit-plane row (k contiguous)
};

template <int NT>
__host__ __device__ constexpr size_t ozgemm_smem(void) {
  return sizeof(uint16_t) * (size_t)kGmDigits * (NT + kGmTR) * GmGeom<NT>::LDK  // T and Y digit planes
         + sizeof(double) * (size_t)NT * kGmTR                                   // FP64 Y tile
         + sizeof(int) * (size_t)(2 * NT + 10 * kGmTR);                         // exponents, flags, scales
}

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

}  // namespace

// One CTA: rows [bx * rows_per_cta, ...) of Y in tiles of 64, Q = Y T.
template <int NT>
__global__ void __launch_bounds__(kGmThreads, 1) ozgemm_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  using G = GmGeom<NT>;
  constexpr int LDK = G::LDK;
  constexpr int NTILE = G::JB / 8;
  constexpr int SLOTS = 4 * NTILE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t *planesT = (uint16_t *)smem;                                  // [9][NT cols j][LDK k]
  uint16_t *planesY = planesT + (size_t)kGmDigits * NT * LDK;            // [9][64 rows r][LDK k]
  double *tile = (double *)(planesY + (size_t)kGmDigits * kGmTR * LDK);  // [NT k][64 r]
  int *fcol = (int *)(tile + (size_t)NT * kGmTR);                       // [NT]
  int *erow = fcol + NT;                                                 // [64]
  int *bad = erow + kGmTR;                                               // [64]
  int *cs = bad + kGmTR;                                                 // [NT] column scales
  int *epart = cs + NT;                                                  // [4][64] partial row maxima
  int *bpart = epart + 4 * kGmTR;                                        // [4][64] partial flags

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n = a.p;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  if (row0 >= row1) return;

  // ---- first tile in flight while T is split
  auto stage = [&](int64_t r0) {
    const int nr = (int)min((int64_t)kGmTR, row1 - r0);
    for (int e = t; e < kGmTR * NT; e += kGmThreads) {
      const int r = e % kGmTR, k = e / kGmTR;
      const bool in = (r < nr) && (k < n);
      const double *src = in ? a.Yin + (r0 + r) + (int64_t)k * a.ldyin : a.Yin;
      cp_async8(tile + k * kGmTR + r, src, in ? 8 : 0);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  stage(row0);

  // ---- D T (n x n, upper, ld n): column exponents, then 9 digit planes
  for (int k = t; k < NT; k += kGmThreads) cs[k] = (k < n) ? a.Tscale[k] : 0;
  for (int j = warp; j < NT; j += kGmWarps) {
    int mx = 1;
    for (int k = lane; k < n; k += 32)
      if (j < n) mx = max(mx, align_exp((unsigned long long)__double_as_longlong(a.Tinv[k + (int64_t)j * n])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) fcol[j] = mx;
  }
  __syncthreads();
  for (int e = t; e < NT * (NT / 2); e += kGmThreads) {
    const int j = e / (NT / 2), k = 2 * (e % (NT / 2));
    unsigned long long b[2] = {0ull, 0ull};
    for (int h = 0; h < 2; ++h)
      if (j < n && k + h < n) b[h] = (unsigned long long)__double_as_longlong(a.Tinv[(k + h) + (int64_t)j * n]);
    const unsigned long long V0 = digits63(b[0], fcol[j], 0), V1 = digits63(b[1], fcol[j], 0);
    const uint32_t sg = ((uint32_t)(b[0] >> 63) << 15) | ((uint32_t)(b[1] >> 63) << 31);
#pragma unroll
    for (int d = 0; d < kGmDigits; ++d)
      *(uint32_t *)(planesT + ((size_t)d * NT + j) * LDK + k) = digit_pair_bf16(V0, V1, d, sg);
  }

  const int strip = warp / G::groups, grp = warp % G::groups;
  const int ib = strip / G::NJ, jb = strip % G::NJ;
  const int i0 = ib * 16, j0 = jb * G::JB;

  for (int64_t r0 = row0; r0 < row1; r0 += kGmTR) {
    const int nr = (int)min((int64_t)kGmTR, row1 - r0);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // ---- row exponents and non-finite rows: thread (r, quarter) scans 1/4
    // of row r (lanes read consecutive rows: no bank conflicts)
    {
      constexpr int KQ = NT / 4;
      const int r = t & (kGmTR - 1), qk = t >> 6;
      int mx = kNoExp, bd = 0;
#pragma unroll 4
      for (int k = qk * KQ; k < (qk + 1) * KQ; ++k) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(tile[k * kGmTR + r]);
        bd |= (((b >> 52) & 0x7FF) == 0x7FF);
        mx = max(mx, scaled_exp(b, cs[k]));
      }
      epart[qk * kGmTR + r] = mx;
      bpart[qk * kGmTR + r] = bd;
    }
    __syncthreads();
    // ---- split the tile into 9 digit planes (row r, k contiguous): a thread
    // takes 8 consecutive k of one row and writes one 16-byte word per digit
    for (int e = t; e < kGmTR * (NT / 8); e += kGmThreads) {
      const int r = e & (kGmTR - 1), k0 = 8 * (e / kGmTR);
      const int er = max(max(epart[r], epart[kGmTR + r]), max(epart[2 * kGmTR + r], epart[3 * kGmTR + r]));
      if (k0 == 0) {
        erow[r] = er;
        bad[r] = bpart[r] | bpart[kGmTR + r] | bpart[2 * kGmTR + r] | bpart[3 * kGmTR + r];
      }
      unsigned long long V[8];
      uint32_t sg[4];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(tile[(k0 + h) * kGmTR + r]);
        V[h] = digits63(b, er, cs[k0 + h]);
        if (h & 1) sg[h >> 1] |= (uint32_t)(b >> 63) << 31;
        else sg[h >> 1] = (uint32_t)(b >> 63) << 15;
      }
#pragma unroll
      for (int d = 0; d < kGmDigits; ++d) {
        uint4 w;
        w.x = digit_pair_bf16(V[0], V[1], d, sg[0]);
        w.y = digit_pair_bf16(V[2], V[3], d, sg[1]);
        w.z = digit_pair_bf16(V[4], V[5], d, sg[2]);
        w.w = digit_pair_bf16(V[6], V[7], d, sg[3]);
        *(uint4 *)(planesY + ((size_t)d * kGmTR + r) * LDK + k0) = w;
      }
    }
    __syncthreads();
    // ---- the next tile loads while this one is multiplied
    if (r0 + kGmTR < row1) stage(r0 + kGmTR);

    // ---- tensor-core products: order d = s + t, T_d in one FP32 accumulator
    long long acc_hi[SLOTS], acc_lo[SLOTS];
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) {
      acc_hi[k] = 0;
      acc_lo[k] = 0;
    }
    int tv[NTILE][4];
#pragma unroll
    for (int d = 2; d <= 10; ++d) {
      if (G::groups == 2 && (d & 1) != grp) continue;
      float c[NTILE][4];
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll 1
      for (int s = (d > kGmDigits + 1) ? d - kGmDigits : 1; s <= kGmDigits && s < d; ++s) {
        const int tt = d - s;
        const uint16_t *As = planesY + ((size_t)(s - 1) * kGmTR + i0) * LDK;
        const uint16_t *Bt = planesT + ((size_t)(tt - 1) * NT + j0) * LDK;
        // T is upper triangular: rows k >= j0 + JB of its strip are zero
        const int kend = min(NT, j0 + G::JB);
#pragma unroll 2
        for (int ks = 0; ks < kend; ks += 16) {
          uint32_t a0, a1, a2, a3;
          {
            const int mi = lane >> 3, rr = lane & 7;
            const uint16_t *pa = As + ((mi & 1) * 8 + rr) * LDK + ks + (mi >> 1) * 8;
            ldsm_x4(smem_u32(pa), a0, a1, a2, a3);
          }
#pragma unroll
          for (int nt = 0; nt < NTILE; nt += 2) {
            uint32_t b0, b1, b2, b3;
            const int mi = lane >> 3, rr = lane & 7;
            const uint16_t *pb = Bt + ((nt + (mi >> 1)) * 8 + rr) * LDK + ks + (mi & 1) * 8;
            ldsm_x4(smem_u32(pb), b0, b1, b2, b3);
            mma_bf16(c[nt], a0, a1, a2, a3, b0, b1);
            mma_bf16(c[nt + 1], a0, a1, a2, a3, b2, b3);
          }
        }
      }
      // drain: hi word = orders 2..5 (weight 2^(7 (5 - d))), lo word = orders
      // 6..10 (weight 2^(7 (10 - d))); with one group the pairs (2,3), (4,5),
      // (6,7), (8,9) are first combined in int32 as T_d 2^7 + T_(d+1)
      const bool hi = d <= 5;
      if (G::groups == 1 && (d == 2 || d == 4 || d == 6 || d == 8)) {
#pragma unroll
        for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) tv[nt][r] = f2i(c[nt][r]);
      } else {
        const bool paired = (G::groups == 1 && d != 10);
        const int shl = hi ? 7 * (5 - d) : 7 * (10 - d);
#pragma unroll
        for (int nt = 0; nt < NTILE; ++nt)
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
    // ---- combine the groups exactly (reusing the Y planes), round once
    __syncthreads();  // every warp is done reading planesY
    long long *ohi = (long long *)planesY;  // [NT j][64 r]
    long long *olo = ohi + (size_t)NT * kGmTR;
    if (G::groups > 1) {
      for (int e = t; e < NT * kGmTR; e += kGmThreads) {
        ohi[e] = 0;
        olo[e] = 0;
      }
      __syncthreads();
    }
    for (int g = 0; g < G::groups; ++g) {
      if (grp == g) {
#pragma unroll
        for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int rr = i0 + (lane >> 2) + ((r >> 1) << 3);
            const int jj = j0 + nt * 8 + 2 * (lane & 3) + (r & 1);
            const int k = nt * 4 + r;
            if (G::groups == 1) {
              ohi[rr + jj * kGmTR] = acc_hi[k];
              olo[rr + jj * kGmTR] = acc_lo[k];
            } else {
              ohi[rr + jj * kGmTR] += acc_hi[k];
              olo[rr + jj * kGmTR] += acc_lo[k];
            }
          }
      }
      __syncthreads();
    }
    // Q_rj = (hi 2^35 + lo) 2^(e_r + f_j - 2114); coalesced column stores
    for (int e = t; e < kGmTR * n; e += kGmThreads) {
      const int r = e % kGmTR, j = e / kGmTR;
      if (r >= nr) continue;
      const double v = bad[r] ? __longlong_as_double(0x7FF8000000000000ll)
                              : fixed_to_double(ohi[r + j * kGmTR], olo[r + j * kGmTR], 35,
                                                erow[r] + fcol[j] - 2114);
      a.Yout[(r0 + r) + (int64_t)j * a.ldyout] = v;
    }
    __syncthreads();  // planesY (ohi/olo) is rewritten by the next tile
  }
}

template <int NT>
static cudaError_t launch_gm(const RowSweep &a, int grid, cudaStream_t s) {
  constexpr size_t smem = ozgemm_smem<NT>();
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(ozgemm_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_done = true;
  }
  ozgemm_kernel<NT><<<grid, kGmThreads, smem, s>>>(a);
  return cudaGetLastError();
}

int ozgemm_grid(int64_t m) {
  const int64_t tiles = (m + kGmTR - 1) / kGmTR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms()));
}

int ozgemm_tile_rows() { return kGmTR; }

double ozgemm_tc_flops_per_row(int n) {
  (void)n;  // one kernel shape (NT = 64) serves 33 <= n <= 64
  constexpr int NT = 64, JB = GmGeom<NT>::JB;
  double kcols = 0.0;  // sum over column strips of (strip width x k extent)
  for (int j0 = 0; j0 < NT; j0 += JB) kcols += (double)JB * std::min(NT, j0 + JB);
  int pairs = 0;
  for (int d = 2; d <= 10; ++d) pairs += std::min(d - 1, kGmDigits) - std::max(1, d - kGmDigits) + 1;
  return 2.0 * pairs * kcols;
}

// Q = Y T for 33 <= n <= 64 (a.Yin, a.Yout, a.Tinv, a.Tscale, a.m, a.p,
// a.rows_per_cta); narrower blocks use the FP64 substitution.
cudaError_t launch_ozgemm(const RowSweep &a, int grid, cudaStream_t s) {
  if (a.Tinv == nullptr || a.Tscale == nullptr) return cudaErrorInvalidValue;
  if (a.p >= kOzGemmMinN && a.p <= 64) return launch_gm<64>(a, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace cqr
