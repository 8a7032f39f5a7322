// Q = Y T on the tensor cores, T = R~^{-1}: the triangular solve of Alg. 1
// in the form the paper's implementation uses (an explicit triangular
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
//     y_rk 2^-c_k = sign * V * 2^(e_r - 1085),  V < 2^63 (63 bits below the
//     row maximum, truncated),
//   V written in 8 balanced base-256 digits, V = sum_{i=0..7} D_i 2^(8 (7 - i)),
//   D_0 in [0, 128] and D_i in [-128, 127] for i >= 1 (add 128 to each of
//   the 7 low bytes, then take bytes minus 128: one byte permute per digit);
//   signed digits of magnitude <= 128 are exact in bf16.  Column j of D T
//   likewise with f_j = the largest exponent in the column.
// Products: Q_rj = 2^(e_r + f_j - 2170) sum_{i,i'} sum_k D_i(y_rk) D_i'(T_kj)
//   2^(8 (14 - i - i')); the 36 ordered digit pairs of order o = i + i' <= 7
//   are kept.
// Exactness: for an order o the sum over k of its o + 1 digit pairs is at
//   most 8 * 64 * 128^2 = 2^23: one FP32 mma.sync accumulator holds it
//   exactly.  Orders are combined exactly in int32 pairs and two int64 words
//   (orders 0..3 with unit 2^88, 4..7 with unit 2^56), and each entry is
//   rounded to FP64 once.
// Geometry: 32-row tiles, loaded straight from global memory into registers
//   (lanes read consecutive rows), 8 digit planes of the tile and of T in
//   shared memory (T's first 32 columns only keep k < 32: T is upper
//   triangular), 96 KB: two CTAs of 8 warps per SM.  A warp owns 16 rows
//   and two 8-column tiles whose triangle extents add up to the same five
//   k-steps of 16 for every warp; it forms all orders itself, in two rounds
//   (orders 0..3, then 4..7) whose accumulators fit in registers, loading
//   each Y digit and each T digit once per k-step.
// Error: the dropped orders (o >= 8) change an entry by at most about
//   2^-55 max_k |y_rk| max_k |T_kj|, below the error bound of an FP64 dot
//   product of length n.
// A row with a NaN or Inf entry gives a NaN row of Q.
#include <algorithm>

#include "cqr_internal.cuh"
#include "ozdigits.cuh"

namespace cqr {

using namespace oz;

namespace {

constexpr int kGmTR = 32;              // tile rows
constexpr int kGmDigits = 8;   // balanced base-256 digits of 63 bits
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
// eref into its 63-bit magnitude V = (M << 10) >> (eref - (ev - c)).
__device__ __forceinline__ unsigned long long digits63(unsigned long long b, int eref, int c) {
  const int ef = (int)((b >> 52) & 0x7FF);
  unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  if (ef) M |= 0x10000000000000ull;
  if (ef == 0x7FF || M == 0) return 0ull;
  const int sh = eref - ((ef ? ef : 1) - c);
  return (sh >= 63) ? 0ull : ((M << 10) >> sh);
}

// Balanced digit i of two elements as a packed bf16 pair, each with the
// sign of its element (s = +-1).  W = V + 0x0080808080808080 (128 added to
// each of the seven low bytes; V < 2^63, so no carry leaves the top byte);
// digit i is byte 7 - i of W, minus 128 for i >= 1.  The byte is placed in
// an FP32 2^23 + x by one byte permute, and s (2^23 + x) - s (2^23 + b) =
// s (x - b) exactly in one FMA.
constexpr unsigned long long kBalance = 0x0080808080808080ull;
__device__ __forceinline__ float balanced_digit(unsigned long long W, int i, float s) {
  const uint32_t word = (i < 4) ? (uint32_t)(W >> 32) : (uint32_t)W;
  const uint32_t byte = 3 - (i & 3);
  const float x = __int_as_float((int)__byte_perm(word, 0x4B000000u, 0x7440u | byte));
  return fmaf(x, s, -s * (i == 0 ? 8388608.0f : 8388736.0f));
}
__device__ __forceinline__ uint32_t digit_pair_bf16(unsigned long long W0, unsigned long long W1, int i,
                                                    float s0, float s1) {
  const __nv_bfloat162 pr = __floats2bfloat162_rn(balanced_digit(W0, i, s0), balanced_digit(W1, i, s1));
  return *(const uint32_t *)&pr;
}

// The products of orders DLO..DHI (digits 1..NS of both operands) for one
// warp's 16 rows, over k-steps kk0..kk1-1: c[d - DLO][tile] accumulates
// sum_{s + t = d} d_s(Y) d_t(D T) exactly.  MODE 0: both column tiles (one
// x4 load of a T digit covers both); 1: tile B alone; 2: tile A alone.
template <int DLO, int DHI, int NS, int MODE>
__device__ __forceinline__ void gm_steps(float (&c)[DHI - DLO + 1][2][4], uint32_t aY, uint32_t strY,
                                         uint32_t bT, uint32_t strT, int kk0, int kk1) {
#pragma unroll 1
  for (int kk = kk0; kk < kk1; ++kk) {
    const uint32_t ko = 32u * kk;
    uint32_t A[NS][4];
#pragma unroll
    for (int s = 0; s < NS; ++s) ldsm_x4(aY + s * strY + ko, A[s][0], A[s][1], A[s][2], A[s][3]);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      // digit t + 1 of T meets digits s + 1 with DLO <= s + t + 2 <= DHI
      const int slo = max(0, DLO - 2 - t), shi = min(NS - 1, DHI - 2 - t);
      if (slo > shi) continue;
      uint32_t b0, b1, b2, b3;
      if (MODE == 0) ldsm_x4(bT + t * strT + ko, b0, b1, b2, b3);
      else ldsm_x2(bT + t * strT + ko, b0, b1);
#pragma unroll
      for (int s = slo; s <= shi; ++s) {
        const int d = s + t + 2 - DLO;
        if (MODE == 0) {
          mma_bf16(c[d][0], A[s][0], A[s][1], A[s][2], A[s][3], b0, b1);
          mma_bf16(c[d][1], A[s][0], A[s][1], A[s][2], A[s][3], b2, b3);
        } else {
          mma_bf16(c[d][MODE == 1 ? 1 : 0], A[s][0], A[s][1], A[s][2], A[s][3], b0, b1);
        }
      }
    }
  }
}

// All of one round of orders for a warp: both tiles below tile A's extent
// kA, tile B alone up to kB; or tile A alone when tile B lies past n.
template <int DLO, int DHI, int NS>
__device__ __forceinline__ void gm_orders(float (&c)[DHI - DLO + 1][2][4], uint32_t aY, uint32_t strY,
                                          uint32_t bA, uint32_t bB, uint32_t bAB, uint32_t strAB,
                                          uint32_t strT0, uint32_t strT1, int kA, int kB, bool needB) {
#pragma unroll
  for (int d = 0; d <= DHI - DLO; ++d)
#pragma unroll
    for (int tl = 0; tl < 2; ++tl) c[d][tl][0] = c[d][tl][1] = c[d][tl][2] = c[d][tl][3] = 0.0f;
  if (needB) {
    gm_steps<DLO, DHI, NS, 0>(c, aY, strY, bAB, strAB, 0, kA);
    gm_steps<DLO, DHI, NS, 1>(c, aY, strY, bB, strT1, kA, kB);
  } else {
    gm_steps<DLO, DHI, NS, 2>(c, aY, strY, bA, strT0, 0, kA);
  }
}

}  // namespace

// One CTA: rows [bx * rows_per_cta, ...) of Y in tiles of 32, Q = (Y D^-1)(D T).
__global__ void __launch_bounds__(kGmThreads, 2) ozgemm_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  constexpr int NT = kGmNT;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t *planesT0 = (uint16_t *)smem;                                 // [8][32 cols][kLdA]
  uint16_t *planesT1 = planesT0 + (size_t)kGmDigits * 32 * kLdA;         // [8][32 cols][kLdB]
  uint16_t *planesY = planesT1 + (size_t)kGmDigits * 32 * kLdB;          // [8][32 rows][kLdB]
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

  // ---- D T (n x n, upper, ld n): column exponents, then 8 digit planes
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
    const unsigned long long V0 = digits63(b[0], fcol[j], 0) + kBalance, V1 = digits63(b[1], fcol[j], 0) + kBalance;
    const float sg0 = (b[0] >> 63) ? -1.0f : 1.0f, sg1 = (b[1] >> 63) ? -1.0f : 1.0f;
    uint16_t *dst = lo ? planesT0 + (size_t)jl * kLdA + k : planesT1 + (size_t)jl * kLdB + k;
    const size_t dstep = lo ? (size_t)32 * kLdA : (size_t)32 * kLdB;
#pragma unroll
    for (int d = 0; d < kGmDigits; ++d) *(uint32_t *)(dst + d * dstep) = digit_pair_bf16(V0, V1, d, sg0, sg1);
  }

  // warp -> 16 rows (ib) and two 8-column tiles of equal triangle work: tile
  // tA = cp (columns 8 cp .. 8 cp + 7, k < 16 (cp / 2 + 1)) and tile
  // tB = 7 - cp (k < 16 (tB / 2 + 1)): five k-steps of 16 per digit pair
  const int ib = warp & 1, cp = warp >> 1;
  const int i0 = ib * 16, tA = cp, tB = 7 - cp;
  const bool needB = 8 * tB < n;
  const int kA = tA / 2 + 1;
  const int kB = min(tB / 2 + 1, (n + 15) / 16);
  const int mi = lane >> 3, rr = lane & 7;
  // per-lane ldmatrix addresses at digit 1, k-step 0 (the k-step adds 32 bytes)
  const uint32_t aY = smem_u32(planesY + (size_t)(i0 + (mi & 1) * 8 + rr) * kLdB + (mi >> 1) * 8);
  const uint32_t bA = smem_u32(planesT0 + (size_t)(8 * tA + rr) * kLdA + (mi & 1) * 8);
  const uint32_t bB = smem_u32(planesT1 + (size_t)(8 * (tB - 4) + rr) * kLdB + (mi & 1) * 8);
  const uint32_t bAB = (mi < 2) ? bA : bB;  // x4: tile A (lanes 0-15), tile B (16-31)
  constexpr uint32_t kStrY = 2u * kGmTR * kLdB, kStrT0 = 2u * 32 * kLdA, kStrT1 = 2u * 32 * kLdB;
  const uint32_t strAB = (mi < 2) ? kStrT0 : kStrT1;
  // loader: thread (r, kc) holds 8 consecutive k of row r (lanes = rows)
  const int lr = t & (kGmTR - 1), kc = t >> 5, k0 = 8 * kc;

  for (int64_t r0 = row0; r0 < row1; r0 += kGmTR) {
    const int nr = (int)min((int64_t)kGmTR, row1 - r0);
    // ---- load 8 entries per thread (coalesced along rows), partial maxima.
    // The previous tile's readers of epart/bpart passed the barrier below.
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
    __syncthreads();  // also: every warp is done with the previous tile's planes
    // ---- row exponent, then 8 digit planes (row r, k contiguous)
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
      float sg[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        V[h] = digits63(bv[h], er, cs[k0 + h]) + kBalance;
        sg[h] = (bv[h] >> 63) ? -1.0f : 1.0f;
      }
#pragma unroll
      for (int d = 0; d < kGmDigits; ++d) {
        uint4 w;
        w.x = digit_pair_bf16(V[0], V[1], d, sg[0], sg[1]);
        w.y = digit_pair_bf16(V[2], V[3], d, sg[2], sg[3]);
        w.z = digit_pair_bf16(V[4], V[5], d, sg[4], sg[5]);
        w.w = digit_pair_bf16(V[6], V[7], d, sg[6], sg[7]);
        *(uint4 *)(planesY + ((size_t)d * kGmTR + lr) * kLdB + k0) = w;
      }
    }
    __syncthreads();

    // ---- orders 0..3 (digits 0..3), drained into hi; then orders 4..7
    // (all 8 digits), drained into lo.  Each k-step loads the warp's Y
    // digits once and each T digit once.
    long long hi[8], lo[8];
    {
      float c[4][2][4];
      gm_orders<2, 5, 4>(c, aY, kStrY, bA, bB, bAB, strAB, kStrT0, kStrT1, kA, kB, needB);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int tl = o >> 2, r = o & 3;
        const int t0 = f2i(c[0][tl][r]), t1 = f2i(c[1][tl][r]), t2 = f2i(c[2][tl][r]);
        const int t3 = f2i(c[3][tl][r]);
        hi[o] = ((long long)(t0 * 256 + t1) << 16) + (long long)(t2 * 256 + t3);
      }
    }
    {
      float c[4][2][4];
      gm_orders<6, 9, 8>(c, aY, kStrY, bA, bB, bAB, strAB, kStrT0, kStrT1, kA, kB, needB);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int tl = o >> 2, r = o & 3;
        const int t4 = f2i(c[0][tl][r]), t5 = f2i(c[1][tl][r]), t6 = f2i(c[2][tl][r]);
        const int t7 = f2i(c[3][tl][r]);
        lo[o] = ((long long)(t4 * 256 + t5) << 16) + (long long)(t6 * 256 + t7);
      }
    }
    // ---- Q_rj = (hi 2^32 + lo) 2^(e_r + f_j - 2114), rounded once, stored
    // straight from the fragment (8 consecutive rows per column segment)
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int tl = o >> 2, r = o & 3;
      if (tl == 1 && !needB) continue;
      const int row = i0 + (lane >> 2) + ((r >> 1) << 3);
      const int col = 8 * (tl ? tB : tA) + 2 * (lane & 3) + (r & 1);
      if (row >= nr || col >= n) continue;
      const double v = bad[row] ? __longlong_as_double(0x7FF8000000000000ll)
                                : fixed_to_double(hi[o], lo[o], 32, erow[row] + fcol[col] - 2114);
      a.Yout[(r0 + row) + (int64_t)col * a.ldyout] = v;
    }
  }
}

// ---- The same product with D T kept compact per 8-column tile (tile u keeps
// k < 16 (u / 2 + 1)), for a padded width NT in {32, 64, 128}: the CTA's
// 8 warps cover NT / 16 pairs of column tiles (u, NT / 8 - 1 - u, equal
// triangle work) times 128 / NT strips of 16 rows, so a tile has 2048 / NT
// rows.  NT = 128 needs 160 KB for the eight digits of D T (one CTA per SM).
__host__ __device__ constexpr int wide_ldt(int u) { return 16 * (u / 2 + 1) + 8; }  // bf16 stride, tile u
__host__ __device__ constexpr int wide_off(int u) {  // bf16 offset of tile u in a digit plane
  return u <= 0 ? 0 : wide_off(u - 1) + 8 * wide_ldt(u - 1);
}
template <int NT>
struct TiledCfg {
  static constexpr int ntiles = NT / 8, ncp = NT / 16, nib = 8 / ncp, tr = 16 * nib, kc = NT / 8;
  static constexpr int ldy = NT + 8;
  static constexpr int plane = wide_off(ntiles);  // bf16 per T digit plane
  static constexpr size_t smem = sizeof(uint16_t) * (size_t)kGmDigits * plane
                                 + sizeof(uint16_t) * (size_t)kGmDigits * tr * ldy
                                 + sizeof(int) * (size_t)(2 * NT + 2 * tr + 2 * 256);
  static constexpr int ctas = NT > 64 ? 1 : 2;
};

template <int NT>
__global__ void __launch_bounds__(kGmThreads, TiledCfg<NT>::ctas) ozgemm_tiled_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  using Cfg = TiledCfg<NT>;
  constexpr int TR = Cfg::tr, LDY = Cfg::ldy, PL = Cfg::plane;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t *planesT = (uint16_t *)smem;                          // [8][PL]
  uint16_t *planesY = planesT + (size_t)kGmDigits * PL;          // [8][TR rows][LDY]
  int *fcol = (int *)(planesY + (size_t)kGmDigits * TR * LDY);  // [NT]
  int *cs = fcol + NT;                                           // [NT] column scales
  int *erow = cs + NT;                                           // [TR]
  int *bad = erow + TR;                                          // [TR]
  int *epart = bad + TR;                                         // [KC][TR] partial row maxima
  int *bpart = epart + 256;                                      // [KC][TR] partial flags

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n = a.p;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  if (row0 >= row1) return;

  // ---- D T: column exponents, then 8 compact digit planes per column tile
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
  // items: (tile u, column c of the tile, k pair); tile u has 8 (u / 2 + 1)
  // k pairs per column, 64 (u / 2 + 1) items
  constexpr int items = 64 * (Cfg::ncp * (Cfg::ncp + 1));  // 64 * sum_u (u / 2 + 1)
  for (int e = t; e < items; e += kGmThreads) {
    int u = 0, rem = e;
    while (rem >= 64 * (u / 2 + 1)) {
      rem -= 64 * (u / 2 + 1);
      ++u;
    }
    const int kp = 8 * (u / 2 + 1);  // k pairs per column of tile u
    const int c = rem / kp, k = 2 * (rem % kp), j = 8 * u + c;
    unsigned long long b[2] = {0ull, 0ull};
    for (int h = 0; h < 2; ++h)
      if (j < n && k + h < n) b[h] = (unsigned long long)__double_as_longlong(a.Tinv[(k + h) + (int64_t)j * n]);
    const unsigned long long V0 = digits63(b[0], fcol[j], 0) + kBalance, V1 = digits63(b[1], fcol[j], 0) + kBalance;
    const float sg0 = (b[0] >> 63) ? -1.0f : 1.0f, sg1 = (b[1] >> 63) ? -1.0f : 1.0f;
    uint16_t *dst = planesT + wide_off(u) + c * wide_ldt(u) + k;
#pragma unroll
    for (int d = 0; d < kGmDigits; ++d) *(uint32_t *)(dst + (size_t)d * PL) = digit_pair_bf16(V0, V1, d, sg0, sg1);
  }

  // warp -> strip ib (16 rows) and column tiles tA = cp (k-steps kA),
  // tB = NT / 8 - 1 - cp (kB)
  const int cp = warp % Cfg::ncp, ib = warp / Cfg::ncp;
  const int i0 = 16 * ib, tA = cp, tB = Cfg::ntiles - 1 - cp;
  const bool needB = 8 * tB < n;
  const int kA = tA / 2 + 1;
  const int kB = min(tB / 2 + 1, (n + 15) / 16);
  const int mi = lane >> 3, rr = lane & 7;
  const uint32_t aY = smem_u32(planesY + (size_t)(i0 + (mi & 1) * 8 + rr) * LDY + (mi >> 1) * 8);
  const uint32_t bA = smem_u32(planesT + wide_off(tA) + rr * wide_ldt(tA) + (mi & 1) * 8);
  const uint32_t bB = smem_u32(planesT + wide_off(tB) + rr * wide_ldt(tB) + (mi & 1) * 8);
  const uint32_t bAB = (mi < 2) ? bA : bB;
  constexpr uint32_t kStrY = 2u * TR * LDY, kStrT = 2u * PL;
  // loader: thread (r, kc) holds 8 consecutive k of row r (lanes = rows)
  const int lr = t % TR, kc = t / TR, k0 = 8 * kc;

  for (int64_t r0 = row0; r0 < row1; r0 += TR) {
    const int nr = (int)min((int64_t)TR, row1 - r0);
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
    epart[kc * TR + lr] = mx;
    bpart[kc * TR + lr] = bd;
    __syncthreads();  // also: every warp is done with the previous tile's planes
    {
      int er = kNoExp, bb = 0;
#pragma unroll
      for (int q = 0; q < Cfg::kc; ++q) {
        er = max(er, epart[q * TR + lr]);
        bb |= bpart[q * TR + lr];
      }
      if (kc == 0) {
        erow[lr] = er;
        bad[lr] = bb;
      }
      unsigned long long V[8];
      float sg[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        V[h] = digits63(bv[h], er, cs[k0 + h]) + kBalance;
        sg[h] = (bv[h] >> 63) ? -1.0f : 1.0f;
      }
#pragma unroll
      for (int d = 0; d < kGmDigits; ++d) {
        uint4 w;
        w.x = digit_pair_bf16(V[0], V[1], d, sg[0], sg[1]);
        w.y = digit_pair_bf16(V[2], V[3], d, sg[2], sg[3]);
        w.z = digit_pair_bf16(V[4], V[5], d, sg[4], sg[5]);
        w.w = digit_pair_bf16(V[6], V[7], d, sg[6], sg[7]);
        *(uint4 *)(planesY + ((size_t)d * TR + lr) * LDY + k0) = w;
      }
    }
    __syncthreads();

    long long hi[8], lo[8];
    {
      float c[4][2][4];
      gm_orders<2, 5, 4>(c, aY, kStrY, bA, bB, bAB, kStrT, kStrT, kStrT, kA, kB, needB);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int tl = o >> 2, r = o & 3;
        const int t0 = f2i(c[0][tl][r]), t1 = f2i(c[1][tl][r]), t2 = f2i(c[2][tl][r]);
        const int t3 = f2i(c[3][tl][r]);
        hi[o] = ((long long)(t0 * 256 + t1) << 16) + (long long)(t2 * 256 + t3);
      }
    }
    {
      float c[4][2][4];
      gm_orders<6, 9, 8>(c, aY, kStrY, bA, bB, bAB, kStrT, kStrT, kStrT, kA, kB, needB);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int tl = o >> 2, r = o & 3;
        const int t4 = f2i(c[0][tl][r]), t5 = f2i(c[1][tl][r]), t6 = f2i(c[2][tl][r]);
        const int t7 = f2i(c[3][tl][r]);
        lo[o] = ((long long)(t4 * 256 + t5) << 16) + (long long)(t6 * 256 + t7);
      }
    }
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int tl = o >> 2, r = o & 3;
      if (tl == 1 && !needB) continue;
      const int row = i0 + (lane >> 2) + ((r >> 1) << 3);
      const int col = 8 * (tl ? tB : tA) + 2 * (lane & 3) + (r & 1);
      if (row >= nr || col >= n) continue;
      const double v = bad[row] ? __longlong_as_double(0x7FF8000000000000ll)
                                : fixed_to_double(hi[o], lo[o], 32, erow[row] + fcol[col] - 2114);
      a.Yout[(r0 + row) + (int64_t)col * a.ldyout] = v;
    }
  }
}

static cudaError_t launch_gm(const RowSweep &a, int grid, cudaStream_t s) {
  static KernelAttr attr;
  set_smem_attr(attr, ozgemm_kernel, (int)kGmSmem, true);
  ozgemm_kernel<<<grid, kGmThreads, kGmSmem, s>>>(a);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_gm_tiled(const RowSweep &a, int grid, cudaStream_t s) {
  static KernelAttr attr;
  set_smem_attr(attr, ozgemm_tiled_kernel<NT>, (int)TiledCfg<NT>::smem, true);
  ozgemm_tiled_kernel<NT><<<grid, kGmThreads, TiledCfg<NT>::smem, s>>>(a);
  return cudaGetLastError();
}

int ozgemm_tile_rows(int n, bool tc05) {
  if (tc05 && n >= kTcGemmMinN && n <= kGmNT) return tcgemm_tile_rows();
  return n > kGmNT ? TiledCfg<128>::tr : (n > 32 ? kGmTR : TiledCfg<32>::tr);
}

int ozgemm_grid(int64_t m, int n, bool tc05) {
  // the tcgen05 solve runs one CTA per SM
  if (tc05 && n >= kTcGemmMinN && n <= kGmNT) return tcgemm_grid(m);
  const int64_t tr = ozgemm_tile_rows(n, false);
  const int64_t tiles = (m + tr - 1) / tr;
  const int64_t per_sm = n > kGmNT ? TiledCfg<128>::ctas : 2;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, per_sm * (int64_t)num_sms()));
}

double ozgemm_tc_flops_per_row(int n, bool tc05) {
  if (tc05 && n >= kTcGemmMinN && n <= kGmNT) return tcgemm_tc_flops_per_row();
  int pairs = 0;
  for (int o = 0; o < kGmDigits; ++o) pairs += o + 1;  // orders 0..7, o + 1 pairs each
  // m16n8k16 products per row: 8-column tiles times their k extent
  double kcols = 0.0;
  if (n > kGmNT || n <= 32) {
    const int nt = n > kGmNT ? 128 : 32;
    for (int u = 0; u < nt / 8; ++u)
      if (8 * u < n) kcols += 8.0 * 16 * std::min(u / 2 + 1, (n + 15) / 16);
  } else {
    kcols = 32.0 * 32 + 32.0 * 64;  // one shape serves 33 <= n <= 64
  }
  return 2.0 * pairs * kcols;
}

// Q = Y T for kOzGemmMinN <= n <= 128 (a.Yin, a.Yout, a.Tinv, a.Tscale, a.m,
// a.p, a.rows_per_cta); narrower blocks use the FP64 substitution.
cudaError_t launch_ozgemm(const RowSweep &a, int grid, cudaStream_t s) {
  if (a.Tinv == nullptr || a.Tscale == nullptr) return cudaErrorInvalidValue;
  if (a.p < kOzGemmMinN || a.p > 128) return cudaErrorInvalidValue;
  if (tcgemm_usable(a)) return launch_tcgemm(a, grid, s);
  if (a.p <= 32) return launch_gm_tiled<32>(a, grid, s);
  if (a.p <= kGmNT) return launch_gm(a, grid, s);
  return launch_gm_tiled<128>(a, grid, s);
}

// ---- The same product for blocks wider than 128 columns (wide solve).
//
// D T no longer fits in shared memory, so the contraction runs in blocks of
// 64 k and the CTA's output is one 64-column block J of Q (k < 64 (J + 1):
// T is upper triangular).  Per pass, two small kernels prepare the operands:
//   * wide_tdigits_kernel: the column exponents f_j of D T and its eight
//     digit planes in global memory, Td[d][j][k] (k < npad = 64 nb, zero for
//     k > j and k >= n), read by every CTA of block J (L2-resident, 4 MB at
//     n = 512);
//   * wide_rowexp_kernel: each row's largest scaled exponent e_r over all n
//     columns (or kBadRow for a row with a NaN or Inf), so that a row has one
//     representation in every K block.
// The digits, orders, drains and the rounding are those of ozgemm_kernel;
// the two int64 words of an entry add up the K blocks exactly (each block
// adds less than 2^47 to either word).  A CTA owns whole rows (tiles of 32)
// and forms their 64-column output blocks one after another, so the product
// may run in place; 8 warps of 16 rows x 16 columns, T's digit block and the
// tile's digit planes in shared memory (110 KB: two CTAs per SM); the next K
// block's Y values are loaded into registers while the current one is
// multiplied.
namespace {

constexpr int kWsTR = 32;        // tile rows
constexpr int kWsJB = 64;        // output columns per CTA
constexpr int kWsKB = 64;        // contraction block
constexpr int kWsLd = kWsKB + 8; // bf16 stride of a digit-plane row (k contiguous)
constexpr int kBadRow = 1 << 29; // row exponent of a row with a NaN or Inf
constexpr size_t kWsSmem = sizeof(uint16_t) * (size_t)kGmDigits * kWsJB * kWsLd     // T digit block
                           + sizeof(uint16_t) * (size_t)kGmDigits * kWsTR * kWsLd   // Y tile digits
                           + sizeof(int) * (size_t)(kWsJB + kWsTR + CQR_MAX_N);

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

}  // namespace

struct WideSolve {
  int64_t m;
  int32_t n, npad;
  const double *Y;
  int64_t ldy;
  double *Q;
  int64_t ldq;
  const int *Tscale;    // n: c_k
  const uint16_t *Td;   // [8][n][npad] bf16 digits of D T
  const int *fcol;      // n: column exponents of D T
  const int *erow;      // m: row exponents (kBadRow: NaN row)
  int64_t rows_per_cta;
  const DevState *st;
};

// f_j and the digit planes of column j of D T (one CTA per column).
__global__ void __launch_bounds__(128) wide_tdigits_kernel(const double *Tinv, int n, int npad, uint16_t *Td,
                                                           int *fcol, const DevState *st) {
  if (st != nullptr && st->done) return;
  __shared__ int red[4];
  const int j = blockIdx.x, t = threadIdx.x;
  const double *col = Tinv + (int64_t)j * n;
  int mx = 1;
  for (int k = t; k <= j; k += 128) mx = max(mx, align_exp((unsigned long long)__double_as_longlong(col[k])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) red[t >> 5] = mx;
  __syncthreads();
  const int f = max(max(red[0], red[1]), max(red[2], red[3]));
  if (t == 0) fcol[j] = f;
  for (int k = 2 * t; k < npad; k += 256) {
    unsigned long long b[2] = {0ull, 0ull};
    for (int h = 0; h < 2; ++h)
      if (k + h <= j) b[h] = (unsigned long long)__double_as_longlong(col[k + h]);
    const unsigned long long V0 = digits63(b[0], f, 0) + kBalance, V1 = digits63(b[1], f, 0) + kBalance;
    const float sg0 = (b[0] >> 63) ? -1.0f : 1.0f, sg1 = (b[1] >> 63) ? -1.0f : 1.0f;
#pragma unroll
    for (int d = 0; d < kGmDigits; ++d)
      *(uint32_t *)(Td + ((size_t)d * n + j) * npad + k) = digit_pair_bf16(V0, V1, d, sg0, sg1);
  }
}

// e_r = max_k (exponent of y_rk - c_k) over the row (zeros ignored), or
// kBadRow when the row holds a NaN or Inf (one thread per row).
__global__ void __launch_bounds__(256) wide_rowexp_kernel(const double *Y, int64_t ldy, int64_t m, int n,
                                                          const int *Tscale, int *erow, const DevState *st) {
  if (st != nullptr && st->done) return;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  int mx = kNoExp;
  bool bad = false;
#pragma unroll 8
  for (int k = 0; k < n; ++k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(Y[r + (int64_t)k * ldy]);
    bad |= ((b >> 52) & 0x7FF) == 0x7FF;
    mx = max(mx, scaled_exp(b, __ldg(Tscale + k)));
  }
  erow[r] = bad ? kBadRow : mx;
}

// CTA x: rows [x rows_per_cta, ...) in tiles of 32; for each tile the
// output blocks J = nb - 1, ..., 0 in turn.  Block J reads columns
// k < 64 (J + 1) and writes columns 64 J .. 64 J + 63, so with Q == Y (in
// place) no later block of the tile reads what an earlier one wrote.
__global__ void __launch_bounds__(kGmThreads, 2) ozwsolve_kernel(WideSolve a) {
  if (a.st != nullptr && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t *planesT = (uint16_t *)smem;                                   // [8][64 j][kWsLd]
  uint16_t *planesY = planesT + (size_t)kGmDigits * kWsJB * kWsLd;        // [8][32 rows][kWsLd]
  int *fc = (int *)(planesY + (size_t)kGmDigits * kWsTR * kWsLd);         // [64]
  int *er = fc + kWsJB;                                                   // [32]
  int *cs = er + kWsTR;                                                   // [n]

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n = a.n, nb = a.npad / kWsKB;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  if (row0 >= row1) return;
  for (int k = t; k < n; k += kGmThreads) cs[k] = a.Tscale[k];

  // warp -> rows 16 ib .. + 15, columns 16 cg .. + 15 (two 8-column tiles)
  const int ib = warp & 1, cg = warp >> 1, i0 = 16 * ib;
  const int mi = lane >> 3, rr = lane & 7;
  const uint32_t aY = smem_u32(planesY + (size_t)(i0 + (mi & 1) * 8 + rr) * kWsLd + (mi >> 1) * 8);
  const uint32_t bT = smem_u32(planesT + (size_t)(16 * cg + (mi >> 1) * 8 + rr) * kWsLd + (mi & 1) * 8);
  constexpr uint32_t kStrY = 2u * kWsTR * kWsLd, kStrT = 2u * kWsJB * kWsLd;
  // loader: thread (lr, kc) holds k = 8 kc .. 8 kc + 7 of row lr of a K block
  const int lr = t & (kWsTR - 1), kc = t >> 5;

  for (int64_t r0 = row0; r0 < row1; r0 += kWsTR) {
    const int nr = (int)min((int64_t)kWsTR, row1 - r0);
    const int e_r = (lr < nr) ? a.erow[r0 + lr] : kNoExp;
    auto load_y = [&](int kb, unsigned long long (&bv)[8]) {
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const int k = kWsKB * kb + 8 * kc + h;
        bv[h] = (lr < nr && k < n) ? (unsigned long long)__double_as_longlong(a.Y[(r0 + lr) + (int64_t)k * a.ldy])
                                   : 0ull;
      }
    };
    for (int J = nb - 1; J >= 0; --J) {
      const int j0 = kWsJB * J;
      unsigned long long bv[8];
      load_y(0, bv);
      long long hi[8], lo[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) hi[o] = lo[o] = 0;
      for (int kb = 0; kb <= J; ++kb) {
        __syncthreads();  // every warp is done with the previous planes (and fc, er)
        if (kb == 0) {
          if (t < kWsJB) fc[t] = (j0 + t < n) ? a.fcol[j0 + t] : 0;
          if (kc == 0 && J == nb - 1) er[lr] = e_r;
        }
        // T's digit block (kb, J): 8 planes x 64 columns x 64 k, zero past n
        for (int e = t; e < kGmDigits * kWsJB * (kWsKB / 8); e += kGmThreads) {
          const int c8 = e & 7, jj = (e >> 3) & (kWsJB - 1), d = e >> 9;
          const bool live = j0 + jj < n;
          const uint16_t *src = live ? a.Td + ((size_t)d * n + j0 + jj) * a.npad + kWsKB * kb + 8 * c8 : a.Td;
          cp_async16(planesT + ((size_t)d * kWsJB + jj) * kWsLd + 8 * c8, src, live ? 16 : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        // the tile's digits of this block
        {
          unsigned long long V[8];
          float sg[8];
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const int k = kWsKB * kb + 8 * kc + h;
            V[h] = digits63(bv[h], e_r, k < n ? cs[k] : 0) + kBalance;
            sg[h] = (bv[h] >> 63) ? -1.0f : 1.0f;
          }
#pragma unroll
          for (int d = 0; d < kGmDigits; ++d) {
            uint4 w;
            w.x = digit_pair_bf16(V[0], V[1], d, sg[0], sg[1]);
            w.y = digit_pair_bf16(V[2], V[3], d, sg[2], sg[3]);
            w.z = digit_pair_bf16(V[4], V[5], d, sg[4], sg[5]);
            w.w = digit_pair_bf16(V[6], V[7], d, sg[6], sg[7]);
            *(uint4 *)(planesY + ((size_t)d * kWsTR + lr) * kWsLd + 8 * kc) = w;
          }
        }
        if (kb < J) load_y(kb + 1, bv);  // in flight during the products
        cp_async_wait_all();
        __syncthreads();
        // orders 0..3 into hi, orders 4..7 into lo (exact: below 2^24 per block)
        {
          float c[4][2][4];
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int tl = 0; tl < 2; ++tl) c[d][tl][0] = c[d][tl][1] = c[d][tl][2] = c[d][tl][3] = 0.0f;
          gm_steps<2, 5, 4, 0>(c, aY, kStrY, bT, kStrT, 0, kWsKB / 16);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            const int tl = o >> 2, r = o & 3;
            const int t0 = f2i(c[0][tl][r]), t1 = f2i(c[1][tl][r]), t2 = f2i(c[2][tl][r]);
            const int t3 = f2i(c[3][tl][r]);
            hi[o] += ((long long)(t0 * 256 + t1) << 16) + (long long)(t2 * 256 + t3);
          }
        }
        {
          float c[4][2][4];
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int tl = 0; tl < 2; ++tl) c[d][tl][0] = c[d][tl][1] = c[d][tl][2] = c[d][tl][3] = 0.0f;
          gm_steps<6, 9, 8, 0>(c, aY, kStrY, bT, kStrT, 0, kWsKB / 16);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            const int tl = o >> 2, r = o & 3;
            const int t4 = f2i(c[0][tl][r]), t5 = f2i(c[1][tl][r]), t6 = f2i(c[2][tl][r]);
            const int t7 = f2i(c[3][tl][r]);
            lo[o] += ((long long)(t4 * 256 + t5) << 16) + (long long)(t6 * 256 + t7);
          }
        }
      }
      // ---- Q_rj = (hi 2^32 + lo) 2^(e_r + f_j - 2114), rounded once
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int tl = o >> 2, r = o & 3;
        const int row = i0 + (lane >> 2) + ((r >> 1) << 3);
        const int jj = 16 * cg + 8 * tl + 2 * (lane & 3) + (r & 1);
        if (row >= nr || j0 + jj >= n) continue;
        const int e = er[row];
        const double v = (e == kBadRow) ? __longlong_as_double(0x7FF8000000000000ll)
                                        : fixed_to_double(hi[o], lo[o], 32, e + fc[jj] - 2114);
        a.Q[(r0 + row) + (int64_t)(j0 + jj) * a.ldq] = v;
      }
    }
  }
}

int wide_solve_npad(int n) { return ((n + kWsKB - 1) / kWsKB) * kWsKB; }

size_t wide_solve_scratch_bytes(int64_t m, int n) {
  return sizeof(uint16_t) * (size_t)kGmDigits * n * wide_solve_npad(n) + sizeof(int) * (size_t)n +
         sizeof(int) * (size_t)m + 1024;
}

// Q = Y T for 128 < n <= CQR_MAX_N (a.Yin, a.Yout, a.Tinv, a.Tscale, a.m,
// a.p, a.st); `scratch` holds wide_solve_scratch_bytes(m, n) bytes.
cudaError_t launch_wide_solve(const RowSweep &a, void *scratch, cudaStream_t s) {
  const int n = a.p;
  if (a.Tinv == nullptr || a.Tscale == nullptr || scratch == nullptr) return cudaErrorInvalidValue;
  if (n <= kOzGemmMaxN || n > CQR_MAX_N) return cudaErrorInvalidValue;
  const int npad = wide_solve_npad(n);
  char *p0 = (char *)scratch;
  uint16_t *Td = (uint16_t *)p0;
  p0 += ((sizeof(uint16_t) * (size_t)kGmDigits * n * npad + 255) & ~(size_t)255);
  int *fcol = (int *)p0;
  p0 += ((sizeof(int) * (size_t)n + 255) & ~(size_t)255);
  int *erow = (int *)p0;
  wide_tdigits_kernel<<<n, 128, 0, s>>>(a.Tinv, n, npad, Td, fcol, a.st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wide_rowexp_kernel<<<(unsigned)((a.m + 255) / 256), 256, 0, s>>>(a.Yin, a.ldyin, a.m, n, a.Tscale, erow, a.st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WideSolve w;
  w.m = a.m;
  w.n = n;
  w.npad = npad;
  w.Y = a.Yin;
  w.ldy = a.ldyin;
  w.Q = a.Yout;
  w.ldq = a.ldyout;
  w.Tscale = a.Tscale;
  w.Td = Td;
  w.fcol = fcol;
  w.erow = erow;
  // two CTAs per SM, each with the same number of tiles (every tile does
  // the same work)
  const int64_t tiles = (a.m + kWsTR - 1) / kWsTR;
  const int64_t G = std::max<int64_t>(1, std::min<int64_t>(tiles, 2 * (int64_t)num_sms()));
  w.rows_per_cta = ((tiles + G - 1) / G) * kWsTR;
  w.st = a.st;
  static KernelAttr attr;
  set_smem_attr(attr, ozwsolve_kernel, (int)kWsSmem, true);
  const int64_t gx = (a.m + w.rows_per_cta - 1) / w.rows_per_cta;
  ozwsolve_kernel<<<(unsigned)gx, kGmThreads, kWsSmem, s>>>(w);
  return cudaGetLastError();
}

// ---- Gramian of a block wider than 128 columns (wide Gramian).
//
// X = Y^T Y by 64 x 64 block pairs (I, J), I <= J, on the tensor cores with
// the digits of the solve above.  Every column is written against its
// largest biased exponent over all m rows, E_c (wide_colexp_kernel; a NaN
// or Inf makes it 2047), as y_rc = sign V 2^(E_c - 1085) with V < 2^63 in 8
// balanced base-256 digits, so no CTA rescales as it goes.  CTA (g, w) takes
// the rows of row group g in tiles of 64 and block pair w: the tile's 64
// columns of block I and of block J become digit planes with the rows
// contiguous (block I alone when I = J), the products of each digit order
// <= 7 (36 pairs) are summed exactly in FP32 over the tile (below 2^23) and
// added into two int64 words per entry (each tile adds less than 2^47; a
// group has at most 2^20 rows, so the words stay below 2^61), and the
// group's partial is rounded to FP64 once:
//   X_ij = (hi 2^32 + lo) 2^(E_i + E_j - 2114).
// The dropped orders change an entry by at most about m 2^-60 max|y_i|
// max|y_j|.  The groups' partials are summed in a fixed order into the upper
// triangle and mirrored, so X is symmetric bit for bit.  16 warps of 16 x 16
// outputs, both blocks' digit planes in shared memory (144 KB, one CTA per
// SM); the next tile's values are loaded while the current one is
// multiplied.
namespace {

constexpr int kWgTR = 64;                   // tile rows (the contraction block)
constexpr int kWgB = 64;                    // columns of a block
constexpr int kWgLd = kWgTR + 8;            // bf16 stride of a digit-plane column (rows contiguous)
constexpr int kWgThreads = 512;             // 16 warps: 4 x 4 output tiles of 16 x 16
constexpr int64_t kWgMaxRows = 1 << 20;     // rows of one group
constexpr int kWgEcolPad = 256;             // doubles reserved ahead of the partials (E_c, 2 KB)
constexpr int kBadExp = 0x7FF;              // E_c of a column holding a NaN or Inf
constexpr size_t kWgSmem = 2 * sizeof(uint16_t) * (size_t)kGmDigits * kWgB * kWgLd + sizeof(int) * 2 * kWgB;

}  // namespace

struct WideGram {
  int64_t m;
  int32_t n, npairs;
  const double *Y;
  int64_t ldy;
  const int *Ecol;      // npad: largest biased exponent of each column (>= 1)
  double *partials;     // [G][npairs][64 x 64]
  int64_t rows_per_cta;
  const DevState *st;
};

// E_c = max over the rows of column c of its biased exponent (zeros and
// subnormals count as 1, NaN and Inf as 2047): CTA (s, c) takes a slice of
// rows, combined by atomicMax into a zeroed E.
__global__ void __launch_bounds__(256) wide_colexp_kernel(const double *Y, int64_t ldy, int64_t m,
                                                          int64_t rows_per_cta, int *Ecol, const DevState *st) {
  if (st != nullptr && st->done) return;
  __shared__ int red[8];
  const int c = blockIdx.y, t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta, r1 = min(m, r0 + rows_per_cta);
  const unsigned long long *col = (const unsigned long long *)(Y + (int64_t)c * ldy);
  int mx = 1;
  int64_t r = r0 + t;
  for (; r + 3 * 256 < r1; r += 4 * 256) {
    unsigned long long v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = __ldg(col + r + u * 256);
#pragma unroll
    for (int u = 0; u < 4; ++u) mx = max(mx, align_exp(v[u]));
  }
  for (; r < r1; r += 256) mx = max(mx, align_exp(__ldg(col + r)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) red[t >> 5] = mx;
  __syncthreads();
  if (t == 0) {
    int b = red[0];
    for (int w = 1; w < 8; ++w) b = max(b, red[w]);
    atomicMax(Ecol + c, b);
  }
}

__global__ void __launch_bounds__(kWgThreads, 1) ozwgram_kernel(WideGram a) {
  if (a.st != nullptr && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t *planesA = (uint16_t *)smem;                                // [8][64 columns of I][kWgLd]
  uint16_t *planesB = planesA + (size_t)kGmDigits * kWgB * kWgLd;      // [8][64 columns of J][kWgLd]
  int *eI = (int *)(planesB + (size_t)kGmDigits * kWgB * kWgLd);      // [64]
  int *eJ = eI + kWgB;                                                // [64]

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int w = blockIdx.y;
  int J = 0;
  while ((J + 1) * (J + 2) / 2 <= w) ++J;
  const int I = w - J * (J + 1) / 2;  // block pair (I, J), I <= J
  const bool diag = I == J;
  const int ci = kWgB * I, cj = kWgB * J, n = a.n;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  if (t < kWgB) {
    eI[t] = a.Ecol[ci + t];
    eJ[t] = a.Ecol[cj + t];
  }
  // warp -> outputs (columns of I) 16 wi .. + 15 x (columns of J) 16 wj .. + 15
  const int wi = warp & 3, wj = warp >> 2;
  const int mi = lane >> 3, rr = lane & 7;
  const uint32_t aA = smem_u32(planesA + (size_t)(16 * wi + (mi & 1) * 8 + rr) * kWgLd + (mi >> 1) * 8);
  const uint16_t *pB = diag ? planesA : planesB;
  const uint32_t bB = smem_u32(pB + (size_t)(16 * wj + (mi >> 1) * 8 + rr) * kWgLd + (mi & 1) * 8);
  constexpr uint32_t kStr = 2u * kWgB * kWgLd;
  // loader: thread t holds rows 8 (t & 7) .. + 7 of column t >> 3 of each block
  const int lc = t >> 3, lr = 8 * (t & 7);
  const bool liveI = ci + lc < n, liveJ = !diag && cj + lc < n;
  __syncthreads();
  const int eIc = eI[lc], eJc = eJ[lc];

  auto load = [&](int64_t r0, unsigned long long (&va)[8], unsigned long long (&vb)[8]) {
    const int nr = (int)min((int64_t)kWgTR, row1 - r0);
    const double *yi = a.Y + r0 + (int64_t)(ci + lc) * a.ldy, *yj = a.Y + r0 + (int64_t)(cj + lc) * a.ldy;
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const bool in = lr + h < nr;
      va[h] = (in && liveI) ? (unsigned long long)__double_as_longlong(yi[lr + h]) : 0ull;
      vb[h] = (in && liveJ) ? (unsigned long long)__double_as_longlong(yj[lr + h]) : 0ull;
    }
  };
  auto split = [&](const unsigned long long (&v)[8], int e, uint16_t *planes) {
    unsigned long long V[8];
    float sg[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      V[h] = digits63(v[h], e, 0) + kBalance;
      sg[h] = (v[h] >> 63) ? -1.0f : 1.0f;
    }
#pragma unroll
    for (int d = 0; d < kGmDigits; ++d) {
      uint4 q;
      q.x = digit_pair_bf16(V[0], V[1], d, sg[0], sg[1]);
      q.y = digit_pair_bf16(V[2], V[3], d, sg[2], sg[3]);
      q.z = digit_pair_bf16(V[4], V[5], d, sg[4], sg[5]);
      q.w = digit_pair_bf16(V[6], V[7], d, sg[6], sg[7]);
      *(uint4 *)(planes + ((size_t)d * kWgB + lc) * kWgLd + lr) = q;
    }
  };

  long long hi[8], lo[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) hi[o] = lo[o] = 0;
  unsigned long long va[8], vb[8];
  if (row0 < row1) load(row0, va, vb);
  for (int64_t r0 = row0; r0 < row1; r0 += kWgTR) {
    __syncthreads();  // every warp is done with the previous tile's planes
    split(va, eIc, planesA);
    if (!diag) split(vb, eJc, planesB);
    if (r0 + kWgTR < row1) load(r0 + kWgTR, va, vb);  // in flight during the products
    __syncthreads();
    {
      float c[4][2][4];
#pragma unroll
      for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int tl = 0; tl < 2; ++tl) c[d][tl][0] = c[d][tl][1] = c[d][tl][2] = c[d][tl][3] = 0.0f;
      gm_steps<2, 5, 4, 0>(c, aA, kStr, bB, kStr, 0, kWgTR / 16);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int tl = o >> 2, r = o & 3;
        const int t0 = f2i(c[0][tl][r]), t1 = f2i(c[1][tl][r]), t2 = f2i(c[2][tl][r]);
        const int t3 = f2i(c[3][tl][r]);
        hi[o] += ((long long)(t0 * 256 + t1) << 16) + (long long)(t2 * 256 + t3);
      }
    }
    {
      float c[4][2][4];
#pragma unroll
      for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int tl = 0; tl < 2; ++tl) c[d][tl][0] = c[d][tl][1] = c[d][tl][2] = c[d][tl][3] = 0.0f;
      gm_steps<6, 9, 8, 0>(c, aA, kStr, bB, kStr, 0, kWgTR / 16);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int tl = o >> 2, r = o & 3;
        const int t4 = f2i(c[0][tl][r]), t5 = f2i(c[1][tl][r]), t6 = f2i(c[2][tl][r]);
        const int t7 = f2i(c[3][tl][r]);
        lo[o] += ((long long)(t4 * 256 + t5) << 16) + (long long)(t6 * 256 + t7);
      }
    }
  }
  // this group's partial of X_IJ, rounded once
  double *P = a.partials + ((int64_t)blockIdx.x * a.npairs + w) * (kWgB * kWgB);
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int tl = o >> 2, r = o & 3;
    const int il = 16 * wi + (lane >> 2) + ((r >> 1) << 3);
    const int jl = 16 * wj + 8 * tl + 2 * (lane & 3) + (r & 1);
    const bool bad = eI[il] == kBadExp || eJ[jl] == kBadExp;
    P[il + kWgB * jl] = bad ? __longlong_as_double(0x7FF8000000000000ll)
                            : fixed_to_double(hi[o], lo[o], 32, eI[il] + eJ[jl] - 2114);
  }
}

// X_ij = X_ji = sum over the groups of their partials, in group order, for
// i <= j < n (one thread per entry of a block pair).
__global__ void __launch_bounds__(256) reduce_wide_pairs_kernel(const double *partials, int G, int npairs, int n,
                                                                double *X, int64_t ldx, const DevState *st) {
  if (st != nullptr && st->done) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)npairs * kWgB * kWgB) return;
  const int w = (int)(e / (kWgB * kWgB)), l = (int)(e % (kWgB * kWgB));
  int J = 0;
  while ((J + 1) * (J + 2) / 2 <= w) ++J;
  const int I = w - J * (J + 1) / 2;
  const int i = kWgB * I + l % kWgB, j = kWgB * J + l / kWgB;
  if (i > j || j >= n) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += partials[((int64_t)g * npairs + w) * (kWgB * kWgB) + l];
  X[i + (int64_t)j * ldx] = s;
  X[j + (int64_t)i * ldx] = s;
}

static int wide_gram_groups(int64_t m, int npairs) {
  const int64_t tiles = std::max<int64_t>(1, (m + kWgTR - 1) / kWgTR);
  int64_t G = std::max<int64_t>(1, num_sms() / npairs);  // about one CTA per SM
  G = std::max<int64_t>(G, (m + kWgMaxRows - 1) / kWgMaxRows);
  return (int)std::min<int64_t>(G, tiles);
}

int64_t wide_gram_partial_elems(int64_t m, int p) {
  const int nb = (p + kWgB - 1) / kWgB, npairs = nb * (nb + 1) / 2;
  return kWgEcolPad + (int64_t)wide_gram_groups(m, npairs) * npairs * (kWgB * kWgB);
}

cudaError_t launch_wide_gram(const double *Y, int64_t ldy, int64_t m, int p, double *partials, double *X,
                             int64_t ldx, const DevState *st, cudaStream_t s, int *launches) {
  if (p <= kOzGemmMaxN || p > CQR_MAX_N || m < 1) return cudaErrorInvalidValue;
  const int nb = (p + kWgB - 1) / kWgB, npairs = nb * (nb + 1) / 2;
  int *Ecol = (int *)partials;  // nb 64 <= 512 ints in the reserved 2 KB
  double *P = partials + kWgEcolPad;
  cudaError_t e = cudaMemsetAsync(Ecol, 0, sizeof(int) * (size_t)nb * kWgB, s);
  if (e != cudaSuccess) return e;
  const int64_t slices = std::max<int64_t>(1, std::min<int64_t>((m + 4095) / 4096, 64));
  const int64_t rpc = (m + slices - 1) / slices;
  wide_colexp_kernel<<<dim3((unsigned)slices, (unsigned)p), 256, 0, s>>>(Y, ldy, m, rpc, Ecol, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WideGram w;
  w.m = m;
  w.n = p;
  w.npairs = npairs;
  w.Y = Y;
  w.ldy = ldy;
  w.Ecol = Ecol;
  w.partials = P;
  const int G = wide_gram_groups(m, npairs);
  const int64_t tiles = (m + kWgTR - 1) / kWgTR;
  w.rows_per_cta = ((tiles + G - 1) / G) * kWgTR;
  w.st = st;
  static KernelAttr attr;
  set_smem_attr(attr, ozwgram_kernel, (int)kWgSmem, true);
  const int gx = (int)((m + w.rows_per_cta - 1) / w.rows_per_cta);
  ozwgram_kernel<<<dim3((unsigned)gx, (unsigned)npairs), kWgThreads, kWgSmem, s>>>(w);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t E = (int64_t)npairs * kWgB * kWgB;
  reduce_wide_pairs_kernel<<<(unsigned)((E + 255) / 256), 256, 0, s>>>(P, gx, npairs, p, X, ldx, st);
  e = cudaGetLastError();
  if (launches != nullptr) *launches += 3;
  return e;
}

}  // namespace cqr
