// Gramian sweep on the tensor cores with exact digit arithmetic (the Ozaki
// splitting scheme: Ozaki, Ogita, Oishi, Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), for the FP64 Gramian
// X = Y^T Y of Alg. 1.
//
// Why: GB300 retires ~1.6 FP64 FMAs per SM per clock but ~570 dense bf16
// TFLOP/s through mma.sync, so the Gramian is computed from bf16 "digits"
// whose products the tensor cores form and add exactly.
//
// Representation (per 64-row tile, per column j):
//   E_j = running maximum of the biased exponent of column j over the rows
//   this CTA has seen; every element is written as
//     x = sign * V * 2^(E_j - 1078),   V < 2^56 (56 bits relative to the
//     column maximum, truncated),
//   V in 7 balanced base-256 digits, V = sum_{i=0..6} D_i 2^(8 (6 - i)),
//   D_0 in [0, 256], D_i in [-128, 127] for i >= 1 (128 added to each of
//   the six low bytes, bytes read back minus 128); a digit with its sign,
//   and twice it, is an integer exact in bf16.
// Products: x_i x_j = 2^(E_i + E_j - 2156) sum_{s,t} D_s(i) D_t(j) 2^(8 (12 - s - t)).
//   Orders o = s + t <= 6 are kept (the rest lies below 2^-53 of the leading
//   term).  Using P_st^T = P_ts, only s <= t is formed; the CTA stores
//   P = sum_o (B_o + C_o / 2) w_o with B_o = sum_{s<t, s+t=o} P_st and
//   C_o = P_{o/2,o/2}, and the reduction returns X = P + P^T.
// Exactness: each order o has one FP32 mma.sync accumulator holding
//   T_o = 2 B_o + C_o over a 64-row tile (the off-diagonal pairs enter with
//   their A digits doubled, exact in bf16); |T_o| <= 9 * 2^20 < 2^24 (the
//   top digit pairs with at most 2^8 * 2^7 per term, the others with 2^14),
//   so the FP32 sums are exact and the FP32 -> int conversion is exact.
//   Orders (0, 1), (2, 3), (4, 5) are combined exactly in int32
//   (T_o 2^8 + T_o+1 < 2^31) and added into two int64 words per entry
//   (orders 0..3 and 4..6), summed over the CTA's tiles (rescaled by right
//   shifts when a column's running exponent grows), and rounded to FP64
//   once per CTA.
// Non-finite inputs make every partial of the CTA NaN (the control kernel
// then reports a breakdown, as the FP64 path does).
#include <algorithm>

#include "cqr_internal.cuh"
#include "ozdigits.cuh"

namespace cqr {

using namespace oz;

namespace {

constexpr int kOzTR = 64;            // tile rows (one exact accumulation window)
constexpr int kOzLDK = kOzTR + 8;    // bf16 stride of a digit-plane column
// Launch shape per width: n <= 64: 8 warps, two CTAs per SM (they hide each
// other's latency), one CTA per row group.  n in (64, 128]: two CTAs per row
// group, each forming one 64-row half of P with 16 warps, one CTA per SM.
template <int NT>
struct OzCfg {
  static constexpr int halves = (NT > 64) ? 2 : 1;   // CTAs per row group
  static constexpr int PR = NT / halves;             // rows of P per CTA
  static constexpr int threads = (NT > 64) ? 512 : 256;
  static constexpr int warps = threads / 32;
  static constexpr int ctas = (NT > 64) ? 1 : 2;     // CTAs per SM
};
constexpr int kOzDigits = 7;   // balanced base-256 digits of 56 bits (planes allocated for all 7)

// Orders 0..6 split into `groups` groups ({0, 6}, {1, 5}, {2, 4}, {3} for
// four groups): does group grp own order o?
__device__ __forceinline__ bool order_in_group(int groups, int grp, int o) {
  return groups == 1 || o == grp || o == 6 - grp;
}
constexpr int kOzMaxOrder = 6;
constexpr unsigned long long kOzBalance = 0x0000808080808080ull;
// Balanced digit i (0..6) of W = V + kOzBalance with sign s: byte 6 - i of W
// minus 128 for i >= 1, placed in an FP32 2^23 + x by one byte permute and
// signed in one FMA (exact); digit 0 is W >> 48 (up to 256: the carry out
// of the six low bytes can reach bit 56).
__device__ __forceinline__ float oz_digit(unsigned long long W, int i, float s) {
  if (i == 0) return fmaf(__int_as_float(0x4B000000 | (int)(W >> 48)), s, -s * 8388608.0f);
  const int b = 6 - i;
  const uint32_t word = (b >= 4) ? (uint32_t)(W >> 32) : (uint32_t)W;
  const float x = __int_as_float((int)__byte_perm(word, 0x4B000000u, 0x7440u | (uint32_t)(b & 3)));
  return fmaf(x, s, -s * 8388736.0f);
}

}  // namespace

struct OzGeom {
  int NI, NJ, JB, groups, units;
};

// Work units of one CTA (PR rows of P by NT columns): strips of 16 rows x JB
// columns, times groups of orders.  NT = 16, 32, 64, 128 give 4, 8, 8 and 16
// units (one per warp).
__host__ __device__ constexpr OzGeom oz_geom(int NT, int PR) {
  return OzGeom{PR / 16, NT / ((NT >= 32) ? 32 : 16), (NT >= 32) ? 32 : 16,
                (PR / 16) * (NT / ((NT >= 32) ? 32 : 16)) >= 8 ? 1 : 4,
                (PR / 16) * (NT / ((NT >= 32) ? 32 : 16)) *
                    ((PR / 16) * (NT / ((NT >= 32) ? 32 : 16)) >= 8 ? 1 : 4)};
}

// One CTA: rows [g * rows_per_cta, ...) of row group g in tiles of 64;
// optional FP64 row solve (Alg. 1, n <= 64) before the Gramian of the
// tile.  Writes rows [h PR, (h+1) PR) of the group's partial P (n x n, ld n)
// to partials[g * n * n], h = the CTA's half.
//
// ND = 7 is the exact FP64 Gramian described above.  ND = 5 (the first pass
// of the mixed-precision variant) keeps the leading 5 balanced digits of
// each element and the orders o <= 4 (9 of the 16 symmetric digit pairs):
// with U_j = 2^(E_j - 1078) and Ubar_j = 2^56 U_j (> |y_rj|), the dropped
// digits are at most 128 (2^8 + 1) U_j < 2^15.006 U_j per element (plus
// < U_j from the truncation to 56 bits) and the dropped orders 5..8 of a
// row's product at most (4 2^70 + 3 2^62 + ...) U_i U_j < 2^72.005 U_i U_j,
// so each row adds less than 2^73.01 U_i U_j = 2^-38.99 Ubar_i Ubar_j of
// error to X_ij (the floor rescalings add < 2^-65 Ubar_i Ubar_j per tile).
// With `emax` set the CTA records its final column exponents there
// (atomicMax), for the shift that covers this error.
template <int NT, int ND>
__global__ void __launch_bounds__(OzCfg<NT>::threads, OzCfg<NT>::ctas) ozgram_kernel(RowSweep a) {
  static_assert(ND == 7 || ND == 5, "digit counts of the Gramian");
  constexpr int kMaxOrder = ND - 1;
  if (a.st != nullptr && a.st->done) return;
  constexpr int JB = (NT >= 32) ? 32 : 16;
  constexpr int NTILE = JB / 8;               // n8 tiles per unit
  constexpr int SLOTS = 4 * NTILE;            // int64 accumulator slots per lane (one unit)
  extern __shared__ __align__(16) unsigned char smem[];
  double *tile = (double *)smem;                                   // [NT][kOzTR] column-major
  uint16_t *planes = (uint16_t *)(smem + sizeof(double) * NT * kOzTR);  // [8][NT][kOzLDK]
  int *Erun = (int *)(planes + (size_t)kOzDigits * NT * kOzLDK);        // [NT]
  int *Edel = Erun + NT;                                                // [NT]
  int *flag = Edel + NT;                                                // [1]

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n = a.p;
  constexpr int kOzThreads = OzCfg<NT>::threads, kOzWarps = OzCfg<NT>::warps, PR = OzCfg<NT>::PR;
  constexpr OzGeom gg = oz_geom(NT, PR);
  const int half = (int)(blockIdx.x % OzCfg<NT>::halves);
  const int64_t grp_id = blockIdx.x / OzCfg<NT>::halves;
  const int64_t row0 = grp_id * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);

  for (int j = t; j < NT; j += kOzThreads) {
    Erun[j] = 1;
    Edel[j] = 0;
  }
  if (t == 0) *flag = 0;

  long long acc_hi[SLOTS], acc_lo[SLOTS];
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    acc_hi[k] = 0;
    acc_lo[k] = 0;
  }
  __syncthreads();

  for (int64_t r0 = row0; r0 < row1; r0 += kOzTR) {
    const int nr = (int)min((int64_t)kOzTR, row1 - r0);
    // ---- stage the tile (column-major, zero padded): every copy of the
    // tile is in flight at once
    for (int e = t; e < kOzTR * NT; e += kOzThreads) {
      const int i = e % kOzTR, j = e / kOzTR;
      const bool in = (i < nr) && (j < n);
      const double *src = in ? a.Yin + (r0 + i) + (int64_t)j * a.ldyin : a.Yin;
      cp_async8(tile + j * kOzTR + i, src, in ? 8 : 0);
    }
    cp_async_wait_all();
    __syncthreads();
    // ---- optional FP64 row solve, then write the rows out
    if (NT <= 64 && a.do_trsm) {
      // forward substitution, 4 threads per row (64 rows x 4 = 256): thread
      // sub of a row sums q_k R_kj over k = sub (mod 4); the four partial
      // sums are combined as (s0 + s1) + (s2 + s3)
      const int row = t >> 2, sub = t & 3;
      for (int j = 0; j < n; ++j) {
        double part = 0.0;
        for (int k = sub; k < j; k += 4) part = fma(tile[k * kOzTR + row], a.Rt[k + (int64_t)j * n], part);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        if (sub == 0 && row < nr) tile[j * kOzTR + row] = (tile[j * kOzTR + row] - part) * a.Rdinv[j];
        __syncwarp();
      }
      __syncthreads();
      for (int e = t; e < nr * n; e += kOzThreads) {
        const int i = e % nr, j = e / nr;
        a.Yout[(r0 + i) + (int64_t)j * a.ldyout] = tile[j * kOzTR + i];
      }
    }
    // ---- column exponents: running maximum, growth since the last tile
    for (int j = warp; j < NT; j += kOzWarps) {
      // biased exponents from the high words; 0x7FF (NaN / Inf) is the
      // largest, so it also flags a non-finite entry
      const uint32_t *hw = (const uint32_t *)(tile + j * kOzTR) + 1;
      int mx = 1;
      for (int i = lane; i < kOzTR; i += 32) mx = max(mx, (int)((hw[2 * i] >> 20) & 0x7FF));
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) {
        const int old = Erun[j];
        const int nw = max(old, mx);
        Edel[j] = nw - old;
        Erun[j] = nw;
        if (mx == 0x7FF) *flag = 1;
      }
    }
    __syncthreads();
    // ---- slice into ND digit planes (two rows per thread step)
    for (int e = t; e < (kOzTR / 2) * NT; e += kOzThreads) {
      const int i = 2 * (e % (kOzTR / 2)), j = e / (kOzTR / 2);
      const int Ej = Erun[j];
      unsigned long long V[2];
      float sg[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(tile[j * kOzTR + i + h]);
        const int ef = (int)((b >> 52) & 0x7FF);
        unsigned long long M = b & 0xFFFFFFFFFFFFFull;
        if (ef) M |= 0x10000000000000ull;
        if (ef == 0x7FF) M = 0;
        const int sh = Ej - (ef ? ef : 1);
        V[h] = ((sh >= 56) ? 0ull : ((M << 3) >> sh)) + kOzBalance;
        sg[h] = (b >> 63) ? -1.0f : 1.0f;
      }
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        // two signed digits -> exact FP32 -> one packed bf16x2
        const __nv_bfloat162 pr = __floats2bfloat162_rn(oz_digit(V[0], d, sg[0]), oz_digit(V[1], d, sg[1]));
        *(uint32_t *)(planes + ((size_t)d * NT + j) * kOzLDK + i) = *(const uint32_t *)&pr;
      }
    }
    __syncthreads();
    // ---- tensor-core products, drained into the int64 accumulators
    {
      const int u = warp;
      if (u < gg.units) {
      const int slot_base = 0;
      const int strip = u / gg.groups, grp = u % gg.groups;
      const int ib = strip / gg.NJ, jb = strip % gg.NJ;
      const int i0 = half * PR + ib * 16, j0 = jb * JB;
      // rescale this unit's accumulators where a column exponent grew
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int gi = i0 + (lane >> 2) + ((r >> 1) << 3);
          const int gj = j0 + nt * 8 + 2 * (lane & 3) + (r & 1);
          const int k = slot_base + nt * 4 + r;
          shift_pair(acc_hi[k], acc_lo[k], Edel[gi] + Edel[gj], 24);
        }
      // order o: T_o = sum over pairs s <= t, s + t = o of (2 if s < t else 1)
      // D_s^T D_t; orders (0, 1), (2, 3), (4, 5) combined in int32, then
      // added to the int64 word of their order group with its weight
      int pend = 0;  // T of the even order of the current pair of orders, per slot
      int tv[NTILE][4];
#pragma unroll
      for (int d = 0; d <= kMaxOrder; ++d) {
        if (!order_in_group(gg.groups, grp, d)) continue;
        float c[NTILE][4];
#pragma unroll
        for (int nt = 0; nt < NTILE; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll 1
        for (int s = 0; 2 * s <= d; ++s) {
          const int tt = d - s;
          const bool diag = (s == tt);
          const uint16_t *As = planes + ((size_t)s * NT + i0) * kOzLDK;
          const uint16_t *Bt = planes + ((size_t)tt * NT + j0) * kOzLDK;
#pragma unroll 2
          for (int ks = 0; ks < kOzTR; ks += 16) {
            uint32_t a0, a1, a2, a3;
            {
              const int mi = lane >> 3, rr = lane & 7;
              const uint16_t *pa = As + ((mi & 1) * 8 + rr) * kOzLDK + ks + (mi >> 1) * 8;
              ldsm_x4(smem_u32(pa), a0, a1, a2, a3);
            }
            if (!diag) {
              a0 = bf16x2_twice(a0);
              a1 = bf16x2_twice(a1);
              a2 = bf16x2_twice(a2);
              a3 = bf16x2_twice(a3);
            }
#pragma unroll
            for (int nt = 0; nt < NTILE; nt += 2) {
              uint32_t b0, b1, b2, b3;
              const int mi = lane >> 3, rr = lane & 7;
              const uint16_t *pb2 = Bt + ((nt + (mi >> 1)) * 8 + rr) * kOzLDK + ks + (mi & 1) * 8;
              ldsm_x4(smem_u32(pb2), b0, b1, b2, b3);
              mma_bf16(c[nt], a0, a1, a2, a3, b0, b1);
              mma_bf16(c[nt + 1], a0, a1, a2, a3, b2, b3);
            }
          }
        }
        // drain: with one group the order pairs (2k, 2k+1) are combined as
        // T_2k 2^8 + T_2k+1 in int32 (order 6 alone); with four groups each
        // order alone.  hi holds orders 0..3 (unit: order 3), lo 4..6.
        const bool hi = d <= 3;
        if (gg.groups == 1 && (d & 1) == 0 && d < kMaxOrder) {
#pragma unroll
          for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) tv[nt][r] = f2i(c[nt][r]);
          pend = 1;
        } else {
          const int shl = hi ? 8 * (3 - d) : 8 * (kOzMaxOrder - d);
#pragma unroll
          for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int v = f2i(c[nt][r]);
              const long long w = pend ? (long long)(tv[nt][r] * 256 + v) : (long long)v;
              const int k = slot_base + nt * 4 + r;
              if (hi) acc_hi[k] += w << shl;
              else acc_lo[k] += w << shl;
            }
          pend = 0;
        }
      }
      }
    }
    __syncthreads();
  }

  // ---- combine the order groups exactly, round to FP64 once per entry
  // (ohi, olo reuse the tile and plane storage, which lie back to back)
  static_assert(sizeof(double) * NT * kOzTR + sizeof(uint16_t) * kOzDigits * NT * kOzLDK >=
                    2 * sizeof(long long) * PR * NT,
                "the group combine must fit in the tile and plane storage");
  long long *ohi = (long long *)smem;  // PR x NT
  long long *olo = ohi + PR * NT;      // PR x NT
  for (int e = t; e < PR * NT; e += kOzThreads) {
    ohi[e] = 0;
    olo[e] = 0;
  }
  __syncthreads();
  for (int g = 0; g < gg.groups; ++g) {
    {
      const int u = warp;
      const int slot_base = 0;
      if (u < gg.units && u % gg.groups == g) {
      const int strip = u / gg.groups;
      const int ib = strip / gg.NJ, jb = strip % gg.NJ;
      const int i0 = ib * 16, j0 = jb * JB;  // local row of P
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int li = i0 + (lane >> 2) + ((r >> 1) << 3);
          const int gj = j0 + nt * 8 + 2 * (lane & 3) + (r & 1);
          const int k = slot_base + nt * 4 + r;
          ohi[li + gj * PR] += acc_hi[k];
          olo[li + gj * PR] += acc_lo[k];
        }
      }
    }
    __syncthreads();
  }
  const bool bad = *flag != 0;
  if (a.emax != nullptr && half == 0)
    for (int j = t; j < n; j += kOzThreads) atomicMax(a.emax + j, Erun[j]);
  double *P = a.partials + grp_id * n * n;
  for (int e = t; e < PR * n; e += kOzThreads) {
    const int li = e % PR, j = e / PR, i = half * PR + li;
    if (i >= n) continue;
    // P_ij = (hi 2^24 + lo) 2^(Erun_i + Erun_j - 2109)
    const double v = bad ? __longlong_as_double(0x7FF8000000000000ll)
                         : fixed_to_double(ohi[li + j * PR], olo[li + j * PR], 24, Erun[i] + Erun[j] - 2109);
    const int64_t pe = i + (int64_t)j * n;
    P[pe] = a.accumulate ? P[pe] + v : v;
  }
}

size_t ozgram_smem_bytes(int NT) {
  return sizeof(double) * NT * kOzTR + sizeof(uint16_t) * kOzDigits * NT * kOzLDK + sizeof(int) * (2 * NT + 4);
}

int ozgram_nt(int n) { return n <= 16 ? 16 : (n <= 32 ? 32 : (n <= 64 ? 64 : 128)); }

template <int NT, int ND>
static cudaError_t launch_oz(const RowSweep &a, int grid, cudaStream_t s) {
  static KernelAttr attr;
  const size_t smem = ozgram_smem_bytes(NT);
  set_smem_attr(attr, ozgram_kernel<NT, ND>, (int)smem, true);
  // the fused solve exists for n <= 64 only
  if (NT > 64 && a.do_trsm) return cudaErrorInvalidValue;
  ozgram_kernel<NT, ND><<<grid * OzCfg<NT>::halves, OzCfg<NT>::threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int ND>
static cudaError_t launch_oz_nd(const RowSweep &a, int grid, cudaStream_t s) {
  switch (ozgram_nt(a.p)) {
    case 16: return launch_oz<16, ND>(a, grid, s);
    case 32: return launch_oz<32, ND>(a, grid, s);
    case 64: return launch_oz<64, ND>(a, grid, s);
    case 128: return launch_oz<128, ND>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ozgram(const RowSweep &a, int grid, cudaStream_t s) {
  if (a.digits == kOzMixedDigits) return launch_oz_nd<kOzMixedDigits>(a, grid, s);
  if (a.digits != 0 && a.digits != kOzDigits) return cudaErrorInvalidValue;
  if (tcgram_usable(a)) return launch_tcgram(a, grid, s);
  return launch_oz_nd<kOzDigits>(a, grid, s);
}

// Number of row groups (= partials) for m rows at width n: every SM holds
// OzCfg::ctas CTAs, a row group takes OzCfg::halves of them.
int ozgram_grid(int64_t m, int n, bool tc05) {
  // the tcgen05 kernel runs one CTA per SM (launch_ozgram falls back to the
  // mma.sync kernel with the same row groups when it does not apply)
  if (tc05 && n >= kTcGramMinN && n <= 64) return tcgram_grid(m);
  const int64_t tiles = (m + kOzTR - 1) / kOzTR;
  const int64_t per_sm = (n > 64) ? 1 : 2, halves = (n > 64) ? 2 : 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, per_sm * num_sms() / halves));
}

int ozgram_tile_rows() { return kOzTR; }

// Reduction of the symmetric-pair partials: X_ij = sum_g (P_g[i,j] + P_g[j,i]).
// CTA j forms column j: thread (i, gq) sums the partials g = gq (mod NG) in
// increasing g, the NG sums are added in increasing gq.  X_ji (CTA i) adds
// the same terms in the same order (a + b = b + a), so X is exactly
// symmetric.  The partials are L2-resident; the loads of a thread are
// independent, so they overlap.
__global__ void __launch_bounds__(256) reduce_oz_kernel(const double *partials, int G, int n, double *C,
                                                        const DevState *st) {
  if (st != nullptr && st->done) return;
  __shared__ double part[256];
  const int j = blockIdx.x, t = threadIdx.x;
  const int ni = n <= 32 ? 32 : (n <= 64 ? 64 : 128);
  const int ng = 256 / ni, i = t % ni, gq = t / ni;
  const int64_t nn = (int64_t)n * n;
  double s = 0.0;
  if (i < n) {
    const double *P0 = partials + i + (int64_t)j * n;
    const double *P1 = partials + j + (int64_t)i * n;
#pragma unroll 4
    for (int g = gq; g < G; g += ng) s += P0[g * nn] + P1[g * nn];
  }
  part[t] = s;
  __syncthreads();
  if (gq == 0 && i < n) {
    double tot = 0.0;
    for (int h = 0; h < ng; ++h) tot += part[h * ni + i];
    C[i + (int64_t)j * n] = tot;
  }
}

cudaError_t launch_reduce_oz(const double *partials, int G, int n, double *C, const DevState *st,
                             cudaStream_t s) {
  if (n < 1 || n > 128) return cudaErrorInvalidValue;
  reduce_oz_kernel<<<n, 256, 0, s>>>(partials, G, n, C, st);
  return cudaGetLastError();
}

}  // namespace cqr
