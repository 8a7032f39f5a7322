// Exact FP64 Gramian X = Y^T Y (Alg. 1) on the Blackwell
// tensor cores with tcgen05: the digit scheme of ozgram.cu (Ozaki, Ogita,
// Oishi, Rump, Numer. Algorithms 59, 2012), moved from warp-level mma.sync to
// tcgen05.mma with TMEM accumulators, TMA row tiles and warp-specialised
// roles.  Widths 17 <= n <= 64 (columns padded to 64 with zeros).
//
// Numbers (the same as ozgram.cu): per CTA and column j, E_j is the running
// maximum biased exponent over the rows seen so far; each element is
// sign * V * 2^(E_j - 1078) with V < 2^56 in 7 balanced base-256 digits
// D_0 in [0, 256], D_1..D_6 in [-128, 127].  Orders o = s + t <= 6 of the
// digit products are kept; with P_st^T = P_ts only s <= t is formed, and
// per 64-row tile the order-o sum
//   T_o = sum_{s < t, s + t = o} 2 D_s^T D_t + [o even] D_{o/2}^T D_{o/2}
// is an exact FP32 integer (|T_o| <= 9 * 2^20 < 2^24).  The CTA keeps
// V_ij = sum over tiles of sum_o T_o 2^(8 (6 - o)) as an exact integer,
// rescaled (floor) when a column exponent grows, and writes its partial
// P_ij = V_ij 2^(E_i + E_j - 2109), rounded to FP64 once; the reduction
// returns X = sum_g (P_g + P_g^T).
//
// Tensor-core mapping.  A tile's digits are written to shared memory as 11
// planes of 64 (columns of Y) x 64 (rows of the tile) bf16 values, K-major
// with the 128-byte swizzle:
//   p0 D3, p1 D0, p2 2D1, p3 D1, p4 2D2, p5 2D3, p6 2D4, p7 2D5, p8 2D6,
//   p9 D2, p10 2D3
// (2D: the digit doubled, exact in bf16).  An MMA with M = 128 takes two
// consecutive planes [p; p+1] as A (lanes 0-63 and 64-127 of D) and one plane
// as B (N = 64), K = 64 in four steps.  Four TMEM regions of 128 lanes x 64
// columns hold the orders (top lanes / bottom lanes):
//   R0 (T0 / T1):  [p1;p2] x D0
//   R1 (T2 / T3):  [p4;p5] x D0, [p3;p4] x D1
//   R2 (T4 / T5):  [p6;p7] x D0, [p5;p6] x D1, [p9;p10] x D2
//   R3 (T6 / -):   [p8;p9] x D0, [p7;p8] x D1, [p6;p7] x D2, [p0;p1] x D3
// which forms each of the 16 blocks once with its weight (the bottom half of
// R3 is not used): 10 MMAs of 128 x 64 x 64 per tile instead of 16 of
// 64 x 64 x 64.  Two region sets (512 TMEM columns) alternate between tiles,
// so the products of one tile overlap the drain of the previous one.
//
// Roles (512 threads, one CTA per SM; 16 warps of up to 128 registers, four
// per 16K-register sub-partition of the SM, so that each scheduler has two
// splitting warps to hide the latency of the digit arithmetic):
//   warps 0-7   split: wait for the TMA tile, hold their 8 columns (two rows
//               per lane) in registers, release the tile, update E_j, write
//               the 11 planes; one mbarrier phase per tile and plane stage.
//               Lane 0 of warp 0 also issues the TMA loads of the 64 x 64
//               FP64 tiles of Y: the next one as soon as every split warp
//               has taken the current one into registers (and prefetches
//               the one after it into L2).  Lane 0 of warps 1, 2 and 3
//               issues the 40 tcgen05.mma of a tile (16, 12 and 12, by
//               accumulator region) once every split warp has written its
//               planes, at the start of the next tile, after releasing the
//               staging tile; warp 1 also allocates and frees the 512 TMEM
//               columns.
//   warps 8-15  drain: lane L of warp w reads TMEM lane L = 32 (w % 4) + lane
//               (entry row L mod 64; orders T0, T2, T4, T6 for L < 64 and T1,
//               T3, T5 for L >= 64) for 32 columns (half (w - 8) / 4), converts
//               the exact FP32 sums to integers and adds them into a 96-bit
//               integer per entry (int64 high part, uint32 low part).  At the
//               end the two halves of each entry are added and rounded.
// Every wait gives up after kWaitNs of wall time; the CTA then writes NaN
// partials (the control step reports a breakdown) and still frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "cqr_internal.cuh"
#include "ozdigits.cuh"
#include "tc05.cuh"

namespace cqr {

using namespace tc05;

namespace {

constexpr int kTR = 64;                               // tile rows (one exact window)
constexpr int kNT = 64;                               // columns, padded
constexpr int kPlanes = 11;
constexpr int kPlaneBytes = kNT * kTR * 2;            // 8 KB
constexpr int kStageBytes = kPlanes * kPlaneBytes;    // 88 KB
constexpr int kRawBytes = kTR * kNT * 8;              // 32 KB
constexpr int kSplitWarps = 8, kDrainWarps = 8;
constexpr int kColsPerSplit = kNT / kSplitWarps;      // 8 columns per split warp
constexpr int kMmaWarp = 1;                           // allocates and frees TMEM; the first MMA issuer
// Lane 0 of split warps kMmaWarp .. kMmaWarp + kIssuers - 1 issues the MMAs
// of a tile, each those of its own accumulator regions (R3; R2; R1 and R0:
// 16, 12 and 12 MMAs), so that no warp spends the whole issue time
constexpr int kIssuers = 3;
__host__ __device__ constexpr int region_issuer(int r) { return r == 3 ? 0 : (r == 2 ? 1 : 2); }
constexpr int kTcThreads = (kSplitWarps + kDrainWarps) * 32;  // 512, launched with 128 registers each
// setmaxnreg: the split warpgroups give registers to the drain warpgroups
// (8 x 32 x 80 + 8 x 32 x 176 = 512 x 128)
constexpr int kSplitRegs = 80, kDrainRegs = 176;
static_assert(kSplitWarps * kSplitRegs + kDrainWarps * kDrainRegs == (kSplitWarps + kDrainWarps) * 128,
              "register reallocation must add up to the launch's registers");
// exponent-growth records in flight: a split warp starts tile k only after
// the drain of tile k - 5 is done, so 8 slots are never overwritten early
constexpr int kRing = 8;
constexpr uint64_t kWaitNs = 2000000000ull;           // 2 s
constexpr int kPrefetchAhead = 2;                     // tiles prefetched into L2 ahead of the TMA load
constexpr unsigned long long kBalance = 0x0000808080808080ull;

// shared-memory layout (offsets from a 1024-byte aligned base)
constexpr int kOffPlanes = 0;
constexpr int kOffRaw = 2 * kStageBytes;
constexpr int kOffCtrl = kOffRaw + kRawBytes;
struct Ctrl05 {
  uint64_t raw_full, raw_empty;
  uint64_t planes_full[2], planes_empty[2];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t meta_full[kRing];
  uint32_t tmem_slot;
  int bad;       // a non-finite entry was seen
  int timeout;   // a wait gave up
  int pad;
  int edel[kRing][kNT];     // exponent growth of each column in tile k (slot k % kRing)
  int grew[kRing][kSplitWarps];  // per split warp: some column of its own grew
  int erun[kNT];            // final running exponents
};
constexpr size_t kSmemBytes = 1024 + kOffCtrl + sizeof(Ctrl05);
static_assert(kSmemBytes <= 227 * 1024, "shared memory of the tcgen05 Gramian");
static_assert(kStageBytes % 1024 == 0 && kOffRaw % 1024 == 0, "1024-byte aligned operands");
static_assert(kDrainWarps * 32 * 12 <= 2 * kStageBytes, "the final combine fits in the plane stages");

// (A plane, B plane, region, overwrites) of the 10 MMAs of a tile, in the
// order they are issued within a K step: regions 0, 1, 2, 3, 1, 2, 3, 2, 3, 3,
// so that consecutive MMAs rarely wait for each other's accumulator; the first
// MMA into each region overwrites it
struct MmaUnit {
  int a, b, r, first;
};
__host__ __device__ constexpr MmaUnit mma_unit(int q) {
  return q == 0   ? MmaUnit{1, 1, 0, 1}
         : q == 1 ? MmaUnit{4, 1, 1, 1}
         : q == 2 ? MmaUnit{6, 1, 2, 1}
         : q == 3 ? MmaUnit{8, 1, 3, 1}
         : q == 4 ? MmaUnit{3, 3, 1, 0}
         : q == 5 ? MmaUnit{5, 3, 2, 0}
         : q == 6 ? MmaUnit{7, 3, 3, 0}
         : q == 7 ? MmaUnit{9, 9, 2, 0}
         : q == 8 ? MmaUnit{6, 9, 3, 0}
                  : MmaUnit{0, 0, 3, 0};
}

// named barriers (0 is __syncthreads)
constexpr int kBarErun = 1;   // split warps publish the final exponents to the drain warps
constexpr int kBarDrain = 2;  // the drain warps among themselves
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// byte offset of element (column j, tile row i) in a plane
__device__ __forceinline__ uint32_t plane_off(int j, int i) {
  return (uint32_t)((j >> 3) * 1024 + (j & 7) * 128 + ((((i >> 3) ^ (j & 7))) << 4) + (i & 7) * 2);
}

// digit i (0..6) of W with sign s as an exact FP32 integer (ozgram.cu)
__device__ __forceinline__ float digit_of(unsigned long long W, int i, float s) {
  if (i == 0) return fmaf(__int_as_float(0x4B000000 | (int)(W >> 48)), s, -s * 8388608.0f);
  const int b = 6 - i;
  const uint32_t word = (b >= 4) ? (uint32_t)(W >> 32) : (uint32_t)W;
  const float x = __int_as_float((int)__byte_perm(word, 0x4B000000u, 0x7440u | (uint32_t)(b & 3)));
  return fmaf(x, s, -s * 8388736.0f);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t twice_bf16x2(uint32_t x) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&x);
  h = __hadd2(h, h);
  return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ int f2i_exact(uint32_t bits) {
  int r;
  asm("cvt.rzi.s32.f32 %0, %1;" : "=r"(r) : "f"(__uint_as_float(bits)));
  return r;
}

// V = hi 2^32 + lo (two's complement, 96 bits) <- floor(V / 2^D), without
// branches; D >= 62 drops the old value (below 2^-62 of the entry's new
// scale), as ozgram.cu does
__device__ __forceinline__ void shift96(long long &hi, uint32_t &lo, int D) {
  const int d = min(max(D, 0), 63);
  const uint32_t lo_small = __funnelshift_r(lo, (uint32_t)hi, (uint32_t)d);  // d < 32
  const uint32_t lo_large = (uint32_t)(hi >> (d >= 32 ? d - 32 : 0));        // d >= 32
  const long long hi_new = hi >> d;
  const bool drop = D >= 62;
  lo = drop ? 0u : (d >= 32 ? lo_large : lo_small);
  hi = drop ? 0ll : hi_new;
}

}  // namespace

// One CTA: rows [g rows_per_cta, ...) of row group g (rows_per_cta a multiple
// of 64), in 64-row tiles; writes P (n x n, ld n) to partials[g n n].
__global__ void __launch_bounds__(kTcThreads, 1) tcgram64_kernel(const __grid_constant__ CUtensorMap tmap, RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  Ctrl05 *cs = (Ctrl05 *)(base + kOffCtrl);
  const uint32_t sbase = smem_addr(base);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int n = a.p;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  const int ntiles = (row1 > row0) ? (int)((row1 - row0 + kTR - 1) / kTR) : 0;
  const uint32_t bar_raw_full = smem_addr(&cs->raw_full), bar_raw_empty = smem_addr(&cs->raw_empty);

  if (t == 0) {
    mbar_init(bar_raw_full, 1);
    mbar_init(bar_raw_empty, kSplitWarps);
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_addr(&cs->planes_full[s]), kSplitWarps);
      mbar_init(smem_addr(&cs->planes_empty[s]), kIssuers);  // one commit per issuer
      mbar_init(smem_addr(&cs->acc_full[s]), kIssuers);
      mbar_init(smem_addr(&cs->acc_empty[s]), kDrainWarps);
    }
    for (int r = 0; r < kRing; ++r) mbar_init(smem_addr(&cs->meta_full[r]), kSplitWarps);
    cs->bad = 0;
    cs->timeout = 0;
    mbar_init_fence();
  }
  if (warp == kMmaWarp) tmem_alloc(smem_addr(&cs->tmem_slot), 512);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = cs->tmem_slot;

  const int dw = warp - kSplitWarps;  // drain warps: 0..7
  const int quad = warp & 3, half = (dw >> 2) & 1;
  const int lrow = quad * 32 + lane;  // TMEM lane
  const int side = lrow >> 6, ent_i = lrow & 63;

  if (warp == 0 && lane == 0 && ntiles > 0) {
    prefetch_tmap(&tmap);
    mbar_arrive_expect_tx(bar_raw_full, kRawBytes);
    tma_load_2d(sbase + kOffRaw, &tmap, (int)row0, 0, bar_raw_full);
    for (int i = 1; i <= kPrefetchAhead; ++i)
      if (row0 + (int64_t)i * kTR < row1) tma_prefetch_l2_2d(&tmap, (int)(row0 + (int64_t)i * kTR), 0);
  }
  if (warp < kSplitWarps) {
    regs_dec<kSplitRegs>();
    // ---- split: columns warp * 8 .. + 7, rows 2 lane, 2 lane + 1 of each tile
    int erun[kColsPerSplit];
#pragma unroll
    for (int c = 0; c < kColsPerSplit; ++c) erun[c] = 1;
    const double *raw = (const double *)(base + kOffRaw);
    constexpr uint32_t idesc = idesc_bf16_f32(128, kNT);
    int issued = 0;  // MMA tiles issued (issuer warps, lane 0)
    // MMA issue of tile kk by this issuer warp (its regions only): every
    // split warp has written its planes and the drain of tile kk - 2 has
    // released the region set.  Returns false (for the whole warp) when a
    // wait gave up.
    const int me = warp - kMmaWarp;  // issuer index, valid for 0 <= me < kIssuers
    const bool issuer = me >= 0 && me < kIssuers;
    auto issue = [&](int kk) -> bool {
      const int ss = kk & 1;
      int ok = 1;
      if (lane == 0) {
        ok = mbar_wait(smem_addr(&cs->planes_full[ss]), (kk >> 1) & 1, kWaitNs) &&
             (kk < 2 || mbar_wait(smem_addr(&cs->acc_empty[ss]), ((kk >> 1) - 1) & 1, kWaitNs));
        if (ok) {
          fence_after_sync();
          const uint32_t stage = sbase + kOffPlanes + ss * kStageBytes;
          const uint32_t dbase = tmem + (uint32_t)(ss * 4 * kNT);
          // K step by K step; the first MMA into each region (its first
          // unit, K step 0) overwrites it
#pragma unroll 1
          for (int ks = 0; ks < 4; ++ks)
#pragma unroll
            for (int q = 0; q < 10; ++q) {
              const MmaUnit U = mma_unit(q);
              if (region_issuer(U.r) != me) continue;
              const uint64_t ad = sdesc_sw128(stage + U.a * kPlaneBytes + ks * 32);
              const uint64_t bd = sdesc_sw128(stage + U.b * kPlaneBytes + ks * 32);
              mma_ss(dbase + (uint32_t)(U.r * kNT), ad, bd, idesc, (U.first && ks == 0) ? 0u : 1u);
            }
          mma_commit(smem_addr(&cs->planes_empty[ss]));
          mma_commit(smem_addr(&cs->acc_full[ss]));
          ++issued;
        }
      }
      return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };
    bool aborted = false;
    for (int k = 0; k < ntiles; ++k) {
      const int s = k & 1, slot = k % kRing;
      if (!__all_sync(0xffffffffu, mbar_wait(bar_raw_full, k & 1, kWaitNs))) {
        cs->timeout = 1;
        aborted = true;
        break;
      }
      double2 v[kColsPerSplit];
#pragma unroll
      for (int c = 0; c < kColsPerSplit; ++c) v[c] = *(const double2 *)(raw + (warp * kColsPerSplit + c) * kTR + 2 * lane);
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_raw_empty);
      if (warp == 0 && lane == 0 && k + 1 < ntiles) {
        // every split warp has the tile in registers: load the next one
        if (!mbar_wait(bar_raw_empty, k & 1, kWaitNs)) {
          cs->timeout = 1;
        } else {
          mbar_arrive_expect_tx(bar_raw_full, kRawBytes);
          tma_load_2d(sbase + kOffRaw, &tmap, (int)(row0 + (int64_t)(k + 1) * kTR), 0, bar_raw_full);
          // and bring the tile after it into L2, so that its load, issued
          // one tile later, waits on L2 rather than HBM
          if (row0 + (int64_t)(k + 1 + kPrefetchAhead) * kTR < row1)
            tma_prefetch_l2_2d(&tmap, (int)(row0 + (int64_t)(k + 1 + kPrefetchAhead) * kTR), 0);
        }
      }
      // the products of the previous tile are issued only now, after this
      // warp has released the staging tile, so that the next TMA load does
      // not wait for the issue
      if (issuer && k >= 1 && !issue(k - 1)) {
        cs->timeout = 1;
        aborted = true;
        break;
      }
      // column exponents: running maximum and its growth in this tile
      int grew = 0, nonfinite = 0;
#pragma unroll
      for (int c = 0; c < kColsPerSplit; ++c) {
        const int e0 = (int)((__double2hiint(v[c].x) >> 20) & 0x7FF);
        const int e1 = (int)((__double2hiint(v[c].y) >> 20) & 0x7FF);
        const int mx = __reduce_max_sync(0xffffffffu, max(1, max(e0, e1)));
        const int nw = max(erun[c], mx);
        const int del = nw - erun[c];
        erun[c] = nw;
        grew |= del;
        nonfinite |= (mx == 0x7FF);
        if (lane == 0) cs->edel[slot][warp * kColsPerSplit + c] = del;
      }
      if (lane == 0) {
        cs->grew[slot][warp] = grew;
        if (nonfinite) cs->bad = 1;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&cs->meta_full[slot]));
      // the plane stage is free once the MMAs of tile k - 2 have completed
      if (k >= 2 && !__all_sync(0xffffffffu, mbar_wait(smem_addr(&cs->planes_empty[s]), ((k >> 1) - 1) & 1, kWaitNs))) {
        cs->timeout = 1;
        aborted = true;
        break;
      }
      unsigned char *stage = base + kOffPlanes + s * kStageBytes;
#pragma unroll
      for (int c = 0; c < kColsPerSplit; ++c) {
        const int j = warp * kColsPerSplit + c;
        const int Ej = erun[c];
        unsigned long long W[2];
        float sg[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(h ? v[c].y : v[c].x);
          const int ef = (int)((b >> 52) & 0x7FF);
          unsigned long long M = b & 0xFFFFFFFFFFFFFull;
          if (ef) M |= 0x10000000000000ull;
          if (ef == 0x7FF) M = 0;
          const int sh = Ej - (ef ? ef : 1);
          W[h] = ((sh >= 56) ? 0ull : ((M << 3) >> sh)) + kBalance;
          sg[h] = (b >> 63) ? -1.0f : 1.0f;
        }
        uint32_t P[7];
#pragma unroll
        for (int d = 0; d < 7; ++d) P[d] = pack_bf16x2(digit_of(W[0], d, sg[0]), digit_of(W[1], d, sg[1]));
        const uint32_t off = plane_off(j, 2 * lane);
        const uint32_t d3x2 = twice_bf16x2(P[3]);
        *(uint32_t *)(stage + 0 * kPlaneBytes + off) = P[3];
        *(uint32_t *)(stage + 1 * kPlaneBytes + off) = P[0];
        *(uint32_t *)(stage + 2 * kPlaneBytes + off) = twice_bf16x2(P[1]);
        *(uint32_t *)(stage + 3 * kPlaneBytes + off) = P[1];
        *(uint32_t *)(stage + 4 * kPlaneBytes + off) = twice_bf16x2(P[2]);
        *(uint32_t *)(stage + 5 * kPlaneBytes + off) = d3x2;
        *(uint32_t *)(stage + 6 * kPlaneBytes + off) = twice_bf16x2(P[4]);
        *(uint32_t *)(stage + 7 * kPlaneBytes + off) = twice_bf16x2(P[5]);
        *(uint32_t *)(stage + 8 * kPlaneBytes + off) = twice_bf16x2(P[6]);
        *(uint32_t *)(stage + 9 * kPlaneBytes + off) = P[2];
        *(uint32_t *)(stage + 10 * kPlaneBytes + off) = d3x2;
      }
      fence_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&cs->planes_full[s]));
    }
    // the products of the last tile
    if (issuer && !aborted && ntiles > 0 && !issue(ntiles - 1)) cs->timeout = 1;
    // every issued product completes before TMEM is freed: each issuer waits
    // for its last tile (whose barrier also counts the other issuers)
    if (issuer && lane == 0 && issued > 0 &&
        !mbar_wait(smem_addr(&cs->acc_full[(issued - 1) & 1]), ((issued - 1) >> 1) & 1, kWaitNs))
      cs->timeout = 1;
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < kColsPerSplit; ++c) cs->erun[warp * kColsPerSplit + c] = erun[c];
    }
    // the final exponents are published to the drain warps
    named_bar_arrive(kBarErun, (kSplitWarps + kDrainWarps) * 32);
  } else {
    regs_inc<kDrainRegs>();
    // ---- drain: TMEM lane lrow, columns half * 32 .. + 31; entry
    // (ent_i, half * 32 + c) of this thread's side in hi[c] 2^32 + lo[c]
    long long hi[32];
    uint32_t lo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      hi[c] = 0;
      lo[c] = 0;
    }
    for (int k = 0; k < ntiles; ++k) {
      const int b = k & 1, slot = k % kRing;
      const bool ready = mbar_wait(smem_addr(&cs->acc_full[b]), (k >> 1) & 1, kWaitNs) &&
                         mbar_wait(smem_addr(&cs->meta_full[slot]), (k / kRing) & 1, kWaitNs);
      if (!__all_sync(0xffffffffu, ready)) {
        cs->timeout = 1;
        break;
      }
      fence_after_sync();
      int anygrew = 0;
#pragma unroll
      for (int w = 0; w < kSplitWarps; ++w) anygrew |= cs->grew[slot][w];
      if (anygrew != 0) {
        const int ei = cs->edel[slot][ent_i];
        const int4 *ej = (const int4 *)&cs->edel[slot][half * 32];
#pragma unroll
        for (int c4 = 0; c4 < 8; ++c4) {
          const int4 d = ej[c4];
          shift96(hi[4 * c4 + 0], lo[4 * c4 + 0], ei + d.x);
          shift96(hi[4 * c4 + 1], lo[4 * c4 + 1], ei + d.y);
          shift96(hi[4 * c4 + 2], lo[4 * c4 + 2], ei + d.z);
          shift96(hi[4 * c4 + 3], lo[4 * c4 + 3], ei + d.w);
        }
      }
      const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * 4 * kNT + half * 32);
      // one region and 8 columns at a time: order o enters V with weight
      // 2^(8 (6 - o)); hi carries 2^32 and up, lo the low 32 bits
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (side == 1 && r == 3) break;  // the bottom half of R3 is unused
        const int o = 2 * r + side;
        const int w = 8 * (6 - o);       // 48, 32, 16, 0 (top) / 40, 24, 8 (bottom)
        // the region's 32 columns in one load and one wait
        uint32_t x[32];
        tmem_ld32(tb + (uint32_t)(r * kNT), x);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const long long tv = (long long)f2i_exact(x[e]);
          if (w >= 32) {
            hi[e] += tv << (w - 32);
          } else {
            const long long sum = (long long)lo[e] + (tv << w);
            lo[e] = (uint32_t)sum;
            hi[e] += sum >> 32;
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&cs->acc_empty[b]));
    }

    // ---- the two halves of each entry, one rounding, the partial.  After
    // the last tile's products every plane stage is free (the MMAs of the
    // last tile, which read the last planes, have completed).
    named_bar_sync(kBarErun, (kSplitWarps + kDrainWarps) * 32);
    long long *cb_hi = (long long *)(base + kOffPlanes);
    uint32_t *cb_lo = (uint32_t *)(base + kOffPlanes + sizeof(long long) * kNT * kNT);
    if (side == 1) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int e = ent_i * kNT + half * 32 + c;
        cb_hi[e] = hi[c];
        cb_lo[e] = lo[c];
      }
    }
    named_bar_sync(kBarDrain, kDrainWarps * 32);
    if (side == 0) {
    const bool bad = (cs->bad != 0) || (cs->timeout != 0);
    double *P = a.partials + (int64_t)blockIdx.x * n * n;
    const int i = ent_i;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int j = half * 32 + c;
      if (i >= n || j >= n) continue;
      const int e = i * kNT + j;
      long long H = hi[c] + cb_hi[e];
      const long long s = (long long)lo[c] + (long long)cb_lo[e];
      const uint32_t L = (uint32_t)s;
      H += s >> 32;
      // V = H 2^32 + L  ->  (V >> 24) 2^24 + (V mod 2^24)
      const long long h24 = (long long)(((unsigned long long)H << 8) | (unsigned long long)(L >> 24));
      const long long l24 = (long long)(L & 0xFFFFFFu);
      const double v = bad ? __longlong_as_double(0x7FF8000000000000ll)
                           : oz::fixed_to_double(h24, l24, 24, cs->erun[i] + cs->erun[j] - 2109);
      const int64_t pe = i + (int64_t)j * n;
      P[pe] = a.accumulate ? P[pe] + v : v;
    }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == kMmaWarp) {
    fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- host side

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, through the runtime (no link
// against libcuda); null if unavailable
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    (void)cudaGetLastError();
  });
  return fn;
}

// compute capability 10.3 (GB300) on the current device, cached per device
bool device_is_sm103() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return false;
  }
  int v = cached[dev].load();
  if (v == 0) {
    int ma = 0, mi = 0;
    cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev);
    (void)cudaGetLastError();
    v = (ma == 10 && mi == 3) ? 1 : 2;
    cached[dev].store(v);
  }
  return v == 1;
}

// the kernel launches with its 384 threads on this device (registers and
// shared memory), checked once per device
bool kernel_launchable() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return false;
  }
  int v = cached[dev].load();
  if (v == 0) {
    cudaFuncAttributes fa;
    int optin = 0;
    const bool ok = cudaFuncGetAttributes(&fa, tcgram64_kernel) == cudaSuccess &&
                    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
                    fa.maxThreadsPerBlock >= kTcThreads && (size_t)optin >= kSmemBytes + fa.sharedSizeBytes;
    (void)cudaGetLastError();
    v = ok ? 1 : 2;
    cached[dev].store(v);
  }
  return v == 1;
}

}  // namespace

// Rows of a CTA are capped so that the exact sums stay below 2^86 (8192 tiles).
constexpr int64_t kTcGramMaxRowsPerCta = (int64_t)8192 * kTR;

bool tcgram_usable(const RowSweep &a) {
  return (a.tc05 & kTc05Gram) && a.q == 0 && a.p >= kTcGramMinN && a.p <= kNT && !a.do_trsm && a.m >= 1 &&
         a.digits == 0 && a.emax == nullptr &&
         (((uintptr_t)a.Yin) & 15) == 0 && (a.ldyin % 2) == 0 && a.rows_per_cta % kTR == 0 &&
         a.rows_per_cta <= kTcGramMaxRowsPerCta && a.m <= 0x7FFFFFFF && device_is_sm103() &&
         encode_tiled() != nullptr && kernel_launchable();
}

int tcgram_grid(int64_t m) {
  const int64_t tiles = (m + kTR - 1) / kTR;
  const int64_t need = (tiles + 8191) / 8192;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, std::max<int64_t>(num_sms(), need)));
}

cudaError_t launch_tcgram(const RowSweep &a, int grid, cudaStream_t s) {
  if (!tcgram_usable(a)) return cudaErrorInvalidValue;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)a.m, (cuuint64_t)a.p};
  const cuuint64_t strides[1] = {(cuuint64_t)a.ldyin * sizeof(double)};
  const cuuint32_t box[2] = {(cuuint32_t)kTR, (cuuint32_t)kNT};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_tiled()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(a.Yin), dims,
                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  static KernelAttr attr;
  set_smem_attr(attr, tcgram64_kernel, (int)kSmemBytes, true);
  tcgram64_kernel<<<grid, kTcThreads, kSmemBytes, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace cqr
