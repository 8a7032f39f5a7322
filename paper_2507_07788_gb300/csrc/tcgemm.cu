// Q = Y T on the Blackwell tensor cores with tcgen05, T = D R~^{-1} (the
// triangular solve of Alg. 1 as an explicit inverse and a product,
// App. A), for widths 17 <= n <= 64 (padded to 64 with zeros).  The
// arithmetic is exactly that of ozgemm.cu (the Ozaki splitting scheme with
// balanced base-256 digits): Y's rows, scaled by D^-1, and T's columns are
// truncated to 63 bits below their largest exponent and written in 8 digits;
// the 36 ordered digit pairs of order o = i + i' <= 7 are multiplied, each
// order summed exactly in FP32 (at most 8 * 64 * 128^2 = 2^23), the orders
// combined exactly in two int64 words (orders 0..3, 4..7) and each entry
// rounded to FP64 once.  Every entry depends only on its row and column, so
// the result is bit for bit that of the mma.sync kernel.
//
// Tensor-core mapping: a tile of 128 rows; the 8 digit planes of the tile
// (A: 128 rows x 64 k, bf16, K-major, 128-byte swizzle, 16 KB each) and of T
// (B: 64 columns x 64 k, 8 KB each, written once per CTA) live in shared
// memory; MMA (i, i') = A_i B_i'^T is 128 x 64 x 64 (four K steps of 16).
// Two TMEM rounds of four regions (128 lanes x 64 columns each):
//   round 1, columns   0..255: orders 0..3 (10 digit pairs, 40 tcgen05.mma)
//   round 2, columns 256..511: orders 4..7 (26 digit pairs, 104 tcgen05.mma)
// so the drain of a tile's first round overlaps its second round's products.
//
// Roles (512 threads, one CTA per SM, 16 warps of up to 128 registers):
//   warps 0-7   split: thread (row r = 32 (w % 4) + lane, k half w / 4) loads
//               its 32 entries of the tile straight from global memory
//               (a warp reads 32 consecutive rows of a column: coalesced),
//               the row's largest scaled exponent is combined through shared
//               memory, and the 8 digits of its 32 entries go to the planes
//               as 16-byte stores.  The next tile's loads are issued before
//               waiting for the planes to be free.  Lane 0 of warp 0 issues
//               the tile's 144 MMAs once all eight warps have written it.
//   warps 8-15  drain: TMEM lane 32 (w % 4) + lane = row of the tile, 32
//               columns (half (w - 8) / 4): round 1 into one int64 word per
//               entry, then round 2 sixteen columns at a time, rounding each
//               entry of Q with the branch-free exact rounding (its entries'
//               dependency chains overlap) and storing it (a warp writes 32
//               consecutive rows of a column: coalesced).
// Every wait gives up after kQWaitNs of wall time (the CTA then writes NaN
// rows, and the control step reports a breakdown) and TMEM is still freed.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

#include "cqr_internal.cuh"
#include "ozdigits.cuh"
#include "tc05.cuh"

namespace cqr {

using namespace tc05;

namespace {

constexpr int kQR = 128;                          // tile rows
constexpr int kQN = 64;                           // padded width
constexpr int kQDig = 8;                          // digits of 63 bits
constexpr int kAPlane = kQR * kQN * 2;            // 16 KB
constexpr int kBPlane = kQN * kQN * 2;            // 8 KB
constexpr int kOffA = 0;
constexpr int kOffB = kQDig * kAPlane;            // 128 KB
constexpr int kOffC = kOffB + kQDig * kBPlane;    // 192 KB
constexpr int kQSplitW = 8, kQDrainW = 8;
constexpr int kQThreads = (kQSplitW + kQDrainW) * 32;  // 512, 128 registers each
constexpr int kQRing = 4;
constexpr uint64_t kQWaitNs = 2000000000ull;
constexpr int kNoExpQ = -(1 << 28);               // scaled exponent of a zero
constexpr unsigned long long kBal63 = 0x0080808080808080ull;
constexpr int kBarRowMax = 1;                     // named barrier of the split warps

struct CtrlQ {
  uint64_t planes_full, planes_empty;
  uint64_t r1_full, r1_empty, r2_full, r2_empty;
  uint64_t meta_full[kQRing];
  uint32_t tmem_slot;
  int timeout;
  int pad[2];
  int emax[2][2][kQR];      // [tile parity][k half][row]: partial row maxima
  int ebad[2][2][kQR];      // and non-finite flags
  int erow[kQRing][kQR];    // row exponent of tile k (slot k % kQRing)
  int rbad[kQRing][kQR];
  int fcol[kQN];            // column exponents of T
  int cs[kQN];              // column scales c_k of Y (D = diag(2^c_k))
};
constexpr size_t kQSmem = 1024 + kOffC + sizeof(CtrlQ);
static_assert(kQSmem <= 227 * 1024, "shared memory of the tcgen05 solve");

__device__ __forceinline__ void qbar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// byte offset of element (row r, k) in a K-major 128-byte-swizzled bf16
// plane with 64 k per row
__device__ __forceinline__ uint32_t sw_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7))) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ int scaled_exp_q(unsigned long long b, int c) {
  if ((b & 0x7FFFFFFFFFFFFFFFull) == 0) return kNoExpQ;
  const int ef = (int)((b >> 52) & 0x7FF);
  return (ef ? ef : 1) - c;
}

// 63-bit magnitude of x (bits b, column scale 2^-c) against exponent eref
__device__ __forceinline__ unsigned long long mag63(unsigned long long b, int eref, int c) {
  const int ef = (int)((b >> 52) & 0x7FF);
  unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  if (ef) M |= 0x10000000000000ull;
  if (ef == 0x7FF || M == 0) return 0ull;
  const int sh = eref - ((ef ? ef : 1) - c);
  return (sh >= 63) ? 0ull : ((M << 10) >> sh);
}

// balanced digit i of W = V + kBal63 with the element's sign s, exact FP32
__device__ __forceinline__ float bdigit(unsigned long long W, int i, float s) {
  const uint32_t word = (i < 4) ? (uint32_t)(W >> 32) : (uint32_t)W;
  const uint32_t byte = 3 - (i & 3);
  const float x = __int_as_float((int)__byte_perm(word, 0x4B000000u, 0x7440u | byte));
  return fmaf(x, s, -s * (i == 0 ? 8388608.0f : 8388736.0f));
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ int f2i_q(uint32_t bits) {
  int r;
  asm("cvt.rzi.s32.f32 %0, %1;" : "=r"(r) : "f"(__uint_as_float(bits)));
  return r;
}

}  // namespace

// One CTA: rows [g rows_per_cta, ...) of Y (rows_per_cta a multiple of 128)
// in 128-row tiles; Q = (Y D^-1)(D T) into a.Yout.
__global__ void __launch_bounds__(kQThreads, 1) tcgemm64_kernel(RowSweep a) {
  if (a.st != nullptr && a.st->done) return;
  const int64_t row0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);
  if (row0 >= row1) return;
  const int ntiles = (int)((row1 - row0 + kQR - 1) / kQR);
  extern __shared__ unsigned char smem_q[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_q + 1023) & ~(uintptr_t)1023);
  CtrlQ *cs = (CtrlQ *)(base + kOffC);
  const uint32_t sbase = smem_addr(base);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int n = a.p;

  if (t == 0) {
    mbar_init(smem_addr(&cs->planes_full), kQSplitW);
    mbar_init(smem_addr(&cs->planes_empty), 1);
    mbar_init(smem_addr(&cs->r1_full), 1);
    mbar_init(smem_addr(&cs->r1_empty), kQDrainW);
    mbar_init(smem_addr(&cs->r2_full), 1);
    mbar_init(smem_addr(&cs->r2_empty), kQDrainW);
    for (int r = 0; r < kQRing; ++r) mbar_init(smem_addr(&cs->meta_full[r]), kQSplitW);
    cs->timeout = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(smem_addr(&cs->tmem_slot), 512);

  // ---- D T: column exponents, column scales, then its 8 digit planes
  for (int k = t; k < kQN; k += kQThreads) cs->cs[k] = (k < n) ? a.Tscale[k] : 0;
  for (int j = warp; j < kQN; j += kQThreads / 32) {
    int mx = 1;
    if (j < n)
      for (int k = lane; k < n; k += 32)
        mx = max(mx, oz::align_exp((unsigned long long)__double_as_longlong(a.Tinv[k + (int64_t)j * n])));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) cs->fcol[j] = mx;
  }
  __syncthreads();
  for (int e = t; e < kQN * kQN / 2; e += kQThreads) {
    const int j = e >> 5, k = 2 * (e & 31);
    unsigned long long b[2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
      b[h] = (j < n && k + h < n) ? (unsigned long long)__double_as_longlong(a.Tinv[(k + h) + (int64_t)j * n]) : 0ull;
    const unsigned long long W0 = mag63(b[0], cs->fcol[j], 0) + kBal63, W1 = mag63(b[1], cs->fcol[j], 0) + kBal63;
    const float s0 = (b[0] >> 63) ? -1.0f : 1.0f, s1 = (b[1] >> 63) ? -1.0f : 1.0f;
    const uint32_t off = sw_off(j, k);
#pragma unroll
    for (int d = 0; d < kQDig; ++d)
      *(uint32_t *)(base + kOffB + d * kBPlane + off) = bf2(bdigit(W0, d, s0), bdigit(W1, d, s1));
  }
  fence_async_shared();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = cs->tmem_slot;

  if (warp < kQSplitW) {
    // ---- split: row r of the tile, k in [32 kh, 32 kh + 32)
    const int r = (warp & 3) * 32 + lane, kh = warp >> 2, k0 = 32 * kh;
    constexpr uint32_t idesc = idesc_bf16_f32(128, kQN);
    int issued = 0;
    unsigned long long bv[32];
    auto load = [&](int tile) {
      const int64_t rr = row0 + (int64_t)tile * kQR + r;
      const bool in = rr < row1;
#pragma unroll
      for (int h = 0; h < 32; ++h)
        bv[h] = (in && k0 + h < n) ? (unsigned long long)__double_as_longlong(a.Yin[rr + (int64_t)(k0 + h) * a.ldyin])
                                   : 0ull;
    };
    load(0);
    for (int k = 0; k < ntiles; ++k) {
      const int par = k & 1, slot = k % kQRing;
      // row exponent: this thread's half, then both halves through shared memory
      int mx = kNoExpQ, bd = 0;
#pragma unroll
      for (int h = 0; h < 32; ++h) {
        bd |= (((bv[h] >> 52) & 0x7FF) == 0x7FF);
        mx = max(mx, scaled_exp_q(bv[h], cs->cs[k0 + h]));
      }
      cs->emax[par][kh][r] = mx;
      cs->ebad[par][kh][r] = bd;
      qbar_sync(kBarRowMax, kQSplitW * 32);
      // a wait that gave up anywhere in the last tile is seen by every split
      // warp after the barrier: they leave the loop together (no warp may
      // leave alone, the others would wait at the barrier for it)
      if (cs->timeout) break;
      const int er = max(cs->emax[par][0][r], cs->emax[par][1][r]);
      const int bb = cs->ebad[par][0][r] | cs->ebad[par][1][r];
      if (kh == 0) {
        cs->erow[slot][r] = er;
        cs->rbad[slot][r] = bb;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&cs->meta_full[slot]));
      // the planes are free once the products of tile k - 1 have completed
      if (k >= 1 && !__all_sync(0xffffffffu, mbar_wait(smem_addr(&cs->planes_empty), (k - 1) & 1, kQWaitNs))) {
        cs->timeout = 1;
        continue;  // to the next barrier, where every split warp stops
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        unsigned long long W[8];
        float sg[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          const unsigned long long b = bv[8 * c + h];
          W[h] = mag63(b, er, cs->cs[k0 + 8 * c + h]) + kBal63;
          sg[h] = (b >> 63) ? -1.0f : 1.0f;
        }
        const uint32_t off = sw_off(r, k0 + 8 * c);
        // two digits per iteration: the fully unrolled split and drain
        // overflowed the instruction cache (no-instruction stalls)
#pragma unroll 2
        for (int d = 0; d < kQDig; ++d) {
          uint4 w;
          w.x = bf2(bdigit(W[0], d, sg[0]), bdigit(W[1], d, sg[1]));
          w.y = bf2(bdigit(W[2], d, sg[2]), bdigit(W[3], d, sg[3]));
          w.z = bf2(bdigit(W[4], d, sg[4]), bdigit(W[5], d, sg[5]));
          w.w = bf2(bdigit(W[6], d, sg[6]), bdigit(W[7], d, sg[7]));
          *(uint4 *)(base + kOffA + d * kAPlane + off) = w;
        }
      }
      fence_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&cs->planes_full));
      if (k + 1 < ntiles) load(k + 1);  // in flight while the products run
      if (warp == 0) {
        // ---- MMA issue: round 1 (orders 0..3), round 2 (orders 4..7)
        int ok = 1;
        if (lane == 0) {
          ok = mbar_wait(smem_addr(&cs->planes_full), k & 1, kQWaitNs) &&
               (k < 1 || mbar_wait(smem_addr(&cs->r1_empty), (k - 1) & 1, kQWaitNs));
          if (ok) {
            fence_after_sync();
            // K step by K step, alternating the orders' accumulators (the
            // first pair of each order, at K step 0, overwrites it)
#pragma unroll 1
            for (int ks = 0; ks < 4; ++ks)
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int o = i; o < 4; ++o)
                  mma_ss(tmem + (uint32_t)(o * kQN), sdesc_sw128(sbase + kOffA + i * kAPlane + ks * 32),
                         sdesc_sw128(sbase + kOffB + (o - i) * kBPlane + ks * 32), idesc,
                         (i == 0 && ks == 0) ? 0u : 1u);
            mma_commit(smem_addr(&cs->r1_full));
            ok = (k < 1 || mbar_wait(smem_addr(&cs->r2_empty), (k - 1) & 1, kQWaitNs));
          }
          if (ok) {
            fence_after_sync();
#pragma unroll 1
            for (int ks = 0; ks < 4; ++ks)
#pragma unroll
              for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int o = 4; o < 8; ++o)
                  if (i <= o)
                    mma_ss(tmem + (uint32_t)(256 + (o - 4) * kQN), sdesc_sw128(sbase + kOffA + i * kAPlane + ks * 32),
                           sdesc_sw128(sbase + kOffB + (o - i) * kBPlane + ks * 32), idesc,
                           (i == 0 && ks == 0) ? 0u : 1u);
            mma_commit(smem_addr(&cs->r2_full));
            mma_commit(smem_addr(&cs->planes_empty));
            ++issued;
          }
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) cs->timeout = 1;  // every split warp stops at the next barrier
      }
    }
    if (warp == 0 && lane == 0 && issued > 0 &&
        !mbar_wait(smem_addr(&cs->r2_full), (issued - 1) & 1, kQWaitNs))
      cs->timeout = 1;  // every issued product completes before TMEM is freed
  } else {
    // ---- drain: TMEM lane `row`, columns half * 32 .. + 31
    const int dw = warp - kQSplitW, quad = warp & 3, half = dw >> 2;
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32);
    for (int k = 0; k < ntiles; ++k) {
      const int slot = k % kQRing;
      const bool ready = mbar_wait(smem_addr(&cs->r1_full), k & 1, kQWaitNs) &&
                         mbar_wait(smem_addr(&cs->meta_full[slot]), (k / kQRing) & 1, kQWaitNs);
      if (!__all_sync(0xffffffffu, ready)) {
        cs->timeout = 1;
        break;
      }
      fence_after_sync();
      // round 1: hi = T0 2^24 + T1 2^16 + T2 2^8 + T3
      long long hi[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) hi[c] = 0;
#pragma unroll
      for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int c16 = 0; c16 < 32; c16 += 16) {
          uint32_t x[16];
          tmem_ld16(tl + (uint32_t)(o * kQN + c16), x);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; ++e) hi[c16 + e] += (long long)f2i_q(x[e]) << (8 * (3 - o));
        }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&cs->r1_empty));
      if (!__all_sync(0xffffffffu, mbar_wait(smem_addr(&cs->r2_full), k & 1, kQWaitNs))) {
        cs->timeout = 1;
        break;
      }
      fence_after_sync();
      const int er = cs->erow[slot][row];
      const bool bad = cs->rbad[slot][row] != 0 || cs->timeout != 0;
      const int64_t rr = row0 + (int64_t)k * kQR + row;
      // round 2: lo = T4 2^24 + T5 2^16 + T6 2^8 + T7, sixteen columns at a
      // time; Q_rj = (hi 2^32 + lo) 2^(e_r + f_j - 2114), rounded once
#pragma unroll
      for (int c16 = 0; c16 < 32; c16 += 16) {
        long long lo[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) lo[e] = 0;
#pragma unroll
        for (int o = 4; o < 8; ++o) {
          uint32_t x[16];
          tmem_ld16(tl + (uint32_t)(256 + (o - 4) * kQN + c16), x);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; ++e) lo[e] += (long long)f2i_q(x[e]) << (8 * (7 - o));
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = half * 32 + c16 + e;
          if (rr < row1 && j < n) {
            const double v = bad ? __longlong_as_double(0x7FF8000000000000ll)
                                 : oz::fixed_to_double_bf(hi[c16 + e], lo[e], 32, er + cs->fcol[j] - 2114);
            a.Yout[rr + (int64_t)j * a.ldyout] = v;
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&cs->r2_empty));
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- host side

namespace {

bool sm103_q() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return false;
  }
  int v = cached[dev].load();
  if (v == 0) {
    int ma = 0, mi = 0, optin = 0;
    cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    const bool ok = (ma == 10 && mi == 3) && cudaFuncGetAttributes(&fa, tcgemm64_kernel) == cudaSuccess &&
                    fa.maxThreadsPerBlock >= kQThreads && (size_t)optin >= kQSmem + fa.sharedSizeBytes;
    (void)cudaGetLastError();
    v = ok ? 1 : 2;
    cached[dev].store(v);
  }
  return v == 1;
}

}  // namespace

bool tcgemm_usable(const RowSweep &a) {
  return (a.tc05 & kTc05Solve) && a.q == 0 && a.p >= kTcGemmMinN && a.p <= kQN && a.Tinv != nullptr &&
         a.Tscale != nullptr &&
         a.rows_per_cta % kQR == 0 && sm103_q();
}

int tcgemm_tile_rows() { return kQR; }

int tcgemm_grid(int64_t m) {
  const int64_t tiles = (m + kQR - 1) / kQR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms()));
}

// bf16 digit FLOPs per row: 36 ordered digit pairs, each a full 64 x 64 block
double tcgemm_tc_flops_per_row() { return 2.0 * 36 * kQN * kQN; }

cudaError_t launch_tcgemm(const RowSweep &a, int grid, cudaStream_t s) {
  if (!tcgemm_usable(a)) return cudaErrorInvalidValue;
  static KernelAttr attr;
  set_smem_attr(attr, tcgemm64_kernel, (int)kQSmem, true);
  tcgemm64_kernel<<<grid, kQThreads, kQSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cqr
