// Cross Gramian of the update, C = [Q_in Y]^T Y (Alg. 2 and
// 15-16: B~ = Q_in^T Y and Y^T Y in one read of [Q_in Y]), on the tensor cores
// with exact digit arithmetic (the Ozaki splitting scheme), for the
// Cholesky-QR update of tall bases.
//
// Representation (per 64-row tile, per column c of Z = [Q_in Y] and j of Y):
//   each column keeps the running maximum E of its biased exponents over the
//   rows the CTA has seen, and every element is x = sign V 2^(E - 1078),
//   V = sum_{t=1..8} d_t 2^(56 - 7 t), 8 digits in [0, 127] (exact in bf16).
// Products: z_c y_j = 2^(E_c + E_j - 2156) sum_{s,t} d_s(z_c) d_t(y_j)
//   2^(112 - 7(s+t)); all ordered digit pairs with s + t <= 9 are kept (Z and
//   Y are different operands, so there is no symmetric half).
// Exactness: an order d has at most 8 pairs, |sum over a tile| <= 8 * 64 *
//   127^2 < 2^24, exact in one FP32 mma.sync accumulator; orders are combined
//   exactly in int32 pairs and two int64 words per entry (orders 2..5, 6..9),
//   rescaled by exact shifts when a column's exponent grows, and each entry
//   of a CTA's partial is rounded to FP64 once.
// Work split: CTA (g, b) takes the rows of row group g and the 64 columns
//   [64 b, 64 b + 64) of Z against all of Y; it writes rows 64 b .. of the
//   group's partial ((q + p) x p, ld q + p).  A fixed-order sum of the row
//   groups' partials gives C.
// Non-finite inputs make every partial of the CTA NaN (the control kernel
// then reports a breakdown, as the FP64 path does).
#include <algorithm>

#include "cqr_internal.cuh"
#include "ozdigits.cuh"

namespace cqr {

using namespace oz;

namespace {

constexpr int kXTR = 64;          // tile rows
constexpr int kXZ = 64;           // Z columns per CTA
constexpr int kXLDK = kXTR + 8;   // bf16 stride of a digit-plane column
constexpr int kXThreads = 256;    // 8 warps, one CTA per SM
constexpr int kXWarps = kXThreads / 32;
constexpr int kXDigits = 8;

template <int NY>  // NY in {32, 64}: the padded width of Y
struct XGeom {
  static constexpr int JB = 32;
  static constexpr int NJ = NY / JB;
  static constexpr int strips = (kXZ / 16) * NJ;
  static constexpr int groups = (strips >= 8) ? 1 : 2;  // even / odd orders
};

template <int NY>
constexpr size_t xgram_smem() {
  return sizeof(double) * (size_t)(kXZ + NY) * kXTR                    // FP64 tiles of Z and Y
         + sizeof(uint16_t) * (size_t)kXDigits * (kXZ + NY) * kXLDK    // digit planes
         + sizeof(int) * (size_t)(2 * (kXZ + NY) + 4);
}

}  // namespace

template <int NY>
__global__ void __launch_bounds__(kXThreads, 1) ozxgram_kernel(RowSweep a, int nzb) {
  if (a.st != nullptr && a.st->done) return;
  using G = XGeom<NY>;
  constexpr int JB = G::JB, NTILE = JB / 8, SLOTS = 4 * NTILE, NC = kXZ + NY;
  extern __shared__ __align__(16) unsigned char smem[];
  double *tile = (double *)smem;                                        // [NC cols][64 rows]
  uint16_t *planes = (uint16_t *)(tile + (size_t)NC * kXTR);            // [8][NC][kXLDK]
  int *Erun = (int *)(planes + (size_t)kXDigits * NC * kXLDK);          // [NC]
  int *Edel = Erun + NC;                                                // [NC]
  int *flag = Edel + NC;                                                // [1]

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int q = a.q, p = a.p, nz = q + p;
  const int zb = (int)(blockIdx.x % nzb);
  const int64_t grp_id = blockIdx.x / nzb;
  const int64_t row0 = grp_id * a.rows_per_cta;
  const int64_t row1 = min(a.m, row0 + a.rows_per_cta);

  for (int c = t; c < NC; c += kXThreads) {
    Erun[c] = 1;
    Edel[c] = 0;
  }
  if (t == 0) *flag = 0;
  {
    const int zc0 = min(kXZ, max(0, nz - kXZ * zb));  // live Z columns of this block
    for (int e = t; e < NC * kXTR; e += kXThreads) {
      const int c = e / kXTR;
      const bool dead = (c < kXZ) ? (c >= zc0) : (c - kXZ >= p);
      if (dead) tile[e] = 0.0;
    }
    for (int e = t; e < kXDigits * NC * (kXLDK / 2); e += kXThreads) {
      const int c = (e / (kXLDK / 2)) % NC;
      const bool dead = (c < kXZ) ? (c >= zc0) : (c - kXZ >= p);
      if (dead) ((uint32_t *)planes)[e] = 0u;
    }
  }
  long long acc_hi[SLOTS], acc_lo[SLOTS];
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    acc_hi[k] = 0;
    acc_lo[k] = 0;
  }
  __syncthreads();

  // local column c < 64: Z column 64 zb + c (a basis column below q, a
  // column of Y from q on); c >= 64: column c - 64 of Y
  auto src_col = [&](int c, int64_t r) -> const double * {
    const int zc = (c < kXZ) ? kXZ * zb + c : q + (c - kXZ);
    if (c < kXZ && zc >= nz) return nullptr;
    if (c >= kXZ && c - kXZ >= p) return nullptr;
    return (zc < q) ? a.Qin + r + (int64_t)zc * a.ldqin : a.Yin + r + (int64_t)(zc - q) * a.ldyin;
  };

  // columns that hold data (the rest of the NC slots stay zero: no staging,
  // exponent tracking or digit split for them)
  const int zcols = min(kXZ, nz - kXZ * zb);
  auto live = [&](int c) { return (c < kXZ) ? (c < zcols) : (c - kXZ < p); };
  const int strip = warp / G::groups, grp = warp % G::groups;
  const int ib = strip / G::NJ, jb = strip % G::NJ;
  const int i0 = ib * 16, j0 = jb * JB;  // Z-column strip, Y-column strip

  for (int64_t r0 = row0; r0 < row1; r0 += kXTR) {
    const int nr = (int)min((int64_t)kXTR, row1 - r0);
    // ---- stage Z's 64 columns and Y (column-major, zero padded)
    for (int e = t; e < kXTR * NC; e += kXThreads) {
      const int i = e % kXTR, c = e / kXTR;
      if (!live(c)) continue;  // zero-filled once, before the first tile
      const double *s = (i < nr) ? src_col(c, r0 + i) : nullptr;
      cp_async8(tile + c * kXTR + i, s ? s : a.Yin, s ? 8 : 0);
    }
    cp_async_wait_all();
    __syncthreads();
    // ---- column exponents: running maximum, growth since the last tile
    for (int c = warp; c < NC; c += kXWarps) {
      if (!live(c)) continue;
      // biased exponents from the high words; 0x7FF (NaN / Inf) is the
      // largest, so it also flags a non-finite entry
      const uint32_t *hw = (const uint32_t *)(tile + c * kXTR) + 1;
      int mx = 1;
      for (int i = lane; i < kXTR; i += 32) mx = max(mx, (int)((hw[2 * i] >> 20) & 0x7FF));
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) {
        const int old = Erun[c];
        const int nw = max(old, mx);
        Edel[c] = nw - old;
        Erun[c] = nw;
        if (mx == 0x7FF) *flag = 1;
      }
    }
    __syncthreads();
    // ---- 8 digit planes per column (two rows per thread step)
    for (int e = t; e < (kXTR / 2) * NC; e += kXThreads) {
      const int i = 2 * (e % (kXTR / 2)), c = e / (kXTR / 2);
      if (!live(c)) continue;  // its digit planes were zeroed before the first tile
      const int Ec = Erun[c];
      unsigned long long V[2];
      uint32_t sgnmask = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(tile[c * kXTR + i + h]);
        const int ef = (int)((b >> 52) & 0x7FF);
        unsigned long long M = b & 0xFFFFFFFFFFFFFull;
        if (ef) M |= 0x10000000000000ull;
        if (ef == 0x7FF) M = 0;
        const int sh = Ec - (ef ? ef : 1);
        V[h] = (sh >= 56) ? 0ull : ((M << 3) >> sh);
        sgnmask |= (uint32_t)(b >> 63) << (15 + 16 * h);
      }
#pragma unroll
      for (int d = 0; d < kXDigits; ++d) {
        const float f0 = __int_as_float(0x4B000000 | (int)((V[0] >> (49 - 7 * d)) & 127u)) - 8388608.0f;
        const float f1 = __int_as_float(0x4B000000 | (int)((V[1] >> (49 - 7 * d)) & 127u)) - 8388608.0f;
        const __nv_bfloat162 pr = __floats2bfloat162_rn(f0, f1);
        *(uint32_t *)(planes + ((size_t)d * NC + c) * kXLDK + i) = *(const uint32_t *)&pr | sgnmask;
      }
    }
    __syncthreads();
    // ---- tensor-core products (A = Z digits, B = Y digits), drained
    {
      // rescale where a column exponent grew
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int zi = i0 + (lane >> 2) + ((r >> 1) << 3);
          const int yj = j0 + nt * 8 + 2 * (lane & 3) + (r & 1);
          shift_pair(acc_hi[nt * 4 + r], acc_lo[nt * 4 + r], Edel[zi] + Edel[kXZ + yj]);
        }
      int tv[NTILE][4];
#pragma unroll
      for (int d = 2; d <= 9; ++d) {
        if (G::groups == 2 && (d & 1) != grp) continue;
        float c[NTILE][4];
#pragma unroll
        for (int nt = 0; nt < NTILE; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll 1
        for (int s = (d > kXDigits + 1) ? d - kXDigits : 1; s < d && s <= kXDigits; ++s) {
          const int tt = d - s;
          const uint16_t *As = planes + ((size_t)(s - 1) * NC + i0) * kXLDK;
          const uint16_t *Bt = planes + ((size_t)(tt - 1) * NC + kXZ + j0) * kXLDK;
#pragma unroll 2
          for (int ks = 0; ks < kXTR; ks += 16) {
            uint32_t a0, a1, a2, a3;
            {
              const int mi = lane >> 3, rr = lane & 7;
              const uint16_t *pa = As + ((mi & 1) * 8 + rr) * kXLDK + ks + (mi >> 1) * 8;
              ldsm_x4(smem_u32(pa), a0, a1, a2, a3);
            }
#pragma unroll
            for (int nt = 0; nt < NTILE; nt += 2) {
              uint32_t b0, b1, b2, b3;
              const int mi = lane >> 3, rr = lane & 7;
              const uint16_t *pb = Bt + ((nt + (mi >> 1)) * 8 + rr) * kXLDK + ks + (mi & 1) * 8;
              ldsm_x4(smem_u32(pb), b0, b1, b2, b3);
              mma_bf16(c[nt], a0, a1, a2, a3, b0, b1);
              mma_bf16(c[nt + 1], a0, a1, a2, a3, b2, b3);
            }
          }
        }
        // drain: hi word = orders 2..5 (weight 2^(7 (5 - d))), lo word =
        // orders 6..9 (2^(7 (9 - d))); with one group the pairs (2,3),
        // (4,5), (6,7), (8,9) are first combined in int32 as T_d 2^7 + T_d+1
        const bool hi = d <= 5;
        if (G::groups == 1 && (d & 1) == 0) {
#pragma unroll
          for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) tv[nt][r] = f2i(c[nt][r]);
        } else {
          const int shl = hi ? 7 * (5 - d) : 7 * (9 - d);
#pragma unroll
          for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int v = f2i(c[nt][r]);
              const long long w = (G::groups == 1) ? (long long)(tv[nt][r] * 128 + v) : (long long)v;
              const int k = nt * 4 + r;
              if (hi) acc_hi[k] += w << shl;
              else acc_lo[k] += w << shl;
            }
        }
      }
    }
    __syncthreads();
  }

  // ---- combine the order groups exactly, round to FP64 once per entry
  long long *ohi = (long long *)planes;  // [NY][kXZ]
  long long *olo = ohi + (size_t)NY * kXZ;
  for (int e = t; e < NY * kXZ; e += kXThreads) {
    ohi[e] = 0;
    olo[e] = 0;
  }
  __syncthreads();
  for (int g = 0; g < G::groups; ++g) {
    if (grp == g) {
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int zi = i0 + (lane >> 2) + ((r >> 1) << 3);
          const int yj = j0 + nt * 8 + 2 * (lane & 3) + (r & 1);
          ohi[zi + yj * kXZ] += acc_hi[nt * 4 + r];
          olo[zi + yj * kXZ] += acc_lo[nt * 4 + r];
        }
    }
    __syncthreads();
  }
  const bool bad = *flag != 0;
  double *P = a.partials + grp_id * (int64_t)nz * p;
  for (int e = t; e < kXZ * p; e += kXThreads) {
    const int zi = e % kXZ, j = e / kXZ, zc = kXZ * zb + zi;
    if (zc >= nz) continue;
    // C_cj = (hi 2^28 + lo) 2^(E_c + E_j - 2107)
    const double v = bad ? __longlong_as_double(0x7FF8000000000000ll)
                         : fixed_to_double(ohi[zi + j * kXZ], olo[zi + j * kXZ], 28,
                                           Erun[zi] + Erun[kXZ + j] - 2107);
    P[zc + (int64_t)j * nz] = v;
  }
}

template <int NY>
static cudaError_t launch_x(const RowSweep &a, int groups, int nzb, cudaStream_t s) {
  constexpr size_t smem = xgram_smem<NY>();
  static KernelAttr attr;
  set_smem_attr(attr, ozxgram_kernel<NY>, (int)smem, false);
  ozxgram_kernel<NY><<<groups * nzb, kXThreads, smem, s>>>(a, nzb);
  return cudaGetLastError();
}

int ozxgram_zblocks(int q, int p) { return (q + p + kXZ - 1) / kXZ; }

// Row groups for m rows: all CTAs (row groups x Z blocks) about one per SM.
int ozxgram_grid(int64_t m, int q, int p) {
  const int64_t tiles = (m + kXTR - 1) / kXTR;
  const int nzb = ozxgram_zblocks(q, p);
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, std::max<int64_t>(1, num_sms() / nzb)));
}

int ozxgram_tile_rows() { return kXTR; }

// C partials for kOzUpdMinP <= p <= 64 (a.m, a.q, a.p, a.Qin, a.ldqin,
// a.Yin, a.ldyin, a.partials, a.rows_per_cta, a.st); `groups` row groups.
cudaError_t launch_ozxgram(const RowSweep &a, int groups, cudaStream_t s) {
  const int nzb = ozxgram_zblocks(a.q, a.p);
  if (a.p < kOzUpdMinP) return cudaErrorInvalidValue;
  if (a.p <= 32) return launch_x<32>(a, groups, nzb, s);
  if (a.p <= 64) return launch_x<64>(a, groups, nzb, s);
  return cudaErrorInvalidValue;
}

// C = sum of the row groups' partials in a fixed order (dense (q + p) x p).
__global__ void reduce_dense_kernel(const double *partials, int G, int64_t E, double *C,
                                    const DevState *st) {
  if (st != nullptr && st->done) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += partials[(int64_t)g * E + e];
  C[e] = s;
}

cudaError_t launch_reduce_dense(const double *partials, int G, int64_t E, double *C, const DevState *st,
                                cudaStream_t s) {
  reduce_dense_kernel<<<(unsigned)((E + 127) / 128), 128, 0, s>>>(partials, G, E, C, st);
  return cudaGetLastError();
}


}  // namespace cqr
