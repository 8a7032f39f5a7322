// Building blocks of the tensor-core kernels that do FP64 arithmetic exactly
// on bf16 digits (the Ozaki splitting scheme: Ozaki, Ogita, Oishi, Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012):
// shared-memory staging, ldmatrix / mma.sync wrappers, exact conversions.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>
#include <math.h>

namespace cqr {
namespace oz {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                        uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t &r0, uint32_t &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

// A register-only operation: not volatile, so the compiler may interleave it
// with the fragment loads.
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Asynchronous 8-byte global -> shared copy; src_bytes = 0 zero-fills.
__device__ __forceinline__ void cp_async8(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes));
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// FP32 -> int32 for an integer-valued FP32 (exact: the value is an integer).
__device__ __forceinline__ int f2i(float v) {
  int r;
  asm("cvt.rzi.s32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// Doubles both bf16 halves (exact for the integer digits, |2 d| <= 254).
__device__ __forceinline__ uint32_t bf16x2_twice(uint32_t x) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&x);
  h = __hadd2(h, h);
  return *reinterpret_cast<uint32_t *>(&h);
}

// Biased exponent used for alignment (subnormals and zeros count as 1).
__device__ __forceinline__ int align_exp(unsigned long long b) {
  const int ef = (int)((b >> 52) & 0x7FF);
  return ef ? ef : 1;
}

__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// (hi 2^hs + lo) 2^e rounded to the nearest FP64 (ties to even), on the
// integer pipe in 64-bit words, 0 < hs < 63, |hi| + |lo| 2^-hs < 2^62:
//   v = a 2^hs + r with a = hi + floor(lo / 2^hs), 0 <= r < 2^hs;
//   |v| = A 2^hs + R (for v < 0, A = -a - 1, R = 2^hs - r when r > 0);
//   the top 64 bits of |v| (msb at bit 63) and a sticky bit for the bits of
//   R below them give the 53-bit significand and its rounding.
// Results outside the normal range (rare: entries below 2^-1022 or above
// 2^1023) take the FP64 path, whose ldexp rounds subnormals correctly.
__host__ __device__ __forceinline__ double fixed_to_double(long long hi, long long lo, int hs, int e) {
  const unsigned long long rmask = (1ull << hs) - 1ull;
  const long long a = hi + (lo >> hs);
  const unsigned long long r = (unsigned long long)lo & rmask;
  if (a == 0 && r == 0) return 0.0;
  unsigned long long A, R, sign = 0ull;
  if (a < 0) {
    sign = 0x8000000000000000ull;
    A = (unsigned long long)(-a) - (r ? 1ull : 0ull);
    R = r ? (1ull << hs) - r : 0ull;
  } else {
    A = (unsigned long long)a;
    R = r;
  }
  unsigned long long W;
  bool sticky = false;
  int M;  // |v| in [2^M, 2^(M+1))
  if (A == 0) {
    M = 63 - clz64(R);
    W = R << (63 - M);
  } else {
    const int mA = 63 - clz64(A);
    M = mA + hs;
    W = A << (63 - mA);
    if (M <= 63) {
      W |= R << (63 - M);
    } else {
      const int k = M - 63;  // 0 < k < hs
      W |= R >> k;
      sticky = (R & ((1ull << k) - 1ull)) != 0ull;
    }
  }
  unsigned long long mant = W >> 11;
  const unsigned long long rb = W & 0x7FFull;
  if (rb > 0x400ull || (rb == 0x400ull && (sticky || (mant & 1ull)))) {
    ++mant;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++M;
    }
  }
  const int E = M + e;
  if (E < -1022 || E > 1023) {
    const double vh = ldexp((double)hi, e + hs);
    const double vl = ldexp((double)lo, e);
    return vh + vl;
  }
  unsigned long long bits = sign | ((unsigned long long)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
  double out;
  memcpy(&out, &bits, sizeof(out));
  return out;
}

// fixed_to_double out of line, for the rare results outside the normal range
// (one copy of its code instead of one per inlined call site)
__host__ __device__ __noinline__ inline double fixed_to_double_outlined(long long hi, long long lo, int hs, int e) {
  return fixed_to_double(hi, lo, hs, e);
}

// The same rounding without data-dependent branches (for epilogues that
// round many entries: independent entries overlap their dependency
// chains).  The value v = hi 2^hs + lo is formed exactly as a 128-bit two's
// complement integer T 2^64 + B, its magnitude taken with masks, the
// leading one found with one count-leading-zeros, the 53-bit significand
// rounded to nearest even with a sticky bit for the bits below it, and the
// bits assembled; results outside the normal range take fixed_to_double.
// Same arguments and result as fixed_to_double.
__host__ __device__ __forceinline__ double fixed_to_double_bf(long long hi, long long lo, int hs, int e) {
  // v = hi 2^hs + lo as (T, B): high and low 64-bit words, T signed
  const unsigned long long hb = (unsigned long long)hi << hs;
  const unsigned long long B0 = hb + (unsigned long long)lo;
  const unsigned long long c0 = B0 < hb ? 1ull : 0ull;
  const unsigned long long T0 = (unsigned long long)(hi >> (64 - hs)) + (unsigned long long)(lo >> 63) + c0;
  // |v|: complement both words and add 1 when v < 0
  const unsigned long long neg = (unsigned long long)((long long)T0 >> 63);  // all ones when v < 0
  const unsigned long long B1 = (B0 ^ neg) + (neg & 1ull);
  const unsigned long long T1 = (T0 ^ neg) + ((neg & 1ull) & (B1 == 0ull ? 1ull : 0ull));
  // leading one at bit 127 - lz of the 128-bit magnitude
  const int lzT = clz64(T1), lzB = clz64(B1);
  const int lz = T1 != 0ull ? lzT : 64 + lzB;
  const int sh = lz & 63;
  const unsigned long long Bs = B1 << sh;
  const unsigned long long cross = sh ? (B1 >> (64 - sh)) : 0ull;
  const unsigned long long W = lz >= 64 ? Bs : ((T1 << sh) | cross);  // msb at bit 63
  const unsigned long long rest = lz >= 64 ? 0ull : Bs;               // bits below W
  unsigned long long mant = W >> 11;
  const unsigned long long rb = W & 0x7FFull;
  const bool up = (rb > 0x400ull) || (rb == 0x400ull && (rest != 0ull || (mant & 1ull)));
  mant += up ? 1ull : 0ull;
  const unsigned long long ov = mant >> 53;  // the significand rounded up to 2^53
  mant >>= ov;
  const int E = 127 - lz + (int)ov + e;
  if ((T1 | B1) == 0ull) return 0.0;
  if (E < -1022 || E > 1023) return fixed_to_double_outlined(hi, lo, hs, e);
  const unsigned long long bits =
      (neg & 0x8000000000000000ull) | ((unsigned long long)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
  double out;
  memcpy(&out, &bits, sizeof(out));
  return out;
}

// Rescales an accumulator pair (value = hi * 2^hs u + lo * u) to a unit 2^D
// times larger when a column's running exponent grows by D: the bits that
// leave hi move into lo before lo is shifted, so only bits below the new
// lo unit are dropped.  For D >= 62 the old value lies below 2^-62 of the
// entry's new magnitude and is dropped.
__device__ __forceinline__ void shift_pair(long long &hi, long long &lo, int D, int hs = 28) {
  if (D <= 0) return;
  if (D >= 62) {
    hi = 0;
    lo = 0;
    return;
  }
  const long long q = hi >> D;
  const long long rm = hi - (q << D);  // 0 <= rm < 2^D
  if (D + hs <= 62) lo = (lo + (rm << hs)) >> D;
  else lo = (lo >> D) + (rm >> (D - hs));
  hi = q;
}

}  // namespace oz
}  // namespace cqr
