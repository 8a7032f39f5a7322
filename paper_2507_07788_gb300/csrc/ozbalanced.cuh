// Balanced base-256 digits of a 56-bit magnitude (the digit cache of a
// basis): an element x with reference exponent E (E >= its biased exponent,
// zeros and subnormals counting as 1) is
//   x = sign * V * 2^(E - 1078),  V = (M << 3) >> (E - e_x) < 2^56
// (M the 53-bit significand with its implicit bit; bits below 2^(E - 1078)
// are truncated), and V = sum_{i=0..6} D_i 2^(8 (6 - i)) with D_0 in [0, 256]
// and D_i in [-128, 127]: add 128 to each of the six low bytes of V (W =
// V + kCBal), then D_0 = W >> 48 and D_i = byte (6 - i) of W minus 128.
// Each signed digit is an integer of magnitude <= 256, exact in bf16.
// Host-callable, so the representation is tested on the CPU.
#pragma once

#include <stdint.h>
#include <string.h>

namespace cqr {

constexpr unsigned long long kCBal = 0x0000808080808080ull;

// W = V + kCBal of the element with bit pattern b against exponent E.
__host__ __device__ __forceinline__ unsigned long long cwords(unsigned long long b, int E) {
  const int ef = (int)((b >> 52) & 0x7FF);
  unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  if (ef) M |= 0x10000000000000ull;
  if (ef == 0x7FF) M = 0;
  const int sh = E - (ef ? ef : 1);
  return ((sh >= 56 || sh < 0) ? 0ull : ((M << 3) >> sh)) + kCBal;
}

__host__ __device__ __forceinline__ float bits_to_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __int_as_float((int)u);
#else
  float f;
  memcpy(&f, &u, sizeof(f));
  return f;
#endif
}

// Digit i of W with the element's sign s (+-1) as an exact FP32 integer: the
// digit byte is placed in 2^23 + x (a shift for i = 0, a byte permute
// otherwise) and s (2^23 + x) - s (2^23 + b) = s (x - b) in one FMA.
__host__ __device__ __forceinline__ float cdigit(unsigned long long W, int i, float s) {
  if (i == 0) return fmaf(bits_to_float(0x4B000000u | (uint32_t)(W >> 48)), s, -s * 8388608.0f);
  const int b = 6 - i;
  const uint32_t word = (b >= 4) ? (uint32_t)(W >> 32) : (uint32_t)W;
#ifdef __CUDA_ARCH__
  const uint32_t xb = __byte_perm(word, 0x4B000000u, 0x7440u | (uint32_t)(b & 3));
#else
  const uint32_t xb = 0x4B000000u | ((word >> (8 * (b & 3))) & 0xFFu);
#endif
  return fmaf(bits_to_float(xb), s, -s * 8388736.0f);
}

}  // namespace cqr
