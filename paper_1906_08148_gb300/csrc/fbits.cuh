// fbits.cuh -- IEEE binary64 -> binary32 rounding on bit patterns.
//
// The tensor-core forms convert every FP64 leaf element to FP32 before
// splitting it into 16-bit terms.  This part issues FP64 instructions at two
// per clock per SM, so the conversion is done with integer operations instead
// (round to nearest, ties to even, from the definition of the two formats),
// with an exact power-of-two scale 2^shift folded into the exponent.
// Host-compilable so that it can be checked against the host's own rounding.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define FBITS_HD __host__ __device__ __forceinline__
#else
#define FBITS_HD static inline
#endif

// Bits of the float nearest to x * 2^shift (x given by its bits b).  Zeros,
// FP64 subnormals and results below the FP32 normal range give a signed zero
// (flush); results above the FP32 range give a signed infinity; NaN stays NaN.
FBITS_HD uint32_t fbits_from_double_rn(uint64_t b, int shift) {
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7FF);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;  // 52 fraction bits
  if (E == 0x7FF) return sign | 0x7F800000u | (m ? 0x00400000u : 0u);
  if (E == 0) return sign;
  const int e = E - 1023 + shift;  // unbiased exponent of the result
  if (e < -126) return sign;
  if (e > 127) return sign | 0x7F800000u;
  uint32_t f = ((uint32_t)(e + 127) << 23) | (uint32_t)(m >> 29);
  const uint32_t rest = (uint32_t)(m & 0x1FFFFFFFu);  // the 29 bits rounded away
  if (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ++f;  // a carry moves into the exponent
  return sign | f;
}

// Exponent e of a leaf's scale 2^e such that max|a| 2^e lies in [2^14, 2^15),
// from the largest |a| as bits (0: an all-zero leaf, e = 0), clamped to
// [-120, 120]; a subnormal maximum takes the clamp.
FBITS_HD int fp16_leaf_shift(uint64_t max_abs_bits) {
  if (max_abs_bits == 0) return 0;
  const int E = (int)(max_abs_bits >> 52);
  int e = E == 0 ? 120 : 1037 - E;  // max in [2^(E-1023), 2^(E-1022))
  return e > 120 ? 120 : (e < -120 ? -120 : e);
}
