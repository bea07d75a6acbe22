// convert.cuh -- exact FP32 -> FP64 conversion on bit patterns.
//
// Every FP32 value is exactly representable in FP64; the conversion only
// re-biases the exponent (127 -> 1023), moves the 23 fraction bits to the top
// of the 52, normalises subnormal inputs (an FP32 subnormal m 2^-149 is a
// normal FP64 number) and keeps zeros, infinities and NaNs (payload moved the
// same way).  Done in the integer pipe because this part issues two FP64
// instructions per clock per SM.  Host-compilable so that it can be checked
// against the compiler's conversion for every class of input.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define CONV_HD __host__ __device__ __forceinline__
#else
#define CONV_HD static inline
#endif

CONV_HD int conv_clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __clz(x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

CONV_HD uint64_t f32_to_f64_bits(uint32_t b) {
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  if (e == 0xffu) return sign | (0x7ffull << 52) | ((uint64_t)m << 29);
  if (e != 0u) return sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  if (m == 0u) return sign;
  const int sh = conv_clz32(m) - 8;  // moves the leading bit to position 23
  return sign | ((uint64_t)(897 - sh) << 52) | ((uint64_t)((m << sh) & 0x7fffffu) << 29);
}
