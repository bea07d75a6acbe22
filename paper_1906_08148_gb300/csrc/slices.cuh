// slices.cuh -- error-free BF16 slices of an FP64 operand (the BF16 split
// forms of the tensor-core leaf GEMM), on bit patterns.
//
// The element x of one line of a leaf (a row of an A leaf, a column of a B
// leaf: the elements that share an output row or column) is written, after a
// per-leaf power-of-two scale 2^f, as S digits on a grid fixed by the largest
// element of its line:
//     x 2^f = sum_{s < S} d_s 2^(e - 8 - 9 s) + r,
//     e = (biased exponent of the line's largest |x|) - 1022 + f, so every
//         |x 2^f| of the line is < 2^e,
//     |d_0| <= 256, -256 <= d_s <= 255 for s >= 1 (balanced base-512 digits),
//     |r| <= 2^(e - 9 S)  (half a unit of the last digit).
// Each digit times its power of two has at most 8 significant bits, so it is
// a BF16 value.  Because every slice of a line sits on the same grid, the
// product of slice s of an A row and slice t of a B column is an integer
// multiple of 2^(eA + eB - 16 - 9 (s + t)) of magnitude <= 2^16 units, and a
// K = 64 sum of such products for one s + t (at most two pairs) is an integer
// of at most 2^23 units: exact in the FP32 accumulator of the tensor core.
// This is the error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer.
// Algorithms 59, 2012) with per-row/column alignment, done here with integer
// arithmetic because this part issues FP64 instructions at two per clock per
// SM.  Host-compilable so it can be checked against exact arithmetic.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define SLICE_HD __host__ __device__ __forceinline__
#else
#define SLICE_HD static inline
#endif

// Biased binary64 exponent of x given its bits; zeros and subnormals give 0
// and count as zero in the split (they are below 2^-1022).
SLICE_HD int slice_biased_exp(uint64_t b) { return (int)((b >> 52) & 0x7FF); }

// Per-leaf scale exponent f from the largest biased exponent in the leaf:
// max|x| 2^f in [1, 2), clamped to [-120, 120]; 0 for an all-zero leaf.
SLICE_HD int slice_leaf_shift(int emax_biased) {
  if (emax_biased == 0) return 0;
  const int f = 1023 - emax_biased;
  return f > 120 ? 120 : (f < -120 ? -120 : f);
}

// Line exponent e (see above) from the line's largest biased exponent and f.
SLICE_HD int slice_line_exp(int emax_line_biased, int f) { return emax_line_biased - 1022 + f; }

// The S digits of x (bits b) on the grid of a line whose largest biased
// exponent is emax_line (>= x's own).  x is rounded to the last digit's unit
// (half away from zero), then split into balanced base-512 digits from the
// last one up, so the leading digit takes what is left (|d_0| <= 256).
template <int S>
SLICE_HD void slice_digits(uint64_t b, int emax_line, int32_t* d) {
  static_assert(S >= 1 && S <= 6, "the shift below needs 9 S <= 54");
  const int E = slice_biased_exp(b);
  int64_t M = 0;
  if (E != 0) {
    const int sh = 54 + emax_line - E - 9 * S;  // >= 0: E <= emax_line, 9 S <= 54
    if (sh <= 54) {
      const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const uint64_t mag = sh == 0 ? m : ((m + (1ull << (sh - 1))) >> sh);
      M = (b >> 63) ? -(int64_t)mag : (int64_t)mag;
    }
  }
  for (int s = S - 1; s >= 1; --s) {
    int32_t t = (int32_t)(M & 511);
    if (t >= 256) t -= 512;
    d[s] = t;
    M = (M - t) >> 9;  // exact: M - t is a multiple of 512 (arithmetic shift of a two's-complement multiple)
  }
  d[0] = (int32_t)M;
}

SLICE_HD uint32_t slice_f32_bits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

SLICE_HD float slice_f32_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}

// BF16 bits of d 2^p (|d| <= 256, so at most 8 significant bits: exact).
// A digit whose unit 2^p lies below the FP32 normal range (p < -126) is
// dropped: with the leaf scaled to max|x| in [1, 2) it is below 2^-118.
// The integer d becomes a float without a conversion instruction: 1.5 2^23 + d
// is a float whose low mantissa bits are d (|d| < 2^22), and subtracting
// 1.5 2^23 leaves d exactly; scaling by 2^p is exact too.
SLICE_HD uint16_t slice_bf16_bits(int32_t d, int p) {
  if (p < -126) return 0;
  const float f = slice_f32_from_bits(0x4B400000u + (uint32_t)d) - 12582912.0f;
  const float v = f * slice_f32_from_bits((uint32_t)(p + 127) << 23);
  return (uint16_t)(slice_f32_bits(v) >> 16);
}
