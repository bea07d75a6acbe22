// screen.cuh -- the norm test ||A_ik|| ||B_kj|| >= tau of Algorithm 1 (the
// product rounded to FP64, as the oracle computes it), screened without FP64
// arithmetic.  This part issues two FP64 operations per clock per SM, so the
// task-list builder first decides with integer exponents and an FP32 product
// of leading mantissa bits; only pairs the screen cannot decide take the FP64
// product.  With |A| = fa 2^ea, |B| = fb 2^eb, tau = ft 2^et (f in [1, 2),
// e unbiased) and E = ea + eb - et:
//   E >= 2:  p >= 2^(et+2) > tau, kept;
//   E <= -2: the exact product is at most (1 - 2^-53)^2 2^et, whose FP64
//            rounding stays below 2^et <= tau, skipped;
//   |E| <= 1: m = fl32(fa' fb') of the mantissas truncated to 13 bits lies
//            within (1 - 2^-24, 1 + 2^-11.9) times fa fb, so m above hi[E+1] =
//            ft (1 + 2^-10) 2^-E (rounded up to FP32) keeps and m below
//            lo[E+1] = ft (1 - 2^-10) 2^-E (rounded down) skips; the FP64
//            rounding of p is far inside these margins;
//   a zero or subnormal norm, or tau zero or subnormal: undecided.
// A norm is packed into a 24-bit key: its biased exponent field in the top
// 11 bits, the leading 13 mantissa bits below; 0xFFFFFF (an exponent field no
// finite norm has) marks a null child.
// Host-compilable so that the screen can be checked against FP64 products.
// (Short keys keep a node's four children and their keys in one 16-byte record.)
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cmath>

#if defined(__CUDACC__)
#define SCREEN_HD __host__ __device__ __forceinline__
#else
#define SCREEN_HD static inline
#endif

struct TauScreen {
  int K;            // biased field of tau + 1023: E = eA + eB - K from biased fields
  float hi[3], lo[3];
  int exact_only;   // tau zero or subnormal
};

constexpr uint32_t kNullKey = 0xFFFFFFu;

// The 24-bit key of a norm (non-negative finite double).
SCREEN_HD uint32_t pack_norm(double x) {
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return (uint32_t)((b >> 52) & 0x7ff) << 13 | (uint32_t)((b >> 39) & 0x1fff);
}

// 1: kept, 0: skipped, -1: undecided (take the FP64 product).
SCREEN_HD int screen_decide(uint32_t ka, uint32_t kb, const TauScreen& sc) {
  const int ea = (int)(ka >> 13), eb = (int)(kb >> 13);
  if (sc.exact_only || ea == 0 || eb == 0) return -1;
  const int E = ea + eb - sc.K;
  if (E >= 2) return 1;
  if (E <= -2) return 0;
  const uint32_t fa = 0x3f800000u | ((ka & 0x1fffu) << 10), fb = 0x3f800000u | ((kb & 0x1fffu) << 10);
  float ma, mb;
  memcpy(&ma, &fa, sizeof ma);
  memcpy(&mb, &fb, sizeof mb);
  const float mp = ma * mb;  // one FP32 rounding (no contraction: a plain product)
  const float hi = E == -1 ? sc.hi[0] : (E == 0 ? sc.hi[1] : sc.hi[2]);
  const float lo = E == -1 ? sc.lo[0] : (E == 0 ? sc.lo[1] : sc.lo[2]);
  if (mp > hi) return 1;
  if (mp < lo) return 0;
  return -1;
}

// Thresholds for tau (host side), rounded outwards to FP32.
static inline TauScreen make_screen(double tau) {
  TauScreen sc;
  memset(&sc, 0, sizeof sc);
  uint64_t b;
  memcpy(&b, &tau, sizeof b);
  const int et = (int)((b >> 52) & 0x7ff);
  sc.K = et + 1023;
  sc.exact_only = (et == 0);
  int e2 = 0;
  const double ft = et ? 2.0 * std::frexp(tau, &e2) : 1.0;
  for (int i = 0; i < 3; ++i) {
    const int E = i - 1;
    const double h = std::ldexp(ft * (1.0 + std::ldexp(1.0, -10)), -E);
    const double l = std::ldexp(ft * (1.0 - std::ldexp(1.0, -10)), -E);
    float hf = (float)h, lf = (float)l;
    if ((double)hf < h) hf = std::nextafter(hf, INFINITY);
    if ((double)lf > l) lf = std::nextafter(lf, -INFINITY);
    sc.hi[i] = hf;
    sc.lo[i] = lf;
  }
  return sc;
}
