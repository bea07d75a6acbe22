/*
 * decaygen.h -- seeded synthetic matrices with exponential decay.
 *
 * This header is the ONE piece of code shared by the CPU oracle and the CUDA
 * library: it only draws inputs and holds none of the multiplication method's
 * arithmetic (no norms, no thresholds, no products).
 *
 * Element rule (Definition 1 of the paper, |a_ij| <= c exp(-alpha d(i,j))):
 *     a_ij = c * u_ij * exp(-alpha * d(i,j)),   set to 0 when |a_ij| < cutoff
 * or, with law = SYNTH_LAW_ALGEBRAIC (the algebraic decay Section 1 mentions
 * beside the exponential one), alpha an integer p >= 1:
 *     a_ij = c * u_ij / (1 + d(i,j))^p
 * with u_ij uniform in [-1, 1) and symmetric in (i, j):
 *     u_ij = 2 * (h >> 11) * 2^-53 - 1,   h = SplitMix64 output number
 *     (min(i,j) << 32 | max(i,j)) of the stream seeded with `seed`
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014).  The matrix is therefore symmetric; two seeds give A != B.
 *
 * Distance functions (Section 3, pseudo-metrics on the index set):
 *   SYNTH_KIND_1D : d(i,j) = |i - j|          (the paper's model problem, Sec. 5.3)
 *   SYNTH_KIND_3D : index i sits at lattice point deinterleave3(i) (bit b of x,
 *                   y, z is bit 3b, 3b+1, 3b+2 of i: Morton order with x first),
 *                   d = Euclidean distance between the points (unit spacing).
 *                   The first n indices of this order form a 2^a x 2^b x 2^c
 *                   box whenever n is a power of two (e.g. 65536 -> 64x32x32).
 *
 * Bit-identical on host and device: every floating-point step is a single
 * IEEE operation in round-to-nearest (explicit _rn intrinsics on the device,
 * -ffp-contract=off on the host), sqrt is correctly rounded on both, and the
 * exponential below is our own, so the same (seed, i, j) gives the same bits.
 */
#ifndef SYNTH_DECAYGEN_H
#define SYNTH_DECAYGEN_H
#include <stdint.h>

#ifdef __CUDACC__
#define SYNTH_HD __host__ __device__ __forceinline__
#else
#define SYNTH_HD static inline
#endif

#if defined(__CUDA_ARCH__)
#define SYNTH_MUL(a, b) __dmul_rn((a), (b))
#define SYNTH_ADD(a, b) __dadd_rn((a), (b))
#define SYNTH_SUB(a, b) __dsub_rn((a), (b))
#define SYNTH_SQRT(a) __dsqrt_rn(a)
#define SYNTH_DIV(a, b) __ddiv_rn((a), (b))
#else
#include <math.h>
#define SYNTH_MUL(a, b) ((a) * (b))
#define SYNTH_ADD(a, b) ((a) + (b))
#define SYNTH_SUB(a, b) ((a) - (b))
#define SYNTH_SQRT(a) sqrt(a)
#define SYNTH_DIV(a, b) ((a) / (b))
#endif

enum { SYNTH_KIND_1D = 0, SYNTH_KIND_3D = 1 };
enum { SYNTH_LAW_EXPONENTIAL = 0, SYNTH_LAW_ALGEBRAIC = 1 };

typedef struct synth_params {
  int64_t n;       /* matrix size */
  int32_t kind;    /* SYNTH_KIND_1D or SYNTH_KIND_3D */
  int32_t law;     /* SYNTH_LAW_EXPONENTIAL or SYNTH_LAW_ALGEBRAIC */
  double alpha;    /* decay rate (exponential) or integer power p (algebraic) */
  double c;        /* decay constant (c = 1 in the paper) */
  double cutoff;   /* |a| < cutoff -> 0 (1e-16 in the paper's model problem) */
  uint64_t seed;
} synth_params;

/* SplitMix64: output number `counter` of the stream started at `seed`. */
SYNTH_HD uint64_t synth_splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* u in [-1, 1), exact: a 53-bit integer times 2^-52, minus 1. */
SYNTH_HD double synth_uniform(uint64_t seed, int64_t i, int64_t j) {
  uint64_t lo = (uint64_t)(i < j ? i : j), hi = (uint64_t)(i < j ? j : i);
  uint64_t h = synth_splitmix64(seed, (lo << 32) | hi);
  return SYNTH_SUB(SYNTH_MUL((double)(h >> 11), 0x1.0p-52), 1.0);
}

/* exp(x) for x <= 0.  Cody-Waite reduction x = k ln2 + r with ln2 split as
 * LN2_HI (ln2 rounded to 32 fractional bits, so k*LN2_HI is exact) plus
 * LN2_LO; e^r from its Taylor series to degree 14 (|r| <= 0.35, remainder
 * below 2^-60) in Horner form; 2^k built from its exponent bits.  Accurate to
 * a few ulp; its job is to be reproducible, not to be the fastest exp. */
#define SYNTH_LN2_HI 0x1.62e42ff000000p-1
#define SYNTH_LN2_LO (-0x1.718432a1b0e26p-35)
#define SYNTH_INV_LN2 0x1.71547652b82fep+0
SYNTH_HD double synth_exp_nonpos(double x) {
  if (!(x > -700.0)) return 0.0;
  if (x > 0.0) x = 0.0;
  double t = SYNTH_ADD(SYNTH_MUL(x, SYNTH_INV_LN2), 0.5);
  double kd = (double)(int64_t)t; /* trunc toward zero */
  if (kd > t) kd = SYNTH_SUB(kd, 1.0); /* -> floor(t) */
  double r = SYNTH_SUB(SYNTH_SUB(x, SYNTH_MUL(kd, SYNTH_LN2_HI)), SYNTH_MUL(kd, SYNTH_LN2_LO));
  /* Horner: p = 1 + r(1 + r/2(1 + r/3(... (1 + r/14)))) written with 1/k! */
  const double inv_fact[15] = {1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0,
                               1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0,
                               1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0,
                               1.0 / 87178291200.0};
  double p = inv_fact[14];
  for (int m = 13; m >= 0; --m) p = SYNTH_ADD(SYNTH_MUL(p, r), inv_fact[m]);
  int64_t k = (int64_t)kd; /* in [-1010, 0] */
  union { uint64_t u; double d; } s;
  s.u = (uint64_t)(k + 1023) << 52;
  return SYNTH_MUL(p, s.d);
}

/* 1 / (1 + d)^p for integer p >= 1 (p < 1 taken as 1): p - 1 multiplications
 * and one division, each correctly rounded, so host and device agree. */
SYNTH_HD double synth_algebraic(double d, double p) {
  const double x = SYNTH_ADD(1.0, d);
  int k = (int)p;
  if (k < 1) k = 1;
  double pw = x;
  for (int i = 1; i < k; ++i) pw = SYNTH_MUL(pw, x);
  return SYNTH_DIV(1.0, pw);
}

/* The decay factor of distance d under the law of p. */
SYNTH_HD double synth_decay(const struct synth_params* p, double d) {
  return p->law == SYNTH_LAW_ALGEBRAIC ? synth_algebraic(d, p->alpha) : synth_exp_nonpos(SYNTH_MUL(-p->alpha, d));
}

SYNTH_HD uint32_t synth_compact1by2(uint64_t v) {
  /* keep bits 0, 3, 6, ... of v and pack them (21 bits) */
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10C30C30C30C30C3ull;
  v = (v ^ (v >> 4)) & 0x100F00F00F00F00Full;
  v = (v ^ (v >> 8)) & 0x001F0000FF0000FFull;
  v = (v ^ (v >> 16)) & 0x001F00000000FFFFull;
  v = (v ^ (v >> 32)) & 0x00000000001FFFFFull;
  return (uint32_t)v;
}

SYNTH_HD void synth_lattice_point(int64_t i, int32_t* x, int32_t* y, int32_t* z) {
  *x = (int32_t)synth_compact1by2((uint64_t)i);
  *y = (int32_t)synth_compact1by2((uint64_t)i >> 1);
  *z = (int32_t)synth_compact1by2((uint64_t)i >> 2);
}

SYNTH_HD double synth_distance(const synth_params* p, int64_t i, int64_t j) {
  if (p->kind == SYNTH_KIND_1D) return (double)(i > j ? i - j : j - i);
  int32_t xi, yi, zi, xj, yj, zj;
  synth_lattice_point(i, &xi, &yi, &zi);
  synth_lattice_point(j, &xj, &yj, &zj);
  int64_t dx = xi - xj, dy = yi - yj, dz = zi - zj;
  return SYNTH_SQRT((double)(dx * dx + dy * dy + dz * dz));
}

/* Element a_ij (0 outside [0,n)^2: the zero padding of the last leaf). */
SYNTH_HD double synth_element(const synth_params* p, int64_t i, int64_t j) {
  if (i < 0 || j < 0 || i >= p->n || j >= p->n) return 0.0;
  double d = synth_distance(p, i, j);
  double e = synth_decay(p, d);
  double v = SYNTH_MUL(SYNTH_MUL(p->c, synth_uniform(p->seed, i, j)), e);
  double av = v < 0.0 ? -v : v;
  return av < p->cutoff ? 0.0 : v;
}

/* Upper bound of |a_ij| over the leaf rows [bi*bs, bi*bs+bs) x columns
 * [bj*bs, bj*bs+bs) (bs a power of two): c exp(-alpha dmin), dmin the least
 * distance between the two index sets (for the 3-D kind an aligned
 * power-of-two run of Morton indices is an axis-aligned box).  Slightly
 * enlarged so rounding cannot make it smaller than a true element. */
SYNTH_HD double synth_leaf_bound(const synth_params* p, int32_t bs, int64_t bi, int64_t bj) {
  double dmin;
  if (p->kind == SYNTH_KIND_1D) {
    int64_t gap = (bi > bj ? bi - bj : bj - bi) * (int64_t)bs - (bs - 1);
    dmin = gap > 0 ? (double)gap : 0.0;
  } else {
    int32_t a0[3], a1[3], b0[3], b1[3];
    synth_lattice_point(bi * bs, &a0[0], &a0[1], &a0[2]);
    synth_lattice_point(bi * bs + bs - 1, &a1[0], &a1[1], &a1[2]);
    synth_lattice_point(bj * bs, &b0[0], &b0[1], &b0[2]);
    synth_lattice_point(bj * bs + bs - 1, &b1[0], &b1[1], &b1[2]);
    int64_t d2 = 0;
    for (int ax = 0; ax < 3; ++ax) {
      int64_t g = 0;
      if (b0[ax] > a1[ax]) g = b0[ax] - a1[ax];
      if (a0[ax] > b1[ax]) g = a0[ax] - b1[ax];
      d2 += g * g;
    }
    dmin = SYNTH_SQRT((double)d2);
  }
  double e = synth_decay(p, dmin);
  return SYNTH_MUL(SYNTH_MUL(p->c < 0.0 ? -p->c : p->c, e), 1.0 + 0x1.0p-40);
}

#endif /* SYNTH_DECAYGEN_H */
