// tcforms.cuh -- the operand-term layout shared by the operand preparation
// (prep.cu) and the tensor-core leaf GEMM (gemm_tc.cu).  Per leaf, TERMS
// two-byte term (slice) tiles, every tile swizzled and K-major (tile row =
// leaf row for an A operand, leaf column for a B operand; k along the row), so
// one 1-D bulk copy lands a tile ready for tcgen05.  A form stages a step's K
// in KPARTS parts; part h of term s sits at (h * TERMS + s) * (8 KB / KPARTS):
//   KPARTS = 1: a 64 x 64 tile in the 128-byte swizzle (a row holds all 64 k);
//   KPARTS = 2: a 64 x 32 tile (k = 32 h ..) in the 64-byte swizzle;
//   KPARTS = 4: a 64 x 16 tile (k = 16 h ..) in the 32-byte swizzle.
// Smaller parts give smaller pipeline stages, so more of them fit in shared
// memory and more copies are in flight for the same bytes.
#pragma once
#include <cstdint>

#include "spamm.h"

namespace spamm {

constexpr uint32_t kTerm = 64 * 64 * 2;  // one 64 x 64 two-byte term tile: 8 KB

// TERMS: terms per operand.  NACC: TMEM accumulators per step (accumulator a
// takes the term products of index sum a, the last one every larger sum).
// KPARTS: parts a step's K is staged in.  NS: pipeline stages, each
// 4 leaves x TERMS x 8 KB / KPARTS.
#ifndef SPAMM_KPARTS_BF16_SPLIT
#define SPAMM_KPARTS_BF16_SPLIT 1
#endif
#ifndef SPAMM_KPARTS_BF16_SPLIT4
#define SPAMM_KPARTS_BF16_SPLIT4 2
#endif
#ifndef SPAMM_KPARTS_FP16_SCALED
#define SPAMM_KPARTS_FP16_SCALED 1
#endif
constexpr int kStageBudget = 196608;  // shared memory for the stages: 192 KB
template <int PREC>
struct FormCfg;
template <>
struct FormCfg<SPAMM_PREC_BF16_SPLIT> {
  static constexpr int TERMS = 3, NACC = 2, KPARTS = SPAMM_KPARTS_BF16_SPLIT;
  static constexpr int NS = kStageBudget / (4 * TERMS * (int)kTerm / KPARTS);
  static constexpr uint32_t AB = 1u;  // operand format bf16
};
template <>
struct FormCfg<SPAMM_PREC_BF16_SPLIT4> {
  static constexpr int TERMS = 4, NACC = 3, KPARTS = SPAMM_KPARTS_BF16_SPLIT4;
  static constexpr int NS = kStageBudget / (4 * TERMS * (int)kTerm / KPARTS);
  static constexpr uint32_t AB = 1u;
};
template <>
struct FormCfg<SPAMM_PREC_FP16_SCALED> {
  static constexpr int TERMS = 2, NACC = 1, KPARTS = SPAMM_KPARTS_FP16_SCALED;
  static constexpr int NS = kStageBudget / (4 * TERMS * (int)kTerm / KPARTS);
  static constexpr uint32_t AB = 0u;  // f16
};
template <int PREC>
__host__ __device__ constexpr uint32_t leaf_bytes() {
  return FormCfg<PREC>::TERMS * kTerm;
}

// Byte offset of element (row, k) in a 128-byte-swizzled K-major tile of
// 64 two-byte elements per row: 16-byte chunk index XOR (row mod 8).
__host__ __device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ row) & 7) << 4) + (k & 7) * 2);
}

// Byte offset of element (row, k), 0 <= k < 32, in a 64-byte-swizzled K-major
// tile of 32 two-byte elements per row: 16-byte chunk index XOR bits 1..2 of
// the row (the swizzle repeats every 8 rows = 512 bytes).
__host__ __device__ __forceinline__ uint32_t sw64_offset(int row, int k) {
  return (uint32_t)(row * 64 + ((((k >> 3) ^ (row >> 1)) & 3) << 4) + (k & 7) * 2);
}

// Byte offset of element (row, k), 0 <= k < 16, in a 32-byte-swizzled K-major
// tile of 16 two-byte elements per row: 16-byte chunk index XOR bit 2 of the
// row (the swizzle repeats every 8 rows = 256 bytes).
__host__ __device__ __forceinline__ uint32_t sw32_offset(int row, int k) {
  return (uint32_t)(row * 32 + ((((k >> 3) ^ (row >> 2)) & 1) << 4) + (k & 7) * 2);
}

// Offset of element (row, k), 0 <= k < 64, of term s in a leaf's terms.
template <int KPARTS>
__host__ __device__ __forceinline__ uint32_t term_offset(int terms, int s, int row, int k) {
  constexpr uint32_t part = kTerm / KPARTS;
  constexpr int kw = 64 / KPARTS;  // k per part
  const int h = k / kw, kk = k % kw;
  const uint32_t base = (uint32_t)(h * terms + s) * part;
  if constexpr (KPARTS == 1) return base + sw128_offset(row, kk);
  if constexpr (KPARTS == 2) return base + sw64_offset(row, kk);
  return base + sw32_offset(row, kk);
}

}  // namespace spamm
