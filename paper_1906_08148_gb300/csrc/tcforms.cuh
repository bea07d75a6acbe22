// tcforms.cuh -- the operand-term layout shared by the operand preparation
// (prep.cu) and the tensor-core leaf GEMM (gemm_tc.cu).  Per leaf, TERMS
// two-byte term (slice) tiles, every tile swizzled and K-major (tile row =
// leaf row for an A operand, leaf column for a B operand; k along the row).
// A form stages a step's K in KPARTS parts: a row of a part holds 64 / KPARTS
// k (128, 64 or 32 bytes, in the 128-, 64- or 32-byte swizzle), and 8 rows of
// it make one swizzle atom (1 KB, 512 B or 256 B).  Part h of a leaf is one
// contiguous block of TERMS x 8 KB / KPARTS: atom g (rows 8 g ..) of term s at
// (g TERMS + s) x atom -- the terms interleaved atom by atom.  So one 1-D bulk
// copy lands a leaf's part with all its terms, and the 128-row operand of
// term s over two leaves placed one after the other is a single matrix
// descriptor: start at s x atom, stride between 8-row groups TERMS x atom.
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

// Bytes of one 8-row swizzle atom of a part.
template <int KPARTS>
__host__ __device__ constexpr uint32_t term_atom() {
  return 8u * 2u * (64u / KPARTS);
}

// Offset of element (row, k), 0 <= k < 64, of term s in a leaf's terms.
template <int KPARTS>
__host__ __device__ __forceinline__ uint32_t term_offset(int terms, int s, int row, int k) {
  constexpr uint32_t part = kTerm / KPARTS, atom = term_atom<KPARTS>();
  constexpr int kw = 64 / KPARTS;  // k per part
  const int h = k / kw, kk = k % kw, g = row >> 3, r8 = row & 7;
  const uint32_t base = (uint32_t)h * terms * part + (uint32_t)(g * terms + s) * atom;
  if constexpr (KPARTS == 1) return base + sw128_offset(r8, kk);
  if constexpr (KPARTS == 2) return base + sw64_offset(r8, kk);
  return base + sw32_offset(r8, kk);
}

}  // namespace spamm
