// tcforms.cuh -- the operand-term layout shared by the operand preparation
// (prep.cu) and the tensor-core leaf GEMM (gemm_tc.cu).  Per leaf, TERMS
// two-byte term (slice) tiles, every tile swizzled and K-major (tile row =
// leaf row for an A operand, leaf column for a B operand; k along the row), so
// one 1-D bulk copy lands a tile ready for tcgen05:
//   whole-K forms (FP16 scaled, BF16 3-slice split): term s at s * 8 KB, a
//     64 x 64 tile in the 128-byte swizzle (a row holds all 64 k);
//   K-half form (BF16 4-slice split): half h, slice s at (h * TERMS + s) * 4 KB,
//     a 64 x 32 tile (k = 32 h .. 32 h + 31) in the 64-byte swizzle, so a
//     pipeline stage holds half of a step's K and four slices still fit twice
//     in shared memory.
#pragma once
#include <cstdint>

#include "spamm.h"

namespace spamm {

constexpr uint32_t kTerm = 64 * 64 * 2;  // one 64 x 64 two-byte term tile: 8 KB
constexpr uint32_t kHalfTerm = kTerm / 2;  // one 64 x 32 K-half tile: 4 KB

// TERMS: terms per operand.  NACC: TMEM accumulators per step (accumulator a
// takes the term products of index sum a, the last one every larger sum).
// KHALF: a step's K is staged in two halves.  NS: pipeline stages.
template <int PREC>
struct FormCfg;
template <>
struct FormCfg<SPAMM_PREC_BF16_SPLIT> {
  static constexpr int TERMS = 3, NACC = 2, NS = 2;  // stages of 96 KB
  static constexpr bool KHALF = false;
  static constexpr uint32_t AB = 1u;  // operand format bf16
};
template <>
struct FormCfg<SPAMM_PREC_BF16_SPLIT4> {
  static constexpr int TERMS = 4, NACC = 3, NS = 3;  // stages of 64 KB (half a step)
  static constexpr bool KHALF = true;
  static constexpr uint32_t AB = 1u;
};
template <>
struct FormCfg<SPAMM_PREC_FP16_SCALED> {
  static constexpr int TERMS = 2, NACC = 1, NS = 3;  // stages of 64 KB
  static constexpr bool KHALF = false;
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

}  // namespace spamm
