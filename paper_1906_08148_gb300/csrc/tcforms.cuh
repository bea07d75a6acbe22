// tcforms.cuh -- the operand-term layout shared by the operand preparation
// (prep.cu) and the tensor-core leaf GEMM (gemm_tc.cu): per leaf, TERMS
// 64 x 64 two-byte term tiles of 8 KB each, term s at s * 8 KB, every tile
// 128-byte swizzled and K-major (tile row = leaf row for an A operand, leaf
// column for a B operand; k along the 128-byte row), so one 1-D bulk copy
// lands a tile ready for tcgen05.
#pragma once
#include <cstdint>

#include "spamm.h"

namespace spamm {

constexpr uint32_t kTerm = 64 * 64 * 2;  // one 64 x 64 two-byte term tile: 8 KB

template <int PREC>
struct FormCfg;
template <>
struct FormCfg<SPAMM_PREC_BF16_SPLIT> {
  static constexpr int TERMS = 3;  // terms per operand
  static constexpr int NS = 2;     // pipeline stages of 96 KB
  static constexpr uint32_t AB = 1u;  // operand format bf16
};
template <>
struct FormCfg<SPAMM_PREC_FP16_SCALED> {
  static constexpr int TERMS = 2;
  static constexpr int NS = 3;     // stages of 64 KB
  static constexpr uint32_t AB = 0u;  // f16
};
template <int PREC>
__host__ __device__ constexpr uint32_t leaf_bytes() {
  return FormCfg<PREC>::TERMS * kTerm;
}

// Byte offset of element (row, k) in a 128-byte-swizzled K-major tile of
// 64 two-byte elements per row: 16-byte chunk index XOR (row mod 8).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ row) & 7) << 4) + (k & 7) * 2);
}

}  // namespace spamm
