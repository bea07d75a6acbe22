// prep.cu -- the operand terms of the tensor-core forms: every (truncated)
// input leaf split into BF16 or per-leaf-scaled FP16 terms in the layout of
// tcforms.cuh, built once per multiply before the leaf products run.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fbits.cuh"
#include "internal.cuh"
#include "tcforms.cuh"

namespace spamm {

// ---------------------------------------------------------------- operand prep
// Terms of one leaf as 16-byte swizzled chunks: chunk (row, c8) holds k =
// 8 c8 .. 8 c8 + 7 of one tile row.  role 0 (A): term s is a 64-row tile at
// s * 8 KB, tile row = leaf row, k = leaf column.  role 1 (B): term s occupies
// tile rows 64 s .. 64 s + 63 (row = leaf column n), k = leaf row.
//
// One CTA of 256 threads per leaf; a thread owns two chunks and loads their 16
// elements first (A: 8 consecutive doubles of a row; B: one column, so the
// lanes of a warp read consecutive doubles of each leaf row).  Each element is
// rounded once to FP32 on its bits (fbits.cuh; the FP16 form's per-leaf scale
// 2^e folded in), then split in FP32:
//   BF16: b0 = bf16(a), b1 = bf16(a - b0), b2 = bf16(a - b0 - b1)
//   FP16: h0 = f16(a 2^e), h1 = f16(a 2^e - h0), max|a 2^e| in [2^14, 2^15)
// (each residual is exact in FP32).
template <int PREC>
__global__ void __launch_bounds__(256) prep_terms_kernel(const double* __restrict__ pool,
                                                         const int64_t* __restrict__ slot, int64_t nleaves, int role,
                                                         uint8_t* __restrict__ out, int32_t* __restrict__ expo) {
  constexpr int TERMS = FormCfg<PREC>::TERMS;
  constexpr uint32_t LEAF = leaf_bytes<PREC>();
  __shared__ unsigned long long smax[8];
  __shared__ int s_shift;
  // BF16 (three terms): the terms are assembled in shared memory and leave as
  // one contiguous block (the B role's direct 16-byte stores would hit a
  // different 128-byte line per lane); FP16 measured no faster that way
  constexpr bool kStage = TERMS == 3;
  __shared__ uint4 stile[kStage ? LEAF / 16 : 1];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int64_t m = blockIdx.x; m < nleaves; m += gridDim.x) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(pool + slot[m] * 4096);
    unsigned long long v[2][8];
    int row[2], c8[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (role == 0) {
        row[j] = (t >> 3) + 32 * j;
        c8[j] = t & 7;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[j][e] = __ldg(src + row[j] * 64 + 8 * c8[j] + e);
      } else {
        row[j] = t & 63;
        c8[j] = (t >> 6) + 4 * j;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[j][e] = __ldg(src + (8 * c8[j] + e) * 64 + row[j]);
      }
    }
    int shift = 0;
    if constexpr (PREC == SPAMM_PREC_FP16_SCALED) {
      // largest |a| of the leaf: |x| of doubles orders like their bits without the sign
      unsigned long long mx = 0;
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const unsigned long long a = v[j][e] & 0x7FFFFFFFFFFFFFFFull;
          mx = a > mx ? a : mx;
        }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
      }
      if (lane == 0) smax[warp] = mx;
      __syncthreads();
      if (t == 0) {
        unsigned long long g = 0;
        for (int w = 0; w < 8; ++w) g = smax[w] > g ? smax[w] : g;
        s_shift = fp16_leaf_shift(g);
        expo[m] = s_shift;
      }
      __syncthreads();
      shift = s_shift;
    }
    uint8_t* dst = out + m * (int64_t)LEAF;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      __align__(16) uint16_t term[TERMS][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float a = __uint_as_float(fbits_from_double_rn(v[j][e], shift));
#pragma unroll
        for (int s = 0; s < TERMS; ++s) {
          if constexpr (PREC == SPAMM_PREC_FP16_SCALED) {
            const __half h = __float2half_rn(a);
            term[s][e] = __half_as_ushort(h);
            a -= __half2float(h);
          } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(a);
            term[s][e] = __bfloat16_as_ushort(h);
            a -= __bfloat162float(h);
          }
        }
      }
#pragma unroll
      for (int s = 0; s < TERMS; ++s) {
        const uint32_t off = s * kTerm + sw128_offset(row[j], 8 * c8[j]);
        if constexpr (kStage)
          stile[off >> 4] = *reinterpret_cast<const uint4*>(term[s]);
        else
          *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(term[s]);
      }
    }
    if constexpr (kStage) {
      __syncthreads();
      // the leaf's terms leave in order: consecutive threads, consecutive 16-byte chunks
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      for (int i = t; i < (int)(LEAF / 16); i += blockDim.x) d4[i] = stile[i];
    }
    __syncthreads();  // stile, smax and s_shift are reused by the next leaf
  }
}

void prep_terms(spamm_mat M, spamm_prec prec, int role, BufP* terms, BufP* expo, spamm_ctx on) {
  spamm_ctx ctx = on ? on : M->ctx;
  if (M->bs != 64) fail(SPAMM_E_UNSUPPORTED, "tensor-core precision forms are built for bs = 64");
  const int64_t want = M->nleaves, cap = (int64_t)ctx->num_sms * 8;
  const unsigned grid = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  if (prec == SPAMM_PREC_BF16_SPLIT) {
    *terms = alloc_n<uint8_t>(ctx, M->nleaves * (int64_t)leaf_bytes<SPAMM_PREC_BF16_SPLIT>());
    if (M->nleaves > 0) {
      prep_terms_kernel<SPAMM_PREC_BF16_SPLIT><<<grid, 256, 0, ctx->stream>>>(
          P<double>(M->pool), P<int64_t>(M->slot), M->nleaves, role, P<uint8_t>(*terms), nullptr);
      CK_LAUNCH("prep_terms_kernel<bf16>");
    }
  } else {
    *terms = alloc_n<uint8_t>(ctx, M->nleaves * (int64_t)leaf_bytes<SPAMM_PREC_FP16_SCALED>());
    *expo = alloc_n<int32_t>(ctx, M->nleaves);
    if (M->nleaves > 0) {
      prep_terms_kernel<SPAMM_PREC_FP16_SCALED><<<grid, 256, 0, ctx->stream>>>(
          P<double>(M->pool), P<int64_t>(M->slot), M->nleaves, role, P<uint8_t>(*terms), P<int32_t>(*expo));
      CK_LAUNCH("prep_terms_kernel<fp16>");
    }
  }
}

}  // namespace spamm
