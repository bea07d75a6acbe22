// prep.cu -- the operand terms of the tensor-core forms: every (truncated)
// input leaf split into BF16 slices or per-leaf-scaled FP16 terms in the
// layout of tcforms.cuh, built once per multiply before the leaf products run.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fbits.cuh"
#include "internal.cuh"
#include "slices.cuh"
#include "tcforms.cuh"

namespace spamm {

// Thread <-> element mapping shared by both kernels: one CTA of 256 threads
// per 64 x 64 tile of a leaf; a thread owns two 16-byte chunks of the
// K-major term tiles (8 consecutive k of one tile row) and loads their 16
// FP64 elements first.
// role 0 (A): tile row = leaf row (t >> 3) + 32 j, k = leaf columns 8 (t & 7) ..
// role 1 (B): tile row = leaf column t & 63, k = leaf rows 8 ((t >> 6) + 4 j) ..,
// so the lanes of a warp read consecutive doubles of each leaf row.
struct ChunkMap {
  int row[2], c8[2];
  __device__ ChunkMap(int t, int role) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      row[j] = role == 0 ? (t >> 3) + 32 * j : (t & 63);
      c8[j] = role == 0 ? (t & 7) : (t >> 6) + 4 * j;
    }
  }
  // src: the tile's first element; ld: the leaf's row length
  __device__ void load(const unsigned long long* src, int ld, int role, unsigned long long (&v)[2][8]) const {
    if (role == 0) {
      // 8 consecutive doubles of one row: four 16-byte loads
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(src + row[j] * ld + 8 * c8[j]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const ulonglong2 w = __ldg(p + e);
          v[j][2 * e] = w.x;
          v[j][2 * e + 1] = w.y;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 8; ++e) v[j][e] = __ldg(src + (8 * c8[j] + e) * ld + row[j]);
    }
  }
};

// Operand tiles of a leaf.  A 64 x 64 leaf is one tile; a 128 x 128 leaf is
// four, tile 2 r2 + kh holding rows 64 r2 .. of the leaf's row dimension for
// the operand (A: leaf rows; B: leaf columns) and k = 64 kh ..  (A: leaf
// columns; B: leaf rows), each split and scaled as a 64 x 64 leaf of its own,
// so the leaf-product kernel runs a 128-leaf product as two K-half steps
// over the four tiles of each operand.  Tile x of leaf m is at index
// m * tiles + x of the term and exponent arrays.
__device__ __forceinline__ const double* tile_src(const double* leaf, int bs, int role, int x) {
  if (bs == 64) return leaf;
  const int r2 = x >> 1, kh = x & 1;
  return role == 0 ? leaf + (int64_t)(64 * r2) * bs + 64 * kh : leaf + (int64_t)(64 * kh) * bs + 64 * r2;
}

// ------------------------------------------------------- BF16 slices (error-free split)
// Per leaf: the largest biased exponent of every line (A: row, B: column) and
// of the leaf, the leaf's scale exponent f (stored in expo[m]), then every
// element's S digits (slices.cuh) as BF16 values d_s 2^(e - 8 - 9 s).  The
// slices are assembled in shared memory and leave as one contiguous block.
template <int S, int KPARTS>
__global__ void __launch_bounds__(256) prep_slices_kernel(const double* __restrict__ pool,
                                                          const int64_t* __restrict__ slot, int64_t nleaves, int bs,
                                                          int role, uint8_t* __restrict__ out,
                                                          int32_t* __restrict__ expo) {
  constexpr uint32_t LEAF = (uint32_t)S * kTerm;
  __shared__ uint4 stile[LEAF / 16];
  __shared__ int s_line[4][64];  // role 1: per-column maxima of each quarter of the leaf rows
  __shared__ int s_warp[8];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const ChunkMap cm(t, role);
  const int tiles = (bs / 64) * (bs / 64);
  for (int64_t m = blockIdx.x; m < nleaves * tiles; m += gridDim.x) {
    const int64_t leaf = m / tiles;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(
        tile_src(pool + slot[leaf] * (int64_t)bs * bs, bs, role, (int)(m - leaf * tiles)));
    unsigned long long v[2][8];
    cm.load(src, bs, role, v);
    // largest biased exponent of each of this thread's two lines
    int em[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int x = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) x = max(x, slice_biased_exp(v[j][e]));
      em[j] = x;
    }
    if (role == 0) {
      // a row's 8 chunks are held by 8 consecutive lanes
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) em[j] = max(em[j], __shfl_xor_sync(0xffffffffu, em[j], off));
    } else {
      // a column's 8 chunks are held by the threads t & 63 == column of 4 warp pairs
      s_line[t >> 6][t & 63] = max(em[0], em[1]);
      __syncthreads();
      const int c = t & 63;
      const int x = max(max(s_line[0][c], s_line[1][c]), max(s_line[2][c], s_line[3][c]));
      em[0] = em[1] = x;
    }
    int lm = max(em[0], em[1]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lm = max(lm, __shfl_xor_sync(0xffffffffu, lm, off));
    if (lane == 0) s_warp[warp] = lm;
    __syncthreads();
    int leaf_max = s_warp[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) leaf_max = max(leaf_max, s_warp[w]);
    const int f = slice_leaf_shift(leaf_max);
    if (t == 0) expo[m] = f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int e = slice_line_exp(em[j], f);
      __align__(16) uint16_t term[S][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int32_t d[S];
        slice_digits<S>(v[j][q], em[j], d);
#pragma unroll
        for (int s = 0; s < S; ++s) term[s][q] = slice_bf16_bits(d[s], e - 8 - 9 * s);
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const uint32_t off = term_offset<KPARTS>(S, s, cm.row[j], 8 * cm.c8[j]);
        stile[off >> 4] = *reinterpret_cast<const uint4*>(term[s]);
      }
    }
    __syncthreads();
    // the leaf's slices leave in order: consecutive threads, consecutive 16-byte chunks
    uint4* d4 = reinterpret_cast<uint4*>(out + m * (int64_t)LEAF);
    for (int i = t; i < (int)(LEAF / 16); i += blockDim.x) d4[i] = stile[i];
    __syncthreads();  // stile, s_line and s_warp are reused by the next leaf
  }
}

// ------------------------------------------------------------ FP16 terms
// Each element is rounded once to FP32 on its bits (fbits.cuh) with the
// per-leaf scale 2^e folded in, max|a 2^e| in [2^14, 2^15), then split in
// FP32: h0 = f16(a 2^e), h1 = f16(a 2^e - h0) (the residual is exact in FP32).
__global__ void __launch_bounds__(256) prep_fp16_kernel(const double* __restrict__ pool,
                                                        const int64_t* __restrict__ slot, int64_t nleaves, int bs,
                                                        int role, uint8_t* __restrict__ out,
                                                        int32_t* __restrict__ expo) {
  constexpr int TERMS = FormCfg<SPAMM_PREC_FP16_SCALED>::TERMS;
  constexpr uint32_t LEAF = leaf_bytes<SPAMM_PREC_FP16_SCALED>();
  __shared__ unsigned long long smax[8];
  __shared__ int s_shift;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const ChunkMap cm(t, role);
  const int tiles = (bs / 64) * (bs / 64);
  for (int64_t m = blockIdx.x; m < nleaves * tiles; m += gridDim.x) {
    const int64_t leaf = m / tiles;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(
        tile_src(pool + slot[leaf] * (int64_t)bs * bs, bs, role, (int)(m - leaf * tiles)));
    unsigned long long v[2][8];
    cm.load(src, bs, role, v);
    // largest |a| of the tile: |x| of doubles orders like their bits without the sign
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
    const int shift = s_shift;
    uint8_t* dst = out + m * (int64_t)LEAF;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      __align__(16) uint16_t term[TERMS][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float a = __uint_as_float(fbits_from_double_rn(v[j][e], shift));
#pragma unroll
        for (int s = 0; s < TERMS; ++s) {
          const __half h = __float2half_rn(a);
          term[s][e] = __half_as_ushort(h);
          a -= __half2float(h);
        }
      }
#pragma unroll
      for (int s = 0; s < TERMS; ++s)
        *reinterpret_cast<uint4*>(dst + term_offset<FormCfg<SPAMM_PREC_FP16_SCALED>::KPARTS>(TERMS, s, cm.row[j],
                                                                                          8 * cm.c8[j])) =
            *reinterpret_cast<const uint4*>(term[s]);
    }
    __syncthreads();  // smax and s_shift are reused by the next leaf
  }
}

static uint32_t form_leaf_bytes(spamm_prec prec) {
  switch (prec) {
    case SPAMM_PREC_BF16_SPLIT: return leaf_bytes<SPAMM_PREC_BF16_SPLIT>();
    case SPAMM_PREC_BF16_SPLIT4: return leaf_bytes<SPAMM_PREC_BF16_SPLIT4>();
    default: return leaf_bytes<SPAMM_PREC_FP16_SCALED>();
  }
}

void prep_terms(spamm_mat M, spamm_prec prec, int role, BufP* terms, BufP* expo, spamm_ctx on) {
  spamm_ctx ctx = on ? on : M->ctx;
  const int bs = M->bs;
  if (bs != 64 && bs != 128) fail(SPAMM_E_UNSUPPORTED, "tensor-core precision forms are built for bs = 64 and 128");
  const int64_t ntiles = M->nleaves * tc_tiles_per_leaf(bs), cap = (int64_t)ctx->num_sms * 8;
  const unsigned grid = (unsigned)(ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap);
  *terms = alloc_n<uint8_t>(ctx, ntiles * (int64_t)form_leaf_bytes(prec));
  *expo = alloc_n<int32_t>(ctx, ntiles);
  if (M->nleaves == 0) return;
  const double* pool = P<double>(M->pool);
  const int64_t* slot = P<int64_t>(M->slot);
  if (prec == SPAMM_PREC_BF16_SPLIT) {
    prep_slices_kernel<3, FormCfg<SPAMM_PREC_BF16_SPLIT>::KPARTS><<<grid, 256, 0, ctx->stream>>>(pool, slot, M->nleaves, bs, role,
                                                                P<uint8_t>(*terms), P<int32_t>(*expo));
    CK_LAUNCH("prep_slices_kernel<3>");
  } else if (prec == SPAMM_PREC_BF16_SPLIT4) {
    prep_slices_kernel<4, FormCfg<SPAMM_PREC_BF16_SPLIT4>::KPARTS><<<grid, 256, 0, ctx->stream>>>(pool, slot, M->nleaves, bs, role,
                                                               P<uint8_t>(*terms), P<int32_t>(*expo));
    CK_LAUNCH("prep_slices_kernel<4>");
  } else {
    prep_fp16_kernel<<<grid, 256, 0, ctx->stream>>>(pool, slot, M->nleaves, bs, role, P<uint8_t>(*terms),
                                                    P<int32_t>(*expo));
    CK_LAUNCH("prep_fp16_kernel");
  }
}

}  // namespace spamm
