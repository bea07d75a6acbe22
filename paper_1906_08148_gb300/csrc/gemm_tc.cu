// gemm_tc.cu -- kernel (c), tensor-core forms (bs = 64): BF16 three-term split
// and FP16 with per-leaf power-of-two scaling, FP32 accumulation, with the
// C-leaf norms of kernel (d) in the epilogue.
//
// Each leaf product of Algorithm 1 ("C = AB" at the lowest level) is a real
// 64 x 64 x 64 contraction on tcgen05.  Operands are split into low-precision
// terms, each the rounding of what the previous terms left:
//   BF16 split : a = a0 + a1 + a2, b = b0 + b1 + b2 (bf16); the six products
//                with term-index sum <= 2 are formed.
//   FP16 scaled: a' = a 2^eA with max|a'| in [2^14, 2^15) per leaf,
//                a' = h0 + h1 (f16), likewise b'; products h0 g0, h0 g1, h1 g0,
//                scaled back by 2^-(eA + eB).
//
// Column pairs.  The two output leaves (2I, j) and (2I+1, j) of a quadtree
// quad share every B leaf (k, j).  Their A terms are stacked in M: for term s
// the 128-row operand is [A(2I,k)_s; A(2I+1,k)_s] (a zero tile where that leaf
// has no kept product for this k), so one B tile serves both and the
// accumulator holds the two output leaves in its row halves.  With
// B = [b0^T; b1^T; b2^T] (BF16) or [g0^T; g1^T] (FP16) one k step issues
//   BF16: a0 x [b0|b1|b2] (N=192), a1 x [b0|b1] (N=128), a2 x b0 (N=64)
//   FP16: h0 x [g0|g1]    (N=128), h1 x g0      (N=64)
// into a fresh TMEM accumulator, whose 64-column blocks add up to the step's
// contribution.  Accumulators are double-buffered: while the tensor cores run
// step t+1, the epilogue drains step t into FP32 registers with round-to-
// nearest adds (one output row per thread, per-leaf FP16 scales applied per
// row), which keeps the error of long k runs at the level of one leaf product.
// The two pairs of a quad run back to back on one CTA, so their shared A
// leaves are still in L2.
//
// Warp roles (one CTA per SM, persistent, quads statically interleaved in
// Morton order so concurrently running CTAs share A rows and B columns in L2):
//   warp 0     TMA producer: ring of NS stages (two A leaves' terms + one B
//              leaf's terms), 1-D bulk copies of pre-swizzled tiles, mbarriers.
//   warp 1     allocates 512 TMEM columns and issues the MMAs of each step.
//   warps 2-5  epilogue: TMEM lane = accumulator row, drain per step, write
//              the FP64 output leaves and their squared norms.
// No atomics on C: one CTA owns each output leaf; k runs in ascending order.
// Every wait is bounded; on timeout the CTA sets the error word and leaves.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace spamm {

constexpr int kTcThreads = 192;
constexpr uint32_t kTerm = 64 * 64 * 2;  // one 64 x 64 two-byte term tile: 8 KB

template <int PREC>
struct PairCfg;
template <>
struct PairCfg<SPAMM_PREC_BF16_SPLIT> {
  static constexpr int TERMS = 3;  // terms per operand
  static constexpr int NS = 3;     // pipeline stages
  static constexpr bool SCALED = false;
};
template <>
struct PairCfg<SPAMM_PREC_FP16_SCALED> {
  static constexpr int TERMS = 2;
  static constexpr int NS = 4;
  static constexpr bool SCALED = true;
};
template <int PREC>
__host__ __device__ constexpr uint32_t leaf_bytes() {
  return PairCfg<PREC>::TERMS * kTerm;
}
template <int PREC>
__host__ __device__ constexpr uint32_t stage_bytes() {
  return 3 * leaf_bytes<PREC>();  // two A leaves (stacked per term) + one B leaf
}
template <int PREC>
constexpr size_t pair_smem_bytes() {
  return 1024 + (size_t)PairCfg<PREC>::NS * stage_bytes<PREC>();
}

// Byte offset of element (row, k) in a 128-byte-swizzled K-major tile of
// 64 two-byte elements per row: 16-byte chunk index XOR (row mod 8).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ row) & 7) << 4) + (k & 7) * 2);
}

// ---------------------------------------------------------------- operand prep
// Terms of one leaf as 16-byte swizzled chunks: chunk (row, c8) holds 8
// consecutive k of one tile row.  role 0 (A): term s is a 64-row tile at
// s * 8 KB, tile row = leaf row, k = leaf column.  role 1 (B): term s occupies
// tile rows 64 s .. 64 s + 63 (row = leaf column n), k = leaf row.
__global__ void prep_bf16_terms_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot,
                                       int64_t nleaves, int role, uint8_t* __restrict__ out) {
  constexpr uint32_t LEAF = leaf_bytes<SPAMM_PREC_BF16_SPLIT>();
  for (int64_t m = blockIdx.x; m < nleaves; m += gridDim.x) {
    const double* src = pool + slot[m] * 4096;
    uint8_t* dst = out + m * (int64_t)LEAF;
    for (int ch = threadIdx.x; ch < 512; ch += blockDim.x) {
      const int row = ch >> 3, c8 = ch & 7;
      __align__(16) __nv_bfloat16 t[3][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = 8 * c8 + e;
        double rest = role == 0 ? src[row * 64 + k] : src[k * 64 + row];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          t[s][e] = __double2bfloat16(rest);
          rest -= (double)__bfloat162float(t[s][e]);
        }
      }
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const uint32_t off = role == 0 ? s * kTerm + sw128_offset(row, 8 * c8) : sw128_offset(64 * s + row, 8 * c8);
        *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(t[s]);
      }
    }
  }
}

// FP16: per-leaf exponent e with max|a| 2^e in [2^14, 2^15), then two terms.
__global__ void prep_fp16_terms_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot,
                                       int64_t nleaves, int role, uint8_t* __restrict__ out,
                                       int32_t* __restrict__ expo) {
  constexpr uint32_t LEAF = leaf_bytes<SPAMM_PREC_FP16_SCALED>();
  __shared__ double smax[8];
  __shared__ int s_e;
  for (int64_t m = blockIdx.x; m < nleaves; m += gridDim.x) {
    const double* src = pool + slot[m] * 4096;
    uint8_t* dst = out + m * (int64_t)LEAF;
    double mx = 0.0;
    for (int e = threadIdx.x; e < 4096; e += blockDim.x) mx = fmax(mx, fabs(src[e]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, smax[w]);
      int x = 0;
      if (t > 0.0) frexp(t, &x);  // t = f 2^x, f in [0.5, 1)
      int ex = t > 0.0 ? 15 - x : 0;
      ex = ex > 120 ? 120 : (ex < -120 ? -120 : ex);
      s_e = ex;
      expo[m] = ex;
    }
    __syncthreads();
    const int e2 = s_e;
    for (int ch = threadIdx.x; ch < 512; ch += blockDim.x) {
      const int row = ch >> 3, c8 = ch & 7;
      __align__(16) __half t[2][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = 8 * c8 + e;
        const double a = ldexp(role == 0 ? src[row * 64 + k] : src[k * 64 + row], e2);
        t[0][e] = __double2half(a);
        t[1][e] = __double2half(a - (double)__half2float(t[0][e]));
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint32_t off = role == 0 ? s * kTerm + sw128_offset(row, 8 * c8) : sw128_offset(64 * s + row, 8 * c8);
        *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(t[s]);
      }
    }
    __syncthreads();
  }
}

// Kept-product runs of the pair (g0 on top, g1 below) merged by k: B leaf
// indices of one column ascend with k and are equal iff k is.
struct PairCursor {
  int64_t p0, e0, p1, e1;
  __device__ void init(const int64_t* gstart, int g0, int g1) {
    p0 = g0 >= 0 ? gstart[g0] : 0;
    e0 = g0 >= 0 ? gstart[g0 + 1] : 0;
    p1 = g1 >= 0 ? gstart[g1] : 0;
    e1 = g1 >= 0 ? gstart[g1 + 1] : 0;
  }
  __device__ bool more() const { return p0 < e0 || p1 < e1; }
  // advance past the next k; reports which rows have a product there
  __device__ void next(const int32_t* tb, bool* u0, bool* u1, int32_t* kb, int64_t* q0, int64_t* q1) {
    const int32_t k0 = p0 < e0 ? tb[p0] : INT32_MAX, k1 = p1 < e1 ? tb[p1] : INT32_MAX;
    *kb = k0 < k1 ? k0 : k1;
    *u0 = k0 == *kb;
    *u1 = k1 == *kb;
    *q0 = p0;
    *q1 = p1;
    p0 += *u0;
    p1 += *u1;
  }
};

// ------------------------------------------------------------------- GEMM
template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 1)
    gemm_pair_kernel(BatchDev batch, const uint8_t* __restrict__ zero_term, int* __restrict__ err) {
  using Cfg = PairCfg<PREC>;
  constexpr int NS = Cfg::NS, TERMS = Cfg::TERMS;
  constexpr uint32_t LEAF = leaf_bytes<PREC>(), STAGE = stage_bytes<PREC>();
  constexpr uint32_t AB = PREC == SPAMM_PREC_BF16_SPLIT ? 1u : 0u;  // operand format: bf16 or f16
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, epi_stop;
  __shared__ double red[4];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    fence_mbar_init();
    abort_flag = 0;
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  volatile int* abortp = &abort_flag;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int64_t t = 0;
      bool stop = false;
      for (int64_t un = blockIdx.x; un < batch.nunits && !stop; un += gridDim.x) {
        const int r = plan_of(batch.ubegin, batch.nplans, un);
        const PlanDev& pl = batch.plans[r];
        const int64_t Q = un - batch.ubegin[r];
        for (int pr = 0; pr < 2 && !stop; ++pr) {
          const int g0 = pl.quads[4 * Q + pr], g1 = pl.quads[4 * Q + 2 + pr];
          if (g0 < 0 && g1 < 0) continue;
          PairCursor cur;
          cur.init(pl.gstart, g0, g1);
          while (cur.more()) {
            bool u0, u1;
            int32_t kb;
            int64_t q0, q1;
            cur.next(pl.tb, &u0, &u1, &kb, &q0, &q1);
            const int s = (int)(t % NS);
            if (t >= NS && !mbar_wait_or_abort(&empty[s], (uint32_t)(((t / NS) - 1) & 1), abortp)) {
              atomicOr(err, DEV_ERR_TIMEOUT);
              *abortp = 1;
              stop = true;
              break;
            }
            uint8_t* st = smem + s * STAGE;
            const uint8_t* a0 = u0 ? pl.termsA + (int64_t)pl.ta[q0] * LEAF : nullptr;
            const uint8_t* a1 = u1 ? pl.termsA + (int64_t)pl.ta[q1] * LEAF : nullptr;
            mbar_arrive_expect_tx(&full[s], STAGE);
#pragma unroll
            for (int term = 0; term < TERMS; ++term) {
              bulk_g2s(st + term * 2 * kTerm, a0 ? a0 + term * kTerm : zero_term, kTerm, &full[s]);
              bulk_g2s(st + term * 2 * kTerm + kTerm, a1 ? a1 + term * kTerm : zero_term, kTerm, &full[s]);
            }
            bulk_g2s(st + 2 * LEAF, pl.termsB + (int64_t)kb * LEAF, LEAF, &full[s]);
            ++t;
          }
        }
      }
      // leave no bulk copy in flight: the last fill of every stage has landed
      for (int64_t k = (t > NS ? t - NS : 0); k < t; ++k) mbar_wait_bounded(&full[k % NS], (uint32_t)((k / NS) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: one k step into accumulator t & 1
    if (lane == 0) {
      int64_t t = 0;
      bool stop = false;
      for (int64_t un = blockIdx.x; un < batch.nunits && !stop; un += gridDim.x) {
        const int r = plan_of(batch.ubegin, batch.nplans, un);
        const PlanDev& pl = batch.plans[r];
        const int64_t Q = un - batch.ubegin[r];
        for (int pr = 0; pr < 2 && !stop; ++pr) {
          const int g0 = pl.quads[4 * Q + pr], g1 = pl.quads[4 * Q + 2 + pr];
          if (g0 < 0 && g1 < 0) continue;
          PairCursor cur;
          cur.init(pl.gstart, g0, g1);
          while (cur.more()) {
            bool u0, u1;
            int32_t kb;
            int64_t q0, q1;
            cur.next(pl.tb, &u0, &u1, &kb, &q0, &q1);
            const int s = (int)(t % NS);
            const int b = (int)(t & 1);
            if (!mbar_wait_or_abort(&full[s], (uint32_t)((t / NS) & 1), abortp) ||
                (t >= 2 && !mbar_wait_or_abort(&tempty[b], (uint32_t)(((t >> 1) - 1) & 1), abortp))) {
              atomicOr(err, DEV_ERR_TIMEOUT);
              *abortp = 1;
              stop = true;
              break;
            }
            tc_fence_after();
            const uint32_t d = tbase + (uint32_t)b * 256u;
            const uint32_t a_s = smem_u32(smem + s * STAGE), b_s = a_s + 2 * LEAF;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t bd = sw128_kmajor_desc(b_s + 32 * ks);
              // term i of A meets terms 0 .. TERMS-1-i of B: N = 64 (TERMS - i)
#pragma unroll
              for (int i = 0; i < TERMS; ++i)
                umma_f16(d, sw128_kmajor_desc(a_s + i * 2 * kTerm + 32 * ks), bd,
                         umma_idesc_f16(AB, 128, 64 * (TERMS - i)), (ks == 0 && i == 0) ? 0u : 1u);
            }
            umma_commit(&empty[s]);
            umma_commit(&tfull[b]);
            ++t;
          }
        }
      }
      // leave no MMA in flight: the last accumulator has been written
      if (t > 0) mbar_wait_bounded(&tfull[(t - 1) & 1], (uint32_t)(((t - 1) >> 1) & 1));
    }
  } else {
    // ---------------- epilogue: warps 2..5; TMEM lane = accumulator row
    const int quarter = warp & 3;
    const int lrow = 32 * quarter + lane;
    const int half = lrow >> 6, row = lrow & 63;
    const int te = threadIdx.x - 64;
    int64_t t = 0;
    float acc[64];
    for (int64_t un = blockIdx.x; un < batch.nunits; un += gridDim.x) {
      const int r = plan_of(batch.ubegin, batch.nplans, un);
      const PlanDev& pl = batch.plans[r];
      const int64_t Q = un - batch.ubegin[r];
      bool stop = false;
      for (int pr = 0; pr < 2; ++pr) {
        const int g0 = pl.quads[4 * Q + pr], g1 = pl.quads[4 * Q + 2 + pr];
        if (g0 < 0 && g1 < 0) continue;
        const int g = half ? g1 : g0;
#pragma unroll
        for (int c = 0; c < 64; ++c) acc[c] = 0.f;
        PairCursor cur;
        cur.init(pl.gstart, g0, g1);
        while (cur.more()) {
          bool u0, u1;
          int32_t kb;
          int64_t q0, q1;
          cur.next(pl.tb, &u0, &u1, &kb, &q0, &q1);
          const int b = (int)(t & 1);
          bool ok = true;
          if (lane == 0) ok = mbar_wait_or_abort(&tfull[b], (uint32_t)((t >> 1) & 1), abortp);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          ++t;
          if (!ok) {
            // the epilogue still runs the barrier sequence below, then stops together
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abortp = 1;
            break;
          }
          tc_fence_after();
          float scale = 1.f;
          if constexpr (Cfg::SCALED) {
            const bool mine = half ? u1 : u0;
            if (mine) {
              const int ea = pl.expA[pl.ta[half ? q1 : q0]], eb = pl.expB[kb];
              // 2^-(ea + eb) as a product of two normal powers of two
              scale = __int_as_float((127 - ea) << 23) * __int_as_float((127 - eb) << 23);
            }
          }
          const uint32_t tl = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)b * 256u;
#pragma unroll
          for (int c0 = 0; c0 < 64; c0 += 32) {
            float v[32], w[32];
            tmem_ld32(tl + 64 * (TERMS - 1) + c0, v);
#pragma unroll
            for (int blk = TERMS - 2; blk >= 0; --blk) {
              tmem_ld32(tl + 64 * blk + c0, w);
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] += w[i];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              if constexpr (Cfg::SCALED)
                acc[c0 + i] = fmaf(v[i], scale, acc[c0 + i]);
              else
                acc[c0 + i] += v[i];
            }
          }
          tc_fence_before();
          mbar_arrive(&tempty[b]);
        }
        // output row `row` of leaf g: FP64, and its squared norm
        double s2 = 0.0;
        if (g >= 0) {
          double2* out = reinterpret_cast<double2*>(pl.cpool + (int64_t)g * 4096 + row * 64);
#pragma unroll
          for (int c = 0; c < 64; c += 2) {
            const double x = (double)acc[c], y = (double)acc[c + 1];
            out[c >> 1] = make_double2(x, y);
            s2 = __fma_rn(x, x, s2);
            s2 = __fma_rn(y, y, s2);
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        if (lane == 0) red[quarter] = s2;
        if (te == 0) epi_stop = *abortp;
        named_barrier(1, 128);
        if (te == 0) {
          if (g0 >= 0) pl.csq[g0] = red[0] + red[1];
          if (g1 >= 0) pl.csq[g1] = red[2] + red[3];
        }
        stop = epi_stop != 0;
        named_barrier(1, 128);
        if (stop) break;
      }
      if (stop) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

static unsigned gemm_grid(spamm_ctx ctx, int64_t nunits) {
  int64_t grid = ctx->gemm_sm_limit > 0 ? ctx->gemm_sm_limit : ctx->num_sms;
  if (grid > nunits) grid = nunits;
  return (unsigned)(grid < 1 ? 1 : grid);
}

const uint8_t* zero_term(spamm_ctx ctx) {
  if (!ctx->d_zero) {
    CK(cudaMalloc(&ctx->d_zero, kTerm));
    CK(cudaMemset(ctx->d_zero, 0, kTerm));
  }
  return static_cast<const uint8_t*>(ctx->d_zero);
}

void prep_terms(spamm_mat M, spamm_prec prec, int role, BufP* terms, BufP* expo, spamm_ctx on) {
  spamm_ctx ctx = on ? on : M->ctx;
  if (M->bs != 64) fail(SPAMM_E_UNSUPPORTED, "tensor-core precision forms are built for bs = 64");
  const unsigned pg = (unsigned)(ctx->num_sms * 8);
  if (prec == SPAMM_PREC_BF16_SPLIT) {
    *terms = alloc_n<uint8_t>(ctx, M->nleaves * (int64_t)leaf_bytes<SPAMM_PREC_BF16_SPLIT>());
    if (M->nleaves > 0) {
      prep_bf16_terms_kernel<<<pg, 256, 0, ctx->stream>>>(P<double>(M->pool), P<int64_t>(M->slot), M->nleaves, role,
                                                          P<uint8_t>(*terms));
      CK_LAUNCH("prep_bf16_terms_kernel");
    }
  } else {
    *terms = alloc_n<uint8_t>(ctx, M->nleaves * (int64_t)leaf_bytes<SPAMM_PREC_FP16_SCALED>());
    *expo = alloc_n<int32_t>(ctx, M->nleaves);
    if (M->nleaves > 0) {
      prep_fp16_terms_kernel<<<pg, 256, 0, ctx->stream>>>(P<double>(M->pool), P<int64_t>(M->slot), M->nleaves, role,
                                                          P<uint8_t>(*terms), P<int32_t>(*expo));
      CK_LAUNCH("prep_fp16_terms_kernel");
    }
  }
}

template <int PREC>
static void launch_pairs(spamm_ctx ctx, const BatchDev& b) {
  if (b.nunits == 0) return;
  const size_t smem = pair_smem_bytes<PREC>();
  CK(cudaFuncSetAttribute(gemm_pair_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  gemm_pair_kernel<PREC><<<gemm_grid(ctx, b.nunits), kTcThreads, smem, ctx->stream>>>(b, zero_term(ctx), ctx->d_err);
  CK_LAUNCH("gemm_pair_kernel");
}

void gemm_bf16_batch(spamm_ctx ctx, const BatchDev& b) { launch_pairs<SPAMM_PREC_BF16_SPLIT>(ctx, b); }
void gemm_fp16_batch(spamm_ctx ctx, const BatchDev& b) { launch_pairs<SPAMM_PREC_FP16_SCALED>(ctx, b); }

}  // namespace spamm
