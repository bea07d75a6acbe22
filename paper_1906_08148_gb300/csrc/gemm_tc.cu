// gemm_tc.cu -- kernel (c), tensor-core forms (bs = 64): BF16 three-term split
// and FP16 with per-leaf power-of-two scaling, FP32 accumulation, with the
// C-leaf norms of kernel (d) in the epilogue.
//
// Each leaf product of Algorithm 1 ("C = AB" at the lowest level) is a real
// 64 x 64 x 64 contraction on tcgen05.  Operands are split into low-precision
// terms (a = a0 + a1 + a2 + ..., each term the rounding of what is left):
//   BF16 split : A tile 1 = [a0; a1], A tile 2 = [a2; a3] (128 x 64 each),
//                B tile = [b0^T; b1^T; b2^T] (192 x 64).  MMA 1 (M=128, N=192)
//                forms a_i b_j for i < 2, j < 3; MMA 2 (M=128, N=64) adds
//                a2 b0 and a3 b0 into the first 64 columns.  Every product
//                with i + j <= 2 is present (plus a1 b2, a3 b0).
//   FP16 scaled: a' = a 2^eA with max|a'| in [2^14, 2^15]; A tile = [h0; h1],
//                B tile = [g0^T; g1^T]; one MMA (M=128, N=128); the product
//                is scaled back by 2^-(eA+eB).
// C = sum of the row halves and column blocks of the 128 x N accumulator.
// The tiles are stored in HBM already in the canonical 128-byte-swizzled
// K-major layout, so one 1-D TMA bulk copy per tile lands them in shared
// memory ready for the MMA descriptors.
//
// Warp roles (one CTA per SM, persistent, output leaves g = blockIdx.x +
// k * gridDim.x in Morton order so that concurrently running CTAs share A
// rows and B columns in L2):
//   warp 0     TMA producer: stage ring of NS (A, B) tile sets, mbarriers.
//   warp 1     allocates 512 TMEM columns, issues the MMAs of one leaf
//              product into one of two TMEM accumulators, commits.
//   warps 2-5  drain an accumulator (tcgen05.ld) into FP32 registers (one
//              row of one half per thread), free it, and at the end of an
//              output leaf add the halves, write the FP64 leaf and its
//              squared norm.
// No atomics on C: one CTA owns each output leaf; k runs in task order.
// Every wait is bounded; on timeout the CTA sets the error word and leaves.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace spamm {

constexpr int kTcThreads = 192;
constexpr int kEbufStride = 65;  // padded row of the epilogue staging buffer (floats)

template <int PREC>
struct TcCfg;
template <>
struct TcCfg<SPAMM_PREC_BF16_SPLIT> {
  static constexpr uint32_t A_BYTES = 2 * 128 * 64 * 2;  // [a0;a1] and [a2;a3]
  static constexpr uint32_t B_BYTES = 192 * 64 * 2;      // [b0^T; b1^T; b2^T]
  static constexpr int NBLK = 3;                         // 64-column blocks of the accumulator
  static constexpr int NS = 3;
  static constexpr uint32_t IDESC1 = umma_idesc_f16(1, 128, 192);
  static constexpr uint32_t IDESC2 = umma_idesc_f16(1, 128, 64);
  static constexpr bool SCALED = false;
};
template <>
struct TcCfg<SPAMM_PREC_FP16_SCALED> {
  static constexpr uint32_t A_BYTES = 128 * 64 * 2;  // [h0; h1]
  static constexpr uint32_t B_BYTES = 128 * 64 * 2;  // [g0^T; g1^T]
  static constexpr int NBLK = 2;
  static constexpr int NS = 5;
  static constexpr uint32_t IDESC1 = umma_idesc_f16(0, 128, 128);
  static constexpr uint32_t IDESC2 = 0;
  static constexpr bool SCALED = true;
};

template <int PREC>
constexpr size_t tc_smem_bytes() {
  return 1024 + (size_t)TcCfg<PREC>::NS * (TcCfg<PREC>::A_BYTES + TcCfg<PREC>::B_BYTES) +
         (size_t)128 * kEbufStride * sizeof(float);
}

// Byte offset of element (row, k) in a 128-byte-swizzled K-major tile of
// 64 two-byte elements per row: 16-byte chunk index XOR (row mod 8).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ row) & 7) << 4) + (k & 7) * 2);
}

// ---------------------------------------------------------------- operand prep
// role 0: leaf used as A (rows = output rows, k = columns); role 1: leaf used
// as B (tile rows = output columns n, k = leaf rows).
__global__ void prep_bf16_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot, int64_t nleaves,
                                 int role, uint8_t* __restrict__ out) {
  const uint32_t bytes = role == 0 ? TcCfg<SPAMM_PREC_BF16_SPLIT>::A_BYTES : TcCfg<SPAMM_PREC_BF16_SPLIT>::B_BYTES;
  for (int64_t m = blockIdx.x; m < nleaves; m += gridDim.x) {
    const double* src = pool + slot[m] * 4096;
    uint8_t* dst = out + m * (int64_t)bytes;
    for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
      const int r = e >> 6, c = e & 63;
      const double a = src[e];
      __nv_bfloat16 s[4];
      double rest = a;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        s[i] = __double2bfloat16(rest);
        rest -= (double)__bfloat162float(s[i]);
      }
      if (role == 0) {
        *reinterpret_cast<__nv_bfloat16*>(dst + sw128_offset(r, c)) = s[0];
        *reinterpret_cast<__nv_bfloat16*>(dst + sw128_offset(64 + r, c)) = s[1];
        *reinterpret_cast<__nv_bfloat16*>(dst + 16384 + sw128_offset(r, c)) = s[2];
        *reinterpret_cast<__nv_bfloat16*>(dst + 16384 + sw128_offset(64 + r, c)) = s[3];
      } else {
        // element (k = r, n = c): tile row s*64 + n, column k
#pragma unroll
        for (int i = 0; i < 3; ++i) *reinterpret_cast<__nv_bfloat16*>(dst + sw128_offset(64 * i + c, r)) = s[i];
      }
    }
  }
}

__global__ void prep_fp16_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot, int64_t nleaves,
                                 int role, uint8_t* __restrict__ out, int32_t* __restrict__ expo) {
  __shared__ double smax[8];
  __shared__ int s_e;
  const uint32_t bytes = TcCfg<SPAMM_PREC_FP16_SCALED>::A_BYTES;
  for (int64_t m = blockIdx.x; m < nleaves; m += gridDim.x) {
    const double* src = pool + slot[m] * 4096;
    uint8_t* dst = out + m * (int64_t)bytes;
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
      s_e = t > 0.0 ? 15 - x : 0;  // max |a| 2^e in [2^14, 2^15)
      expo[m] = s_e;
    }
    __syncthreads();
    const int e2 = s_e;
    for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
      const int r = e >> 6, c = e & 63;
      const double a = ldexp(src[e], e2);
      const __half h0 = __double2half(a);
      const __half h1 = __double2half(a - (double)__half2float(h0));
      if (role == 0) {
        *reinterpret_cast<__half*>(dst + sw128_offset(r, c)) = h0;
        *reinterpret_cast<__half*>(dst + sw128_offset(64 + r, c)) = h1;
      } else {
        *reinterpret_cast<__half*>(dst + sw128_offset(c, r)) = h0;
        *reinterpret_cast<__half*>(dst + sw128_offset(64 + c, r)) = h1;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- GEMM
template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 1)
    gemm_tc_kernel(int64_t G, const int64_t* __restrict__ gstart, const int32_t* __restrict__ ta,
                   const int32_t* __restrict__ tb, const uint8_t* __restrict__ sliceA,
                   const uint8_t* __restrict__ sliceB, const int32_t* __restrict__ expA,
                   const int32_t* __restrict__ expB, double* __restrict__ cpool, double* __restrict__ csq,
                   int* __restrict__ err) {
  using Cfg = TcCfg<PREC>;
  constexpr int NS = Cfg::NS;
  constexpr uint32_t STAGE = Cfg::A_BYTES + Cfg::B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* ebuf = reinterpret_cast<float*>(smem + NS * STAGE);
  __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
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
      for (int64_t g = blockIdx.x; g < G && !*abortp; g += gridDim.x) {
        const int64_t q1 = gstart[g + 1];
        for (int64_t q = gstart[g]; q < q1; ++q, ++t) {
          const int s = (int)(t % NS);
          const int64_t u = t / NS;
          if (u > 0 && !mbar_wait_or_abort(&empty[s], (uint32_t)((u - 1) & 1), abortp)) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abortp = 1;
            break;
          }
          uint8_t* st = smem + s * STAGE;
          mbar_arrive_expect_tx(&full[s], STAGE);
          bulk_g2s(st, sliceA + (int64_t)ta[q] * Cfg::A_BYTES, Cfg::A_BYTES, &full[s]);
          bulk_g2s(st + Cfg::A_BYTES, sliceB + (int64_t)tb[q] * Cfg::B_BYTES, Cfg::B_BYTES, &full[s]);
        }
      }
      // leave no bulk copy in flight: the last fill of every stage has landed
      for (int64_t k = (t > NS ? t - NS : 0); k < t; ++k) mbar_wait_bounded(&full[k % NS], (uint32_t)((k / NS) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int64_t t = 0;
      for (int64_t g = blockIdx.x; g < G && !*abortp; g += gridDim.x) {
        const int64_t q1 = gstart[g + 1];
        for (int64_t q = gstart[g]; q < q1; ++q, ++t) {
          const int s = (int)(t % NS);
          const int b = (int)(t & 1);
          if (!mbar_wait_or_abort(&full[s], (uint32_t)((t / NS) & 1), abortp) ||
              (t >= 2 && !mbar_wait_or_abort(&tempty[b], (uint32_t)(((t >> 1) - 1) & 1), abortp))) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abortp = 1;
            break;
          }
          tc_fence_after();
          const uint32_t d = tbase + (uint32_t)b * 256u;
          const uint32_t a_s = smem_u32(smem + s * STAGE), b_s = a_s + Cfg::A_BYTES;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            umma_f16(d, sw128_kmajor_desc(a_s + 32 * ks), sw128_kmajor_desc(b_s + 32 * ks), Cfg::IDESC1,
                     ks > 0 ? 1u : 0u);
          if constexpr (PREC == SPAMM_PREC_BF16_SPLIT) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              umma_f16(d, sw128_kmajor_desc(a_s + 16384 + 32 * ks), sw128_kmajor_desc(b_s + 32 * ks), Cfg::IDESC2,
                       1u);
          }
          umma_commit(&empty[s]);
          umma_commit(&tfull[b]);
        }
      }
      // leave no MMA in flight: the last accumulator has been written
      if (t > 0) mbar_wait_bounded(&tfull[(t - 1) & 1], (uint32_t)(((t - 1) >> 1) & 1));
    }
  } else {
    // ---------------- epilogue: warps 2..5, TMEM lanes 32*(warp%4)..+31
    const int quarter = warp & 3;
    const int lrow = 32 * quarter + lane;  // accumulator row = TMEM lane
    const int te = threadIdx.x - 64;       // 0..127
    __shared__ int epi_stop;
    float acc[64];
    int64_t t = 0;
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
      const int64_t q0 = gstart[g], q1 = gstart[g + 1];
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = 0.f;
      for (int64_t q = q0; q < q1; ++q, ++t) {
        const int b = (int)(t & 1);
        if (!mbar_wait_or_abort(&tfull[b], (uint32_t)((t >> 1) & 1), abortp)) {
          // the whole epilogue still runs the barrier sequence below, then stops together
          atomicOr(err, DEV_ERR_TIMEOUT);
          *abortp = 1;
          break;
        }
        tc_fence_after();
        float sa = 1.f, sb = 1.f;
        if constexpr (Cfg::SCALED) {
          sa = __int_as_float((127 - expA[ta[q]]) << 23);
          sb = __int_as_float((127 - expB[tb[q]]) << 23);
        }
        const uint32_t tl = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)b * 256u;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float v[32], w[32];
          tmem_ld32(tl + 32 * half, v);
#pragma unroll
          for (int blk = 1; blk < Cfg::NBLK; ++blk) {
            tmem_ld32(tl + 64 * blk + 32 * half, w);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += w[i];
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if constexpr (Cfg::SCALED)
              acc[32 * half + i] += (v[i] * sa) * sb;
            else
              acc[32 * half + i] += v[i];
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[b]);
      }
      // combine the two row halves of the accumulator, write the FP64 leaf
      float* eb = ebuf + lrow * kEbufStride;
#pragma unroll
      for (int c = 0; c < 64; ++c) eb[c] = acc[c];
      named_barrier(1, 128);
      double* C = cpool + g * 4096;
      double s2 = 0.0;
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        const int idx = te + 128 * i, r = idx >> 6, c = idx & 63;
        const double val = (double)ebuf[r * kEbufStride + c] + (double)ebuf[(64 + r) * kEbufStride + c];
        C[idx] = val;
        s2 = __fma_rn(val, val, s2);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      if (lane == 0) red[warp - 2] = s2;
      if (te == 0) epi_stop = *abortp;
      named_barrier(1, 128);
      if (te == 0) csq[g] = ((red[0] + red[1]) + red[2]) + red[3];
      const bool stop = epi_stop != 0;
      named_barrier(1, 128);
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

template <int PREC>
static void launch_tc(spamm_mat A, spamm_mat B, const TaskList& T, double* cpool, double* csq) {
  spamm_ctx ctx = A->ctx;
  using Cfg = TcCfg<PREC>;
  BufP sa = alloc_n<uint8_t>(ctx, A->nleaves * (int64_t)Cfg::A_BYTES);
  BufP sb = alloc_n<uint8_t>(ctx, B->nleaves * (int64_t)Cfg::B_BYTES);
  BufP ea, eb;
  const unsigned pg = (unsigned)(ctx->num_sms * 8);
  if (PREC == SPAMM_PREC_BF16_SPLIT) {
    prep_bf16_kernel<<<pg, 256, 0, ctx->stream>>>(P<double>(A->pool), P<int64_t>(A->slot), A->nleaves, 0,
                                                  P<uint8_t>(sa));
    CK_LAUNCH("prep_bf16_kernel");
    prep_bf16_kernel<<<pg, 256, 0, ctx->stream>>>(P<double>(B->pool), P<int64_t>(B->slot), B->nleaves, 1,
                                                  P<uint8_t>(sb));
    CK_LAUNCH("prep_bf16_kernel");
  } else {
    ea = alloc_n<int32_t>(ctx, A->nleaves);
    eb = alloc_n<int32_t>(ctx, B->nleaves);
    prep_fp16_kernel<<<pg, 256, 0, ctx->stream>>>(P<double>(A->pool), P<int64_t>(A->slot), A->nleaves, 0,
                                                  P<uint8_t>(sa), P<int32_t>(ea));
    CK_LAUNCH("prep_fp16_kernel");
    prep_fp16_kernel<<<pg, 256, 0, ctx->stream>>>(P<double>(B->pool), P<int64_t>(B->slot), B->nleaves, 1,
                                                  P<uint8_t>(sb), P<int32_t>(eb));
    CK_LAUNCH("prep_fp16_kernel");
  }
  const size_t smem = tc_smem_bytes<PREC>();
  CK(cudaFuncSetAttribute(gemm_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t grid = ctx->num_sms;
  if (grid > T.ngroups) grid = T.ngroups;
  gemm_tc_kernel<PREC><<<(unsigned)grid, kTcThreads, smem, ctx->stream>>>(
      T.ngroups, P<int64_t>(T.gstart), P<int32_t>(T.ta), P<int32_t>(T.tb), P<uint8_t>(sa), P<uint8_t>(sb),
      P<int32_t>(ea), P<int32_t>(eb), cpool, csq, ctx->d_err);
  CK_LAUNCH("gemm_tc_kernel");
}

void gemm_tc(spamm_mat A, spamm_mat B, const TaskList& T, spamm_prec prec, double* cpool, double* csq) {
  if (T.ngroups == 0) return;
  if (A->bs != 64) fail(SPAMM_E_UNSUPPORTED, "tensor-core precision forms are built for bs = 64");
  if (prec == SPAMM_PREC_BF16_SPLIT)
    launch_tc<SPAMM_PREC_BF16_SPLIT>(A, B, T, cpool, csq);
  else
    launch_tc<SPAMM_PREC_FP16_SCALED>(A, B, T, cpool, csq);
}

}  // namespace spamm
