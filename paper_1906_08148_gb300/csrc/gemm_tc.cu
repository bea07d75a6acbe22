// gemm_tc.cu -- kernel (c), tensor-core forms (bs = 64): BF16 three-term split
// and FP16 with per-leaf power-of-two scaling, FP32 accumulation, with the
// C-leaf norms of kernel (d) in the epilogue.
//
// Each leaf product of Algorithm 1 ("C = AB" at the lowest level) is a real
// 64 x 64 x 64 contraction on tcgen05.  Operands are split (prep.cu, layout in
// tcforms.cuh) into low-precision terms, each the rounding of what the
// previous terms left:
//   BF16 split : a = a0 + a1 + a2, b = b0 + b1 + b2 (bf16); the six products
//                with term-index sum <= 2 are formed.
//   FP16 scaled: a' = a 2^eA with max|a'| in [2^14, 2^15) per leaf,
//                a' = h0 + h1 (f16), likewise b'; products h0 g0, h0 g1, h1 g0,
//                scaled back by 2^-(eA + eB).
//
// Quads.  The four output leaves (2I + h, 2J + c) of a quadtree node one level
// above the leaves are computed together: at each k the A operand of term s is
// [A(2I,k)_s; A(2I+1,k)_s] (M = 128) and the B operand of term t is
// [B(k,2J)_t | B(k,2J+1)_t] (N = 128), so one step loads two A and two B leaves
// for up to four leaf products.  The steps of each quad (the four kept-product
// runs merged by k, with the leaves to load and each child's scale) are listed
// at plan time, so the kernel reads them sequentially.  A product whose norm
// test failed (or whose leaf is absent) is still formed by the MMA over the
// whole tile, but its quadrant is discarded by the epilogue; an operand leaf no
// kept product of the step needs is not loaded (its stale contents reach only
// discarded quadrants: each output element depends on one A row and one B
// column).  All term products of a step accumulate, smallest first, into one
// fresh 128 x 128 TMEM accumulator; four accumulators rotate, and the epilogue
// drains each step into FP32 registers with round-to-nearest adds (scale
// applied per step), which keeps the error of long k runs at the level of one
// step.
//
// Warp roles (one CTA per SM, persistent; quads are claimed one at a time
// from a global counter in Morton order, so the quads in flight on all SMs
// form one narrow window whose A rows and B columns are shared in L2):
//   warp 0     TMA producer: claims the next quad for all roles (a ring of 4
//              in shared memory), ring of NS stages, 8 KB 1-D bulk copies of
//              pre-swizzled term tiles, mbarriers.
//   warp 1     allocates 512 TMEM columns and issues the MMAs of each step.
//   warps 2-9  epilogue: warps 2-5 column 0, warps 6-9 column 1; TMEM lane =
//              output row; writes the FP64 output leaves and their squared norms.
// No atomics on C: one CTA owns each output quad; k runs in ascending order.
// Every wait is bounded; on timeout the CTA sets the error word and leaves.
#include "internal.cuh"
#include "ptx.cuh"
#include "tcforms.cuh"

namespace spamm {

// ------------------------------------------------------------------- GEMM
constexpr int kQuadThreads = 320;
constexpr int kQuadBufs = 4;  // rotating TMEM accumulators of 128 FP32 columns
constexpr int kQuadQ = 4;     // ring of claimed quads shared by the three roles
template <int PREC>
__host__ __device__ constexpr uint32_t quad_stage_bytes() {
  return 4 * leaf_bytes<PREC>();  // two A and two B leaves, every term
}
template <int PREC>
constexpr size_t quad_smem_bytes() {
  return 1024 + (size_t)FormCfg<PREC>::NS * quad_stage_bytes<PREC>();
}

double quad_step_flops(spamm_prec prec) {
  const int terms = prec == SPAMM_PREC_BF16_SPLIT ? 3 : 2;
  return (double)(terms * (terms + 1) / 2) * 2.0 * 128.0 * 128.0 * 64.0;
}

// Stage layout: A region, term s at s * 16 KB = [A(2I,k)_s; A(2I+1,k)_s]
// (128 rows of 64 k); B region at TERMS * 16 KB, term t at t * 16 KB =
// [B(k,2J)_t; B(k,2J+1)_t] (128 rows n of 64 k).  Both are 128-row K-major
// SW128 operands.
template <int PREC>
__global__ void __launch_bounds__(kQuadThreads, 1)
    gemm_quad_kernel(BatchDev batch, unsigned long long* __restrict__ work, int* __restrict__ err) {
  using Cfg = FormCfg<PREC>;
  constexpr int NS = Cfg::NS, TERMS = Cfg::TERMS, NB = kQuadBufs;
  constexpr uint32_t LEAF = leaf_bytes<PREC>(), STAGE = quad_stage_bytes<PREC>(), BREG = 2 * LEAF;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[NB], tempty[NB], qfull[kQuadQ], qempty[kQuadQ];
  __shared__ int64_t qid[kQuadQ], epi_un;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, epi_stop;
  __shared__ double red[2][4];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 256);
    }
    for (int q = 0; q < kQuadQ; ++q) {
      mbar_init(&qfull[q], 1);
      mbar_init(&qempty[q], 2);  // the MMA issuer and the epilogue's first thread
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
    // ---------------- TMA producer; claims the quads (Morton order, first come first served) for all roles
    if (lane == 0) {
      int64_t t = 0;
      bool stop = false;
      for (int64_t c = 0; !stop; ++c) {
        const int qs = (int)(c % kQuadQ);
        if (c >= kQuadQ && !mbar_wait_or_abort(&qempty[qs], (uint32_t)(((c / kQuadQ) - 1) & 1), abortp)) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          *abortp = 1;
          break;
        }
        const int64_t claimed = (int64_t)atomicAdd(work, 1ull);
        const int64_t un = claimed < batch.nunits ? claimed : -1;
        qid[qs] = un;
        mbar_arrive(&qfull[qs]);
        if (un < 0) break;
        const int r = plan_of(batch.ubegin, batch.nplans, un);
        const PlanDev& pl = batch.plans[r];
        const int64_t Q = un - batch.ubegin[r];
        const int64_t j1 = pl.qstart[Q + 1];
        int64_t j = pl.qstart[Q];
        const int4* rec = reinterpret_cast<const int4*>(pl.qsteps);  // word 2j: a0, a1, b0, b1 of step j
        int4 nx = j < j1 ? __ldg(rec + 2 * j) : make_int4(-1, -1, -1, -1);
        for (; j < j1; ++j) {
          const int4 ab = nx;
          if (j + 1 < j1) nx = __ldg(rec + 2 * (j + 1));  // next step's leaves, in flight during the wait
          const int s = (int)(t % NS);
          if (t >= NS && !mbar_wait_or_abort(&empty[s], (uint32_t)(((t / NS) - 1) & 1), abortp)) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abortp = 1;
            stop = true;
            break;
          }
          uint8_t* st = smem + s * STAGE;
          const uint32_t nload = (uint32_t)((ab.x >= 0) + (ab.y >= 0) + (ab.z >= 0) + (ab.w >= 0));
          mbar_arrive_expect_tx(&full[s], nload * LEAF);
#pragma unroll
          for (int term = 0; term < TERMS; ++term) {
            uint8_t* sa = st + term * 2 * kTerm;
            uint8_t* sb = st + BREG + term * 2 * kTerm;
            if (ab.x >= 0) bulk_g2s(sa, pl.termsA + (int64_t)ab.x * LEAF + term * kTerm, kTerm, &full[s]);
            if (ab.y >= 0) bulk_g2s(sa + kTerm, pl.termsA + (int64_t)ab.y * LEAF + term * kTerm, kTerm, &full[s]);
            if (ab.z >= 0) bulk_g2s(sb, pl.termsB + (int64_t)ab.z * LEAF + term * kTerm, kTerm, &full[s]);
            if (ab.w >= 0) bulk_g2s(sb + kTerm, pl.termsB + (int64_t)ab.w * LEAF + term * kTerm, kTerm, &full[s]);
          }
          ++t;
        }
      }
      // leave no bulk copy in flight: the last fill of every stage has landed
      for (int64_t k = (t > NS ? t - NS : 0); k < t; ++k) mbar_wait_bounded(&full[k % NS], (uint32_t)((k / NS) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: every term product of a step into accumulator t % NB
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc_f16(Cfg::AB, 128, 128);
      int64_t t = 0;
      bool stop = false;
      for (int64_t c = 0; !stop; ++c) {
        const int qs = (int)(c % kQuadQ);
        if (!mbar_wait_or_abort(&qfull[qs], (uint32_t)((c / kQuadQ) & 1), abortp)) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          *abortp = 1;
          break;
        }
        const int64_t un = qid[qs];
        mbar_arrive(&qempty[qs]);
        if (un < 0) break;
        const int r = plan_of(batch.ubegin, batch.nplans, un);
        const PlanDev& pl = batch.plans[r];
        const int64_t Q = un - batch.ubegin[r];
        const int64_t nstep = pl.qstart[Q + 1] - pl.qstart[Q];
        for (int64_t j = 0; j < nstep; ++j) {
          const int s = (int)(t % NS);
          const int b = (int)(t % NB);
          if (!mbar_wait_or_abort(&full[s], (uint32_t)((t / NS) & 1), abortp) ||
              (t >= NB && !mbar_wait_or_abort(&tempty[b], (uint32_t)(((t / NB) - 1) & 1), abortp))) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abortp = 1;
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t d = tbase + (uint32_t)b * 128u;
          const uint32_t a_s = smem_u32(smem + s * STAGE), b_s = a_s + BREG;
          uint32_t accumulate = 0u;
          // term products (i, sum - i), smallest term-index sum first
#pragma unroll
          for (int sum = TERMS - 1; sum >= 0; --sum) {
#pragma unroll
            for (int i = sum; i >= 0; --i) {
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                umma_f16(d, sw128_kmajor_desc(a_s + i * 2 * kTerm + 32 * ks),
                         sw128_kmajor_desc(b_s + (sum - i) * 2 * kTerm + 32 * ks), idesc, accumulate);
                accumulate = 1u;
              }
            }
          }
          umma_commit(&empty[s]);
          umma_commit(&tfull[b]);
          ++t;
        }
      }
      // leave no MMA in flight: the last accumulator has been written
      if (t > 0) mbar_wait_bounded(&tfull[(t - 1) % NB], (uint32_t)(((t - 1) / NB) & 1));
    }
  } else {
    // ---------------- epilogue: warps 2..9; column c = (warp - 2) / 4; TMEM lane = output row
    const int col = (warp - 2) >> 2;
    const int quarter = warp & 3;
    const int lrow = 32 * quarter + lane;
    const int half = lrow >> 6, row = lrow & 63;
    const int child = 2 * half + col;  // warp-uniform
    const int te = threadIdx.x - 64;   // 0..255
    int64_t t = 0;
    float acc[64];
    for (int64_t c = 0;; ++c) {
      // one thread takes the next claimed quad for all 256 (-2: the wait gave up)
      if (te == 0) {
        const int qs = (int)(c % kQuadQ);
        if (mbar_wait_or_abort(&qfull[qs], (uint32_t)((c / kQuadQ) & 1), abortp)) {
          epi_un = qid[qs];
          mbar_arrive(&qempty[qs]);
        } else {
          epi_un = -2;
        }
      }
      named_barrier(2, 256);
      const int64_t un = epi_un;  // rewritten only after the two barriers that end this quad
      if (un < 0) {
        if (un == -2 && te == 0) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          *abortp = 1;
        }
        break;
      }
      const int r = plan_of(batch.ubegin, batch.nplans, un);
      const PlanDev& pl = batch.plans[r];
      const int64_t Q = un - batch.ubegin[r];
      const int32_t g[4] = {pl.quads[4 * Q], pl.quads[4 * Q + 1], pl.quads[4 * Q + 2], pl.quads[4 * Q + 3]};
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = 0.f;
      const int64_t j1 = pl.qstart[Q + 1];
      int64_t j = pl.qstart[Q];
      float sc_next = j < j1 ? __ldg(&pl.qsteps[j].scale[child]) : 0.f;
      for (; j < j1; ++j) {
        const float sc = sc_next;
        if (j + 1 < j1) sc_next = __ldg(&pl.qsteps[j + 1].scale[child]);
        const int b = (int)(t % NB);
        bool ok = true;
        if (lane == 0) ok = mbar_wait_or_abort(&tfull[b], (uint32_t)((t / NB) & 1), abortp);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        ++t;
        if (!ok) {
          // the epilogue still runs the barrier sequence below, then stops together
          atomicOr(err, DEV_ERR_TIMEOUT);
          *abortp = 1;
          break;
        }
        tc_fence_after();
        if (sc != 0.f) {  // this warp's child has a kept product at this k
          float v[64];
          tmem_ld64(tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)b * 128u + 64u * (uint32_t)col, v);
#pragma unroll
          for (int i = 0; i < 64; ++i) acc[i] = fmaf(v[i], sc, acc[i]);
        }
        tc_fence_before();
        mbar_arrive(&tempty[b]);
      }
      // output row `row` of leaf g[child]: FP64, and its squared norm
      const int gl = g[child];
      double s2 = 0.0;
      if (gl >= 0) {
        double2* out = reinterpret_cast<double2*>(pl.cpool + (int64_t)gl * 4096 + row * 64);
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
      if (lane == 0) red[col][quarter] = s2;
      if (te == 0) epi_stop = *abortp;
      named_barrier(1, 256);
      if (te < 4) {
        const int cc = te & 1, hh = te >> 1;  // child 2 hh + cc: its rows are quarters 2 hh, 2 hh + 1
        if (g[2 * hh + cc] >= 0) pl.csq[g[2 * hh + cc]] = red[cc][2 * hh] + red[cc][2 * hh + 1];
      }
      const bool stop = epi_stop != 0;
      named_barrier(1, 256);
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

template <int PREC>
static void launch_quads(spamm_ctx ctx, const BatchDev& b) {
  if (b.nunits == 0) return;
  const size_t smem = quad_smem_bytes<PREC>();
  CK(cudaFuncSetAttribute(gemm_quad_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned long long* work = ctx->d_scratch + 9;  // quad claim counter
  CK(cudaMemsetAsync(work, 0, sizeof(unsigned long long), ctx->stream));
  gemm_quad_kernel<PREC><<<gemm_grid(ctx, b.nunits), kQuadThreads, smem, ctx->stream>>>(b, work, ctx->d_err);
  CK_LAUNCH("gemm_quad_kernel");
}

void gemm_bf16_batch(spamm_ctx ctx, const BatchDev& b) { launch_quads<SPAMM_PREC_BF16_SPLIT>(ctx, b); }
void gemm_fp16_batch(spamm_ctx ctx, const BatchDev& b) { launch_quads<SPAMM_PREC_FP16_SCALED>(ctx, b); }

}  // namespace spamm
