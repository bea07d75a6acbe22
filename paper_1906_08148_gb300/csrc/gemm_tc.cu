// gemm_tc.cu -- kernel (c), tensor-core forms (bs = 64 and 128): BF16 error-free
// slice splits (3 or 4 slices) and FP16 with per-leaf power-of-two scaling;
// and their kernel (d), the pass that finishes the output leaves in FP64 and
// takes their norms.
//
// Each leaf product of Algorithm 1 ("C = AB" at the lowest level) is a real
// 64 x 64 x 64 contraction on tcgen05.  Operands are split at plan time
// (prep.cu, layout in tcforms.cuh):
//   BF16 split : every row of an A leaf and column of a B leaf as S = 3 or 4
//                BF16 slices on a grid set by the line's largest element
//                (slices.cuh); the slice products with index sum < S are
//                formed.  For one output element the products of one index
//                sum are integers on a common grid, so the K = 64 sum of
//                index sum 0 (and 1 for S = 4) is exact in its own FP32
//                accumulator; the smaller rest shares one accumulator.
//   FP16 scaled: a' = a 2^eA with max|a'| in [2^14, 2^15) per leaf,
//                a' = h0 + h1 (f16), likewise b'; products h0 g0, h0 g1, h1 g0
//                into one accumulator.
// Every step's accumulators are scaled back by the step's power of two
// (exact) and drained into registers: the FP16 form adds them to one FP32
// accumulator per output element; the BF16 forms keep a two-float (hi + lo)
// accumulator, adding each exact accumulator with an error-free TwoSum and
// the rest into lo.  The epilogue stores the pairs as they are; the finishing
// pass writes hi + lo in FP64 and the leaf norms, away from the GEMM, because
// this part issues FP64 instructions at two per clock per SM and an epilogue
// busy with them stops draining the accumulators the next MMAs need.
//
// 128 x 128 leaves.  A unit is one output leaf; its four 64 x 64 quadrants
// are the children, and every kept product runs as two K-half steps over the
// tile-split operand terms (prep.cu, steps.cu): the same steps and MMAs.
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
// column).  The 4-slice form stages each step in two K-halves (64 KB each,
// three in flight) so that its 128 KB of operands per step still pipeline.
// Accumulators are 128 x 128 FP32 slots of TMEM; four slots rotate, one per
// accumulator of each step in order, so the MMAs of the next step start as
// soon as the epilogue has drained the slots they reuse.
//
// Warp roles (one CTA per SM, persistent; quads are claimed one at a time
// from a global counter in Morton order, so the quads in flight on all SMs
// form one narrow window whose A rows and B columns are shared in L2):
//   warp 0     TMA producer: claims the next quad for all roles (a ring of 4
//              in shared memory), ring of NS stages, one 1-D bulk copy per
//              leaf and stage (the leaf's K-part with all its pre-swizzled,
//              atom-interleaved terms), mbarriers.
//   warp 1     allocates 512 TMEM columns and issues the MMAs of each step.
//   warps 2-3  idle (they fill the first warpgroup, see the register split)
//   warps 4-11 epilogue: warps 4-7 column 0, warps 8-11 column 1; TMEM lane =
//              output row (warp w reads lanes 32 (w mod 4) ..); writes the
//              output rows as two-float pairs.
// No atomics on C: one CTA owns each output quad; k runs in ascending order.
// Every wait is bounded; on timeout the CTA sets the error word and leaves.
#include "convert.cuh"
#include "internal.cuh"
#include "ptx.cuh"
#include "tcforms.cuh"

namespace spamm {

// ------------------------------------------------------------------- GEMM
// Three warpgroups: warpgroup 0 holds the producer (warp 0) and the MMA issuer
// (warp 1; warps 2-3 idle), warpgroups 1-2 the epilogue (warps 4-11).  The
// launch gives every thread 168 registers (384 x 168 = 64512 of 65536); the
// control warpgroup then gives up 112 of them per thread and the epilogue
// takes 56 more, enough for its two-float accumulators: 128 x 56 + 256 x 224
// = 64512, the launch total, so the increase never waits.
constexpr int kQuadThreads = 384;
constexpr uint32_t kLaunchRegs = 168, kCtlRegs = 56, kEpiRegs = 224;
static_assert(128 * kCtlRegs + 256 * kEpiRegs == kQuadThreads * kLaunchRegs, "register split must match the launch");
static_assert(kQuadThreads * kLaunchRegs <= 65536, "launch registers exceed the register file");
constexpr int kQuadBufs = 4;  // rotating TMEM accumulator slots of 128 FP32 columns
constexpr int kQuadQ = 4;     // ring of claimed quads shared by the three roles

// One stage: two A and two B leaves, every term of a step (whole-K forms) or
// of one K-part of it.  A region: leaf 2I's part (all terms, atom-interleaved,
// tcforms.cuh) then leaf 2I+1's; B region at BREG: leaves 2J, 2J+1 likewise.
// Term s of the 128-row A operand [A(2I,k)_s; A(2I+1,k)_s] starts at s x atom
// with TERMS x atom between 8-row groups, and the same for B.
template <int PREC>
struct QuadLayout {
  using Cfg = FormCfg<PREC>;
  static constexpr uint32_t TILE = kTerm / Cfg::KPARTS;            // one term's part of one leaf
  static constexpr uint32_t LPART = (uint32_t)Cfg::TERMS * TILE;   // one leaf's part, all terms
  static constexpr uint32_t ATOM = term_atom<Cfg::KPARTS>();
  static constexpr uint32_t SBO = (uint32_t)Cfg::TERMS * ATOM;
  static constexpr int SPS = Cfg::KPARTS;      // stages per step
  static constexpr int KS = 4 / Cfg::KPARTS;   // K = 16 MMAs per stage
  static constexpr uint32_t BREG = 2 * LPART;
  static constexpr uint32_t STAGE = 2 * BREG;
  static constexpr size_t SMEM = 1024 + (size_t)Cfg::NS * STAGE;
  __device__ static uint64_t desc(uint32_t saddr) {
    if constexpr (Cfg::KPARTS == 1) return sw128_kmajor_desc(saddr, SBO);
    if constexpr (Cfg::KPARTS == 2) return sw64_kmajor_desc(saddr, SBO);
    return sw32_kmajor_desc(saddr, SBO);
  }
};

double quad_step_flops(spamm_prec prec) {
  const int terms = prec == SPAMM_PREC_BF16_SPLIT ? 3 : (prec == SPAMM_PREC_BF16_SPLIT4 ? 4 : 2);
  return (double)(terms * (terms + 1) / 2) * 2.0 * 128.0 * 128.0 * 64.0;
}

// The MMAs of accumulator `acc` for one stage: term products (i, g - i) with
// index sum g = acc (g from acc to TERMS - 1 for the last accumulator, the
// largest sums first so the smallest products are added first), the first
// of them overwriting the slot when `fresh`.
template <int PREC, int ACC>
__device__ __forceinline__ void issue_acc(uint32_t d, uint32_t a_s, uint32_t b_s, uint32_t idesc, bool fresh) {
  using Cfg = FormCfg<PREC>;
  using Lay = QuadLayout<PREC>;
  constexpr int GLO = ACC, GHI = ACC < Cfg::NACC - 1 ? ACC : Cfg::TERMS - 1;
  uint32_t accumulate = fresh ? 0u : 1u;
#pragma unroll
  for (int g = GHI; g >= GLO; --g) {
#pragma unroll
    for (int i = g; i >= 0; --i) {
#pragma unroll
      for (int ks = 0; ks < Lay::KS; ++ks) {
        umma_f16(d, Lay::desc(a_s + (uint32_t)i * Lay::ATOM + 32 * ks),
                 Lay::desc(b_s + (uint32_t)(g - i) * Lay::ATOM + 32 * ks), idesc, accumulate);
        accumulate = 1u;
      }
    }
  }
}

// (hi, lo) += x sc for two adjacent output elements at once, with an
// error-free TwoSum of hi and x sc (x sc is exact: sc is a power of two) in
// the packed FP32x2 instructions, each lane rounding like the scalar
// round-to-nearest operation: hi + lo gains x sc up to the rounding of lo.
// hi2, lo2 hold (hi, lo) of elements 2q and 2q + 1; v0, v1 are the
// accumulator's FP32 bits of the two elements, sc2 the scale twice.
__device__ __forceinline__ void two_sum_x2(uint64_t& hi2, uint64_t& lo2, uint32_t v0, uint32_t v1, uint64_t sc2) {
  asm("{\n\t.reg .b64 x, s, bp, t1, t2, t3, e;\n\t"
      "mov.b64 x, {%2, %3};\n\t"
      "mul.rn.f32x2 x, x, %4;\n\t"
      "add.rn.f32x2 s, %0, x;\n\t"
      "sub.rn.f32x2 bp, s, %0;\n\t"
      "sub.rn.f32x2 t1, s, bp;\n\t"
      "sub.rn.f32x2 t2, %0, t1;\n\t"
      "sub.rn.f32x2 t3, x, bp;\n\t"
      "add.rn.f32x2 e, t2, t3;\n\t"
      "add.rn.f32x2 %1, %1, e;\n\t"
      "mov.b64 %0, s;\n\t}"
      : "+l"(hi2), "+l"(lo2)
      : "r"(v0), "r"(v1), "l"(sc2));
}
// lo2 += (v0, v1) sc2, packed.
__device__ __forceinline__ void fma_x2(uint64_t& lo2, uint32_t v0, uint32_t v1, uint64_t sc2) {
  asm("{\n\t.reg .b64 x;\n\t"
      "mov.b64 x, {%1, %2};\n\t"
      "fma.rn.f32x2 %0, x, %3, %0;\n\t}"
      : "+l"(lo2)
      : "r"(v0), "r"(v1), "l"(sc2));
}

template <int PREC>
__global__ void __launch_bounds__(kQuadThreads, 1)
    gemm_quad_kernel(BatchDev batch, unsigned long long* __restrict__ work, int* __restrict__ err) {
  using Cfg = FormCfg<PREC>;
  using Lay = QuadLayout<PREC>;
  constexpr int NS = Cfg::NS, TERMS = Cfg::TERMS, NACC = Cfg::NACC, NB = kQuadBufs, SPS = Lay::SPS;
  constexpr uint32_t LEAF = leaf_bytes<PREC>(), STAGE = Lay::STAGE, BREG = Lay::BREG, TILE = Lay::TILE;
  static_assert(NACC <= NB - 1, "the next step needs a free accumulator slot");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[NB], tempty[NB], qfull[kQuadQ], qempty[kQuadQ];
  __shared__ int64_t qid[kQuadQ], epi_un;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, epi_stop;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);  // the eight epilogue warps, one arrival each
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
  if (warp < 4) {
    regs_dec<kCtlRegs>();  // every warp of warpgroup 0, at this one instruction
  if (warp == 0) {
    // ---------------- TMA producer; claims the quads (Morton order, first come first served) for all roles
    if (lane == 0) {
      int64_t t = 0;  // stages filled
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
        const int64_t Qc = un - batch.ubegin[r], Q = pl.uorder ? pl.uorder[Qc] : pl.ufirst + Qc;
        const int64_t j1 = pl.qstart[Q + 1];
        int64_t j = pl.qstart[Q];
        const int4* rec = reinterpret_cast<const int4*>(pl.qsteps);  // word 2j: a0, a1, b0, b1 of step j
        int4 nx = j < j1 ? __ldg(rec + 2 * j) : make_int4(-1, -1, -1, -1);
        for (; j < j1 && !stop; ++j) {
          const int4 ab = nx;
          if (j + 1 < j1) nx = __ldg(rec + 2 * (j + 1));  // next step's leaves, in flight during the wait
          const uint32_t nload = (uint32_t)((ab.x >= 0) + (ab.y >= 0) + (ab.z >= 0) + (ab.w >= 0));
#pragma unroll
          for (int h = 0; h < SPS; ++h) {
            const int s = (int)(t % NS);
            if (t >= NS && !mbar_wait_or_abort(&empty[s], (uint32_t)(((t / NS) - 1) & 1), abortp)) {
              atomicOr(err, DEV_ERR_TIMEOUT);
              *abortp = 1;
              stop = true;
              break;
            }
            uint8_t* st = smem + s * STAGE;
            constexpr uint32_t LP = Lay::LPART;
            mbar_arrive_expect_tx(&full[s], nload * LP);
            // one copy per leaf: its part h, every term
            const int64_t off = (int64_t)h * LP;
            if (ab.x >= 0) bulk_g2s(st, pl.termsA + (int64_t)ab.x * LEAF + off, LP, &full[s]);
            if (ab.y >= 0) bulk_g2s(st + LP, pl.termsA + (int64_t)ab.y * LEAF + off, LP, &full[s]);
            if (ab.z >= 0) bulk_g2s(st + BREG, pl.termsB + (int64_t)ab.z * LEAF + off, LP, &full[s]);
            if (ab.w >= 0) bulk_g2s(st + BREG + LP, pl.termsB + (int64_t)ab.w * LEAF + off, LP, &full[s]);
            ++t;
          }
        }
      }
      // leave no bulk copy in flight: the last fill of every stage has landed
      for (int64_t k = (t > NS ? t - NS : 0); k < t; ++k) mbar_wait_bounded(&full[k % NS], (uint32_t)((k / NS) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the accumulators of step number n are slots (NACC n + a) % NB
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc_f16(Cfg::AB, 128, 128);
      int64_t t = 0, u = 0;  // stages consumed, accumulator units started
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
        const int64_t Qc = un - batch.ubegin[r], Q = pl.uorder ? pl.uorder[Qc] : pl.ufirst + Qc;
        const int64_t nstep = pl.qstart[Q + 1] - pl.qstart[Q];
        for (int64_t j = 0; j < nstep && !stop; ++j) {
#pragma unroll
          for (int h = 0; h < SPS; ++h) {
            const int s = (int)(t % NS);
            if (!mbar_wait_or_abort(&full[s], (uint32_t)((t / NS) & 1), abortp)) {
              stop = true;
              break;
            }
            tc_fence_after();
            const uint32_t a_s = smem_u32(smem + s * STAGE), b_s = a_s + BREG;
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
              const int64_t un_a = u + a;
              const int b = (int)(un_a % NB);
              if (h == 0 && un_a >= NB) {
                if (!mbar_wait_or_abort(&tempty[b], (uint32_t)(((un_a / NB) - 1) & 1), abortp)) {
                  stop = true;
                  break;
                }
                tc_fence_after();
              }
              const uint32_t d = tbase + (uint32_t)b * 128u;
              if (a == 0) issue_acc<PREC, 0>(d, a_s, b_s, idesc, h == 0);
              if constexpr (NACC > 1) if (a == 1) issue_acc<PREC, (NACC > 1 ? 1 : 0)>(d, a_s, b_s, idesc, h == 0);
              if constexpr (NACC > 2) if (a == 2) issue_acc<PREC, (NACC > 2 ? 2 : 0)>(d, a_s, b_s, idesc, h == 0);
              if (h == SPS - 1) umma_commit(&tfull[b]);
            }
            if (stop) break;
            umma_commit(&empty[s]);
            ++t;
          }
          if (!stop) u += NACC;
        }
        if (stop) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          *abortp = 1;
        }
      }
      // leave no MMA in flight: everything issued before the last commit has completed
      if (t > 0) mbar_wait_bounded(&empty[(t - 1) % NS], (uint32_t)(((t - 1) / NS) & 1));
    }
  }
  } else {
    regs_inc<kEpiRegs>();
    // ---------------- epilogue: warps 4..11; column c = (warp - 4) / 4; TMEM lane = output row
    const int col = (warp - 4) >> 2;
    const int quarter = warp & 3;
    const int lrow = 32 * quarter + lane;
    const int half = lrow >> 6, row = lrow & 63;
    const int child = 2 * half + col;  // warp-uniform
    const int te = threadIdx.x - 128;  // 0..255
    const uint32_t taddr0 = tbase + ((uint32_t)(32 * quarter) << 16) + 64u * (uint32_t)col;
    int64_t u = 0;  // accumulator units drained
    // FP16: one FP32 accumulator per element; BF16 splits: (hi, lo) pairs of
    // adjacent elements packed for the FP32x2 instructions
    constexpr int NHI = NACC == 1 ? 64 : 1, NPK = NACC == 1 ? 1 : 32;
    float hi[NHI];
    uint64_t hi2[NPK], lo2[NPK];
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
      const int64_t Qc = un - batch.ubegin[r], Q = pl.uorder ? pl.uorder[Qc] : pl.ufirst + Qc;
      // children: four output leaves (64-leaves), or the four quadrants of output leaf Q (128-leaves)
      const bool big = pl.tc_bs == 128;
      const int32_t g[4] = {big ? (int32_t)Q : pl.quads[4 * Q], big ? (int32_t)Q : pl.quads[4 * Q + 1],
                            big ? (int32_t)Q : pl.quads[4 * Q + 2], big ? (int32_t)Q : pl.quads[4 * Q + 3]};
#pragma unroll
      for (int i = 0; i < NHI; ++i) hi[i] = 0.f;
#pragma unroll
      for (int i = 0; i < NPK; ++i) hi2[i] = lo2[i] = 0ull;
      const int64_t j1 = pl.qstart[Q + 1];
      int64_t j = pl.qstart[Q];
      float sc_next = j < j1 ? __ldg(&pl.qsteps[j].scale[child]) : 0.f;
      bool failed = false;
      for (; j < j1 && !failed; ++j) {
        const float sc = sc_next;
        if (j + 1 < j1) sc_next = __ldg(&pl.qsteps[j + 1].scale[child]);
        // one accumulator at a time, in the order the MMAs commit them; a
        // runtime loop, so the code holds one copy of each update kind
#pragma unroll 1
        for (int a = 0; a < NACC; ++a) {
          const int b = (int)(u % NB);
          bool ok = true;
          if (lane == 0) ok = mbar_wait_or_abort(&tfull[b], (uint32_t)((u / NB) & 1), abortp);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          ++u;
          if (!ok) {
            // the epilogue still runs the barrier sequence below, then stops together
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abortp = 1;
            failed = true;
            break;
          }
          tc_fence_after();
          bool released = false;
          if (sc != 0.f) {  // this warp's child has a kept product at this k
            const bool exact = a < NACC - 1;  // an exact accumulator: TwoSum into (hi, lo)
            const uint64_t sc2 = ((uint64_t)__float_as_uint(sc) << 32) | __float_as_uint(sc);
            // the slot's 64 columns of this thread's row: four loads in flight
            // at once, one wait; the slot is handed back to the MMAs before
            // the registers are added up
            const uint32_t ta = taddr0 + (uint32_t)b * 128u;
            uint32_t buf[4][16];
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) tmem_ld16_async(ta + 16u * hh, buf[hh]);
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) tmem_wait16(buf[hh]);  // the first waits for all four
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);  // one arrival per warp, after all its lanes' loads
            released = true;
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
              const uint32_t* v = buf[hh];
              if constexpr (NACC == 1) {
#pragma unroll
                for (int i = 0; i < 16; ++i) hi[16 * hh + i] = fmaf(__uint_as_float(v[i]), sc, hi[16 * hh + i]);
              } else if (exact) {
#pragma unroll
                for (int i = 0; i < 8; ++i) two_sum_x2(hi2[8 * hh + i], lo2[8 * hh + i], v[2 * i], v[2 * i + 1], sc2);
              } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) fma_x2(lo2[8 * hh + i], v[2 * i], v[2 * i + 1], sc2);
              }
            }
          }
          if (!released) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
          }
        }
      }
      // output row `row` of leaf g[child], unconverted: each element's 8-byte
      // slot receives its two-float pair (hi, lo) (FP16: (hi, 0)); the finishing
      // pass (tc_finish_kernel) turns the slots into FP64 and takes the leaf
      // norms, so no FP64 instruction runs here, where it would hold up the
      // draining of the accumulators the next quad's MMAs wait for
      const int gl = g[child];
      if (gl >= 0) {
        uint4* out = reinterpret_cast<uint4*>(big ? pl.cpool + (int64_t)gl * 16384 + (64 * half + row) * 128 + 64 * col
                                                  : pl.cpool + (int64_t)gl * 4096 + row * 64);
#pragma unroll
        for (int q = 0; q < 64; q += 2) {
          if constexpr (NACC == 1) {
            out[q >> 1] = make_uint4(__float_as_uint(hi[q]), 0u, __float_as_uint(hi[q + 1]), 0u);
          } else {
            const uint64_t h = hi2[q / 2], l = lo2[q / 2];
            out[q >> 1] = make_uint4((uint32_t)h, (uint32_t)l, (uint32_t)(h >> 32), (uint32_t)(l >> 32));
          }
        }
      }
      if (te == 0) epi_stop = *abortp;
      named_barrier(1, 256);
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
  const size_t smem = QuadLayout<PREC>::SMEM;
  // the register split in the kernel assumes exactly kLaunchRegs per thread at
  // launch: with fewer, the epilogue's increase could never be granted
  cudaFuncAttributes attr;
  CK(cudaFuncGetAttributes(&attr, gemm_quad_kernel<PREC>));
  if (attr.numRegs != (int)kLaunchRegs || attr.maxThreadsPerBlock < kQuadThreads)
    fail(SPAMM_E_CUDA, "tensor-core kernel built with an unexpected register count; refusing to launch");
  CK(cudaFuncSetAttribute(gemm_quad_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned long long* work = ctx->d_scratch + 9;  // quad claim counter
  CK(cudaMemsetAsync(work, 0, sizeof(unsigned long long), ctx->stream));
  gemm_quad_kernel<PREC><<<gemm_grid(ctx, b.nunits), kQuadThreads, smem, ctx->stream>>>(b, work, ctx->d_err);
  CK_LAUNCH("gemm_quad_kernel");
}

// ------------------------------------------------------------------ finish
// Kernel (d) for the tensor-core forms: every 8-byte slot of an output leaf
// holds the two-float pair (hi, lo) the GEMM's epilogue left there (FP16: lo =
// 0); the slot becomes the FP64 value hi + lo (the two conversions are exact
// and done on bit patterns, one FP64 addition rounds the sum; FP16: the exact
// conversion of hi alone), and the leaf's squared Frobenius norm is
// accumulated with one FMA per element in the order of kernel (a) -- lane l
// takes the 16-byte pairs l, l + 32, ..., a butterfly combines the lanes -- so
// the stored norm equals kernel (a) applied to the finished leaf, bit for bit.
// One warp per leaf, 64 leaves per block.  Bound by the FP64 pipe: two FP64
// instructions per element (one for FP16) at two per clock per SM.
constexpr int64_t kFinishLeavesPerBlock = 64;

template <bool TWO>
__global__ void __launch_bounds__(256) tc_finish_kernel(double* __restrict__ pool, int64_t m, int bs,
                                                        double* __restrict__ sq) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)bs * bs;
  const int pairs = bs * bs / 2;
  for (int64_t q0 = (int64_t)blockIdx.x * kFinishLeavesPerBlock; q0 < m;
       q0 += (int64_t)gridDim.x * kFinishLeavesPerBlock)
    for (int64_t q = q0 + warp; q < q0 + kFinishLeavesPerBlock && q < m; q += 8) {
      uint4* leaf = reinterpret_cast<uint4*>(pool + q * e);
      double s = 0.0;
      for (int i = lane; i < pairs; i += 32) {
        const uint4 v = leaf[i];  // (hi, lo) of elements 2i and 2i + 1
        double x0 = __longlong_as_double((long long)f32_to_f64_bits(v.x));
        double x1 = __longlong_as_double((long long)f32_to_f64_bits(v.z));
        if (TWO) {
          x0 = __dadd_rn(x0, __longlong_as_double((long long)f32_to_f64_bits(v.y)));
          x1 = __dadd_rn(x1, __longlong_as_double((long long)f32_to_f64_bits(v.w)));
        }
        s = __fma_rn(x0, x0, s);
        s = __fma_rn(x1, x1, s);
        reinterpret_cast<double2*>(leaf)[i] = make_double2(x0, x1);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) sq[q] = s;
    }
}

void tc_finish(spamm_ctx ctx, spamm_prec prec, double* pool, int64_t nleaves, int bs, double* sq) {
  if (nleaves <= 0) return;
  const int64_t nblk = (nleaves + kFinishLeavesPerBlock - 1) / kFinishLeavesPerBlock;
  const unsigned grid = (unsigned)(nblk < (1ll << 30) ? nblk : (1ll << 30));
  if (prec == SPAMM_PREC_FP16_SCALED)
    tc_finish_kernel<false><<<grid, 256, 0, ctx->stream>>>(pool, nleaves, bs, sq);
  else
    tc_finish_kernel<true><<<grid, 256, 0, ctx->stream>>>(pool, nleaves, bs, sq);
  CK_LAUNCH("tc_finish_kernel");
}

void gemm_tc_batch(spamm_ctx ctx, spamm_prec prec, const BatchDev& b) {
  switch (prec) {
    case SPAMM_PREC_BF16_SPLIT: launch_quads<SPAMM_PREC_BF16_SPLIT>(ctx, b); break;
    case SPAMM_PREC_BF16_SPLIT4: launch_quads<SPAMM_PREC_BF16_SPLIT4>(ctx, b); break;
    case SPAMM_PREC_FP16_SCALED: launch_quads<SPAMM_PREC_FP16_SCALED>(ctx, b); break;
    default: fail(SPAMM_E_INVALID_ARG, "not a tensor-core precision form");
  }
}

}  // namespace spamm
