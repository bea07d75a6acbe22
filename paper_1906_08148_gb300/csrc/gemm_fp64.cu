// gemm_fp64.cu -- kernel (c), FP64 form, with the C-leaf norms of kernel (d)
// fused into its epilogue.
//
// C_ij = sum over the kept k (ascending) of A_ik B_kj (Algorithm 1, "C = AB"
// at the lowest level, run batched over the task list as Section 4.4
// describes).  A work unit is one output leaf, or for 128 x 128 and 256 x 256
// leaves one 64 x 64 sub-tile of an output leaf (4 or 16 per leaf: a leaf
// product of that size takes milliseconds on one SM, so whole leaves would
// leave most SMs idle on small problems).  The units of every plan in a batch
// form one work list; persistent CTAs claim them from an atomic counter (the
// large leaves in order of decreasing kept-product count, so the last claims
// are short).  Every output element is computed by one CTA, so there are no
// atomics on C and the k order is fixed (results do not depend on the schedule
// or on the batch); a sub-tile writes its partial squared norm, and a second
// launch adds a leaf's partials in sub-tile order.  Operand panels are staged
// in shared memory by 1-D TMA bulk copies issued by one warp, double-buffered
// on mbarriers; the product is register-tiled DFMA (FP64 has no tcgen05 kind;
// DFMA measures faster than the FP64 mma.sync path on this part).  A 32 x 32
// leaf is staged whole (one copy per operand); a 64 x 64 output tile in
// K-panels of KP = 32 (A's panel as 64 row segments of 256 bytes, B's as 32
// rows: one copy for 64 x 64 leaves, 32 segments of 512 bytes for larger
// ones), so three CTAs share an SM (64 KB of shared memory each).
#include "internal.cuh"
#include "ptx.cuh"

namespace spamm {

constexpr int kGemmThreads = 256;
// sort key of an output leaf: kUnitKeyMax - its kept-product count (at most
// 2^16, the leaf grid side), so an ascending stable sort puts the longest first
constexpr int kUnitKeyBits = 18;
constexpr int64_t kUnitKeyMax = (int64_t)1 << 17;

template <int BS, int KP, int TILE>
__global__ void __launch_bounds__(kGemmThreads)
    gemm_fp64_kernel(BatchDev batch, unsigned long long* __restrict__ work, int* __restrict__ err) {
  constexpr int LEAF = BS * BS;
  constexpr int NP = BS / KP;                    // K-panels per leaf product
  constexpr int NQ = (BS / TILE) * (BS / TILE);  // work units (sub-tiles) per output leaf
  constexpr int PANEL = TILE * KP;               // doubles in one A panel (and one B panel)
  constexpr uint32_t PANEL_BYTES = PANEL * sizeof(double);
  constexpr int TM = TILE / 16;  // per-thread tile TM x TM: rows tr + 16 i, cols tc + 16 j
  static_assert(BS % TILE == 0 && BS % KP == 0 && TILE % 16 == 0 && KP % 2 == 0, "tile shape");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* sA[2] = {reinterpret_cast<double*>(smem_raw), reinterpret_cast<double*>(smem_raw) + 2 * PANEL};
  double* sB[2] = {reinterpret_cast<double*>(smem_raw) + PANEL, reinterpret_cast<double*>(smem_raw) + 3 * PANEL};
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_u;
  __shared__ int s_abort;
  __shared__ double s_red[kGemmThreads / 32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tr = tid >> 4, tc = tid & 15;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  uint32_t phase[2] = {0u, 0u};
  uint32_t inflight = 0;  // bit s: stage s has a copy that nobody waited for

  for (;;) {
    if (tid == 0) s_u = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t u = s_u;
    if (u >= batch.nunits || s_abort) break;
    const int r = plan_of(batch.ubegin, batch.nplans, u);
    const PlanDev& pl = batch.plans[r];
    const int64_t lu = u - batch.ubegin[r];
    const int64_t li = lu / NQ;  // leaf position in claiming order
    const int sub = (int)(lu - li * NQ);
    const int64_t g = pl.uorder ? pl.uorder[li] : li;
    const int64_t r0 = (int64_t)(sub / (BS / TILE)) * TILE, c0 = (int64_t)(sub % (BS / TILE)) * TILE;
    const int64_t q0 = pl.gstart[g], q1 = pl.gstart[g + 1];
    // step t: task q0 + t / NP, K-panel t % NP; issued by the 32 lanes of
    // warp 0 (lane 0 arms the barrier first)
    auto issue = [&](int64_t t, int s) {
      const int64_t q = q0 + t / NP;
      const int p = (int)(t % NP);
      const double* a = pl.poolA + pl.slotA[pl.ta[q]] * LEAF + r0 * BS + p * KP;
      const double* b = pl.poolB + pl.slotB[pl.tb[q]] * LEAF + (int64_t)p * KP * BS + c0;
      fence_proxy_async_smem();
      if (lane == 0) mbar_arrive_expect_tx(&bar[s], 2 * PANEL_BYTES);
      __syncwarp();
      if constexpr (NP == 1 && TILE == BS) {
        if (lane == 0) bulk_g2s(sA[s], a, PANEL_BYTES, &bar[s]);
      } else {
        for (int row = lane; row < TILE; row += 32)
          bulk_g2s(sA[s] + row * KP, a + (int64_t)row * BS, KP * sizeof(double), &bar[s]);
      }
      if constexpr (TILE == BS) {
        if (lane == 0) bulk_g2s(sB[s], b, PANEL_BYTES, &bar[s]);
      } else {
        for (int row = lane; row < KP; row += 32)
          bulk_g2s(sB[s] + row * TILE, b + (int64_t)row * BS, TILE * sizeof(double), &bar[s]);
      }
    };
    double acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) acc[i][j] = 0.0;
    const int64_t nsteps = (q1 - q0) * NP;
    if (warp == 0 && nsteps > 0) issue(0, 0);
    inflight |= 1u;
    for (int64_t t = 0; t < nsteps; ++t) {
      const int s = (int)(t & 1);
      if (t + 1 < nsteps) {
        if (warp == 0) issue(t + 1, s ^ 1);
        inflight |= 1u << (s ^ 1);
      }
      if (!mbar_wait_bounded(&bar[s], phase[s])) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        s_abort = 1;
      } else {
        phase[s] ^= 1u;
        inflight &= ~(1u << s);
      }
      __syncthreads();
      if (s_abort) break;
      const double* As = sA[s];
      const double* Bs = sB[s];
#pragma unroll 4
      for (int kk = 0; kk < KP; ++kk) {
        double a[TM], b[TM];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[(tr + 16 * i) * KP + kk];
#pragma unroll
        for (int j = 0; j < TM; ++j) b[j] = Bs[kk * TILE + tc + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
    if (nsteps <= 0) inflight &= ~1u;
    if (s_abort) break;
    // epilogue: write the output tile and its squared Frobenius norm (kernel (d))
    double* C = pl.cpool + g * LEAF + r0 * BS + c0;
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        C[(tr + 16 * i) * BS + tc + 16 * j] = acc[i][j];
        s2 = __fma_rn(acc[i][j], acc[i][j], s2);
      }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    if (lane == 0) s_red[warp] = s2;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kGemmThreads / 32; ++w) t += s_red[w];
      if constexpr (NQ == 1)
        pl.csq[g] = t;
      else
        pl.csq_part[g * NQ + sub] = t;
    }
  }
  // leave no bulk copy in flight into this CTA's shared memory
  if (tid == 0) {
    for (int s = 0; s < 2; ++s)
      if (inflight & (1u << s)) mbar_wait_bounded(&bar[s], phase[s]);
  }
  __syncthreads();
}

// Squared norm of each output leaf from its sub-tiles' partials, added in
// sub-tile order; one thread per leaf over every plan of the batch.
__global__ void leaf_norm_from_parts_kernel(BatchDev batch, int nq) {
  const int64_t nleaves = batch.nunits / nq;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nleaves;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = x * nq;
    const int r = plan_of(batch.ubegin, batch.nplans, u);
    const PlanDev& pl = batch.plans[r];
    const int64_t li = (u - batch.ubegin[r]) / nq;  // leaf position in claiming order
    const int64_t g = pl.uorder ? pl.uorder[li] : li;
    double t = 0.0;
    for (int k = 0; k < nq; ++k) t += pl.csq_part[g * nq + k];
    pl.csq[g] = t;
  }
}

template <int BS>
static void launch_fp64(spamm_ctx ctx, const BatchDev& b) {
  constexpr int KP = BS <= 32 ? BS : 32;
  constexpr int TILE = BS <= 64 ? BS : 64;
  auto kern = gemm_fp64_kernel<BS, KP, TILE>;
  const size_t smem = 4 * (size_t)TILE * KP * sizeof(double);
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGemmThreads, smem));
  if (per_sm < 1) per_sm = 1;
  const int sms = ctx->gemm_sm_limit > 0 ? ctx->gemm_sm_limit : ctx->num_sms;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > b.nunits) grid = b.nunits;
  unsigned long long* work = ctx->d_scratch + 8;
  CK(cudaMemsetAsync(work, 0, sizeof(unsigned long long), ctx->stream));
  kern<<<(unsigned)grid, kGemmThreads, smem, ctx->stream>>>(b, work, ctx->d_err);
  CK_LAUNCH("gemm_fp64_kernel");
  constexpr int NQ = (BS / TILE) * (BS / TILE);
  if constexpr (NQ > 1) {
    int64_t g2 = (b.nunits / NQ + 255) / 256;
    if (g2 > 4 * (int64_t)ctx->num_sms) g2 = 4 * (int64_t)ctx->num_sms;
    leaf_norm_from_parts_kernel<<<(unsigned)g2, 256, 0, ctx->stream>>>(b, NQ);
    CK_LAUNCH("leaf_norm_from_parts_kernel");
  }
}

int fp64_units_per_leaf(int bs) { return bs <= 64 ? 1 : (bs / 64) * (bs / 64); }

__global__ void unit_order_keys_kernel(const int64_t* __restrict__ gstart, int64_t ng, uint64_t* __restrict__ keys,
                                       int64_t* __restrict__ vals) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = gstart[g + 1] - gstart[g];
    keys[g] = (uint64_t)(kUnitKeyMax - (c < kUnitKeyMax ? c : kUnitKeyMax));
    vals[g] = g;
  }
}

BufP unit_order_longest(spamm_ctx ctx, const int64_t* start, int64_t n) {
  if (n <= 1) return BufP();
  BufP keys = alloc_n<uint64_t>(ctx, n), vals = alloc_n<int64_t>(ctx, n);
  int64_t grid = (n + 255) / 256;
  if (grid > 4 * (int64_t)ctx->num_sms) grid = 4 * (int64_t)ctx->num_sms;
  unit_order_keys_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(start, n, P<uint64_t>(keys), P<int64_t>(vals));
  CK_LAUNCH("unit_order_keys_kernel");
  radix_sort_pairs(ctx, P<uint64_t>(keys), P<int64_t>(vals), n, kUnitKeyBits);
  return vals;
}

void gemm_fp64_batch(spamm_ctx ctx, int bs, const BatchDev& b) {
  if (b.nunits == 0) return;
  switch (bs) {
    case 32: launch_fp64<32>(ctx, b); break;
    case 64: launch_fp64<64>(ctx, b); break;
    case 128: launch_fp64<128>(ctx, b); break;
    case 256: launch_fp64<256>(ctx, b); break;
    default: fail(SPAMM_E_UNSUPPORTED, "FP64 leaf products are built for bs = 32, 64, 128 and 256");
  }
}

}  // namespace spamm
